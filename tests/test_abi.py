"""The C-ABI library builds, loads, and exports every symbol the header declares.

CPU-only: nvcc cross-compiles sm_103a without a GPU, and loading the library
needs only the CUDA runtime, so these run anywhere. No kernel is launched.
"""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
HEADERS = sorted((ROOT / "include").glob("*.h"))


def declared_functions():
    names = []
    for h in HEADERS:
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(hmm_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_03508_gb300 import build
    so = build.build()
    try:
        return ctypes.CDLL(str(so))
    except OSError as e:  # no CUDA runtime at all on this host
        pytest.skip(f"cannot dlopen the library here: {e}")


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hmm_create", "hmm_destroy", "hmm_loglik", "hmm_loglik_batched",
                     "hmm_loglik_batched_host", "hmm_status", "hmm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2003_03508_gb300 import api
    assert sorted(api.SIGNATURES) == declared_functions()


def test_opts_default_is_host_only(lib):
    from paper_2003_03508_gb300 import api
    L = api.load_library()
    o = api.hmm_opts()
    L.hmm_opts_default(ctypes.byref(o))
    assert o.precision == api.HMM_PREC_FP32_SIMT and o.init_mode == 0 and o.chunk_len == 0
    assert o.runlen_min == 0 and list(o.reserved) == [0, 0]


def test_opts_struct_matches_the_header():
    # the binding's hmm_opts has the header's fields, in order, as int32
    import re
    from paper_2003_03508_gb300 import api
    text = (ROOT / "include" / "hmm_gb300.h").read_text()
    body = re.search(r"typedef struct \{([^}]*)\} hmm_opts;", text).group(1)
    fields = re.findall(r"int32_t\s+(\w+)(?:\[(\d+)\])?;", body)
    want = [(n, int(c) if c else 1) for n, c in fields]
    got = [(n, getattr(t, "_length_", 1)) for n, t in api.hmm_opts._fields_]
    assert got == want
    assert ctypes.sizeof(api.hmm_opts) == 4 * sum(c for _, c in want)


def test_host_argument_checks_without_gpu(lib):
    # a NULL context is rejected before any CUDA call
    from paper_2003_03508_gb300 import api
    L = api.load_library()
    assert L.hmm_loglik_batched(None, 1, 4, None, None, None, None, None, 1, None, None, None,
                                None, None, None) == api.HMM_EINVAL
    assert L.hmm_status(None, None) == api.HMM_EINVAL
    assert L.hmm_destroy(None) == api.HMM_OK


C_CLIENT = r"""
#include <stdio.h>
#include "hmm_gb300.h"

int main(void) {
    hmm_opts o;
    hmm_prior pr;
    int32_t cand[32], n = 0;
    hmm_opts_default(&o);
    hmm_prior_default(&pr, 16);
    if (hmm_tune_candidates(HMM_PREC_TF32, 256, 32, (1 << 20) - 1, 152, cand, 32, &n) != HMM_OK) return 2;
    printf("%d %d %d %d\n", o.precision, o.chunk_len, o.renorm_every, (int)hmm_theta_dim(16));
    printf("%.6f %.6f %.6f\n", pr.alpha_P, pr.iw_df, pr.box[1]);
    printf("%d", (int)hmm_default_chunk_len(HMM_PREC_TF32, 256, 32, (1 << 20) - 1, 152));
    for (int i = 0; i < n; ++i) printf(" %d", cand[i]);
    printf("\n");
    /* no context: rejected before any device call */
    printf("%d %d\n", hmm_loglik(NULL, NULL, NULL, NULL, NULL, NULL), hmm_destroy(NULL));
    return 0;
}
"""


def test_plain_c_client(lib, tmp_path):
    """The header is plain C99: a C program includes it, links the library
    (no torch, no C++), and its host-only calls agree with the binding."""
    import shutil
    import subprocess
    from paper_2003_03508_gb300 import api, build
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    so = build.build()
    cuda_lib = Path(build.nvcc()).resolve().parent.parent / "lib64"
    if not any(cuda_lib.glob("libcudart.so*")):
        pytest.skip(f"no libcudart under {cuda_lib}")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", f"-I{ROOT / 'include'}",
                        str(src), "-o", str(exe), str(so), f"-L{cuda_lib}", "-lcudart",
                        f"-Wl,-rpath,{so.parent}:{cuda_lib}"], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    l1, l2, l3, l4 = out.stdout.strip().splitlines()
    assert l1.split() == [str(api.HMM_PREC_FP32_SIMT), "0", "0", str(api.theta_dim(16))]
    a, df, x1 = map(float, l2.split())
    assert abs(a - 0.01) < 1e-7 and df == 16.0 and x1 == 300.0
    vals = [int(v) for v in l3.split()]
    assert vals[0] == api.default_chunk_len("tf32", 256, 32, (1 << 20) - 1, 152)
    assert vals[1:] == api.tune_candidates("tf32", 256, 32, (1 << 20) - 1, 152)
    assert l4.split() == [str(api.HMM_EINVAL), str(api.HMM_OK)]
