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
