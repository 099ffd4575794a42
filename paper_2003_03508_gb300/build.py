"""Build the CUDA library ``libhmm_gb300.so`` in-tree for sm_103a.

Each ``csrc/*.cu`` file is compiled by nvcc in parallel
(``-gencode arch=compute_103a,code=sm_103a``) and linked into one shared
library under ``_build/``. The output name carries a hash of the sources and
flags, so an unchanged tree is not rebuilt.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
INCLUDE = ROOT / "include"

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills", f"-I{INCLUDE}"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found; the CUDA toolkit is required to build the library")


def _sources():
    return sorted(CSRC.glob("*.cu"))


def _digest(extra=()) -> str:
    h = hashlib.sha1()
    for p in sorted(list(CSRC.glob("*.cu")) + list(CSRC.glob("*.cuh")) + list(INCLUDE.glob("*.h"))):
        h.update(p.name.encode())
        h.update(p.read_bytes())
    # flags without the (machine-dependent) include path, so every machine
    # that builds the same sources gets the same library name
    h.update(" ".join(f for f in ARCH + NVCC_FLAGS + list(extra) if not f.startswith("-I")).encode())
    return h.hexdigest()[:12]


def kernel_digest(*names: str) -> str:
    """Hash of the named csrc files, the internal header and the flags: it
    changes exactly when the code of those kernels can have changed."""
    h = hashlib.sha1()
    for n in sorted(set(names) | {"hmm_internal.cuh"}):
        h.update(n.encode())
        h.update((CSRC / n).read_bytes())
    h.update(" ".join(f for f in ARCH + NVCC_FLAGS if not f.startswith("-I")).encode())
    return h.hexdigest()[:12]


def library_path() -> Path:
    return BUILD / f"libhmm_gb300_{_digest()}.so"


def build(verbose: bool = False, force: bool = False, ptxas_verbose: bool = False) -> Path:
    """Compile and link; returns the path of the shared library."""
    BUILD.mkdir(exist_ok=True)
    so = library_path()
    if so.exists() and not force:
        return so
    cc = nvcc()
    tag = so.stem.split("_")[-1]
    objs = []
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(src: Path):
        obj = BUILD / f"{src.stem}_{tag}.o"
        cmd = [cc, *ARCH, *NVCC_FLAGS, *extra, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src.name}:\n{r.stderr}")
        return obj, r.stderr

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        for obj, log in ex.map(compile_one, _sources()):
            objs.append(obj)
            if verbose and log.strip():
                print(log)
    tmp = so.with_suffix(f".tmp{os.getpid()}")
    cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, so)
    for obj in objs:
        obj.unlink(missing_ok=True)
    # drop stale builds
    for old in BUILD.glob("libhmm_gb300_*.so"):
        if old != so:
            old.unlink(missing_ok=True)
    return so


if __name__ == "__main__":
    import sys
    print(build(verbose=True, force="--force" in sys.argv, ptxas_verbose="-v" in sys.argv))
