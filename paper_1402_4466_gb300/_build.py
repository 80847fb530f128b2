"""Build libthr.so in-tree with nvcc for sm_103a (one -gencode, translation
units compiled in parallel, no cmake).  build(checked=True) builds the
checked library, libthr_checked.so (THR_CHECKED defined: every
index-derived access of the query kernels bounds-checked, THR_E_CHECK on a
failure), from the same sources into its own object folder."""
from __future__ import annotations

import fcntl
import glob
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libthr.so")
OUT_CHECKED = os.path.join(PKG, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libthr_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-Wall", f"-I{INCLUDE}"]
_lock = threading.Lock()


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) +
                  glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps() -> list[str]:
    return (sources() + glob.glob(os.path.join(CSRC, "*.cuh")) +
            glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(INCLUDE, "*.h")) + [__file__])


def stale(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _deps())


def _compile(src: str, extra: list[str], out: str) -> str:
    obj = os.path.join(out, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *NVCC_FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if "-v" in extra and r.stderr:
        print(r.stderr)
    return obj


def build(force: bool = False, verbose_ptxas: bool = False, checked: bool = False) -> str:
    """Compile every CUDA/C++ source of the library and link libthr.so (or
    libthr_checked.so)."""
    lib, out = (LIB_CHECKED, OUT_CHECKED) if checked else (LIB, OUT)
    with _lock:
        if not force and not stale(checked):
            return lib
        os.makedirs(out, exist_ok=True)
        # one build at a time across processes too (a process pool whose
        # workers load the library would otherwise compile into the same
        # object folder at once); a process that waited finds it built
        with open(os.path.join(out, ".lock"), "w") as lockf:
            fcntl.flock(lockf, fcntl.LOCK_EX)
            try:
                if not force and not stale(checked):
                    return lib
                return _build_locked(lib, out, checked, verbose_ptxas)
            finally:
                fcntl.flock(lockf, fcntl.LOCK_UN)


def _build_locked(lib: str, out: str, checked: bool, verbose_ptxas: bool) -> str:
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    if checked:
        extra = extra + ["-DTHR_CHECKED"]
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lpthread",
           "-Xlinker", "--no-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
