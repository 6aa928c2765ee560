"""In-tree build of libffa.so (CUDA C++ for sm_103a, static CUDA runtime)."""
from __future__ import annotations

import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libffa.so")
# the bounds-checked debug build: same sources and entry points, compiled with FFA_CHECKED
LIB_CHECKED = os.path.join(PKG, "libffa_checked.so")
SOURCES = ["ffa_kernels.cu", "ffa_api.cu", "ffa_noalloc.cu", "ffa_median.cu",
           "ffa_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fPIC,-ffp-contract=off,-O2", "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libffa")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ffa.h"),
                                                                 __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Builds libffa.so (or, with checked=True, libffa_checked.so) if a source is newer;
    returns its path."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    # several processes (one per GPU rank) may call this at once: one builds, the
    # others wait for the lock and then find the library up to date
    import fcntl
    with open(os.path.join(PKG, ".build_checked.lock" if checked else ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not _stale(lib):
                return lib
            return _build(verbose, checked)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def build_all(force: bool = False, verbose: bool = False) -> list[str]:
    """Both libraries, their translation units compiled in parallel."""
    with ThreadPoolExecutor(2) as ex:
        return list(ex.map(lambda c: build(force, verbose, c), (False, True)))


def _build(verbose: bool, checked: bool) -> str:
    cc = nvcc()
    lib = LIB_CHECKED if checked else LIB
    objdir = os.path.join(PKG, "_build_checked" if checked else "_build")
    os.makedirs(objdir, exist_ok=True)
    extra = ["-DFFA_CHECKED"] if checked else []

    def compile_one(src):
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    subprocess.check_call([cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    if "--checked" in sys.argv:
        print(build(force=True, verbose=True, checked=True))
    else:
        print(build(force=True, verbose=True))
