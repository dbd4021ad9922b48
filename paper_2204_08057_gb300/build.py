"""Builds the solver library ``_build/libsylv.so`` in-tree with nvcc for sm_103a.

Usage: ``python -m paper_2204_08057_gb300.build [--verbose-ptxas]``.  Translation units are
compiled in parallel and linked with the static CUDA runtime; no PyTorch headers are involved.
"""

import concurrent.futures as cf
import fcntl
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(BUILD, "libsylv.so")
SOURCES = ["runtime.cu", "setup_kernels.cu", "pcg_f32.cu", "pcg_f64.cu", "noalloc.cu",
           "lanczos.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc")
    if exe is None:
        cand = "/usr/local/cuda/bin/nvcc"
        if os.path.exists(cand):
            exe = cand
    if exe is None:
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsylv")
    return exe


def _flags(verbose_ptxas=False):
    f = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
         "--expt-relaxed-constexpr"] + ARCH
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src, verbose_ptxas):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose_ptxas)
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj, res.stderr


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose_ptxas=False, quiet=True):
    """Compiles and links libsylv.so if any source is newer than it.  Returns its path.
    Processes that build at once (one per rank) take turns on a lock file; a process that
    finds the library fresh once it holds the lock does not rebuild it."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    with open(os.path.join(BUILD, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        try:
            if not force and not _stale():
                return LIB
            return _build_locked(verbose_ptxas, quiet)
        finally:
            fcntl.flock(lock, fcntl.LOCK_UN)


def _build_locked(verbose_ptxas, quiet):
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose_ptxas), SOURCES))
    objs = [r[0] for r in results]
    if not quiet:
        for _, log in results:
            if log:
                sys.stderr.write(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    v = "--verbose-ptxas" in sys.argv
    print(build(force=True, verbose_ptxas=v, quiet=not v))
