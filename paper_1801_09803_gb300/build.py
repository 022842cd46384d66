"""Build libxc.so in-tree with nvcc for sm_103a (GB300).

The translation units compile in parallel; the shared library links the CUDA
runtime statically.  ``build()`` is a no-op when the library is newer than
every source.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libxc.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libxc")


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hs + [os.path.join(INCLUDE, "xc.h")]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in sources() + headers() + [__file__])


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    with _lock:
        if not force and not stale():
            return LIB
        os.makedirs(BUILD_DIR, exist_ok=True)
        cc = nvcc()
        common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                         "--expt-relaxed-constexpr", "-Xptxas", "-O3"]
        if verbose:
            common += ["-Xptxas", "-v"]
        srcs = sources()
        objs = [os.path.join(BUILD_DIR, os.path.basename(s)[:-3] + ".o") for s in srcs]

        def comp(pair):
            src, obj = pair
            cmd = [cc, "-c", src, "-o", obj] + common
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            return r.stderr

        n = jobs or min(len(srcs), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(n) as ex:
            logs = list(ex.map(comp, zip(srcs, objs)))
        if verbose:
            for s, l in zip(srcs, logs):
                sys.stderr.write(f"== {os.path.basename(s)}\n{l}")
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
