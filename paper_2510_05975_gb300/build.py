"""Build libcng.so (CUDA for sm_103a) in-tree with nvcc: one object per translation unit,
compiled in parallel, linked into a shared library with the CUDA runtime linked statically."""
from __future__ import annotations

import concurrent.futures as cf
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build", platform.machine())  # host objects differ per machine
LIB = os.path.join(HERE, "libcng.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC) if not f.endswith(".cu")] + [
        os.path.join(HERE, "..", "include", "cng.h")]


def _obj(src: str) -> str:
    return os.path.join(OUT_DIR, os.path.basename(src)[:-3] + ".o")


def _compile(src: str, verbose: bool) -> str:
    obj = _obj(src)
    cmd = ["nvcc", *ARCH, *FLAGS, "-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(obj + ".tmp", obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a and link libcng.so; returns its path.  A
    translation unit is recompiled when its object is older than it or than any header."""
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = sources()
    # a library from another machine (or none) forces a full build
    force = force or not os.path.exists(os.path.join(OUT_DIR, "api.o"))
    hdr = max(os.path.getmtime(p) for p in _headers())

    def stale(src):
        obj = _obj(src)
        return force or verbose or not os.path.exists(obj) or \
            os.path.getmtime(obj) < max(hdr, os.path.getmtime(src))

    todo = [s for s in srcs if stale(s)]
    objs = [_obj(s) for s in srcs]
    if not todo and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(map(os.path.getmtime, objs)):
        return LIB
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(8, len(todo))) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
