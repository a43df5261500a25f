"""Build the in-tree CUDA library ``libheff.so`` for sm_103a.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel into
``_build/`` and linked into ``libheff.so`` next to this file.  A source is
recompiled when it, or any header it may include, is newer than its object.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libheff.so")
SOURCES = ["layout.cpp", "plan.cpp", "apply.cu", "tc_gemm.cu", "noalloc.cu", "lanczos.cu", "blockops_tc.cu",
           "blockops.cu", "env.cu", "grad.cu", "svd.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", "-Xptxas", "-v",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "heff.h"))
    return hs


def _stale(src, obj, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + headers)


def _compile(src, verbose):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [_nvcc()] + FLAGS + ARCH + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    log = os.path.join(BUILD, os.path.basename(src) + ".log")
    with open(log, "w") as f:
        f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
    if verbose:
        sys.stdout.write(f"compiled {os.path.basename(src)}\n")
    return obj


def build(verbose=False, force=False):
    """Compile and link ``libheff.so``; returns its path."""
    import platform
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "host")
    host = platform.machine()
    try:
        with open(stamp) as f:
            force = force or f.read().strip() != host     # objects from another machine
    except OSError:
        force = True
    with open(stamp, "w") as f:
        f.write(host)
    headers = _headers()
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    objs = [os.path.join(BUILD, os.path.basename(s) + ".o") for s in srcs]
    todo = [s for s, o in zip(srcs, objs) if force or _stale(s, o, headers)]
    if todo:
        with cf.ThreadPoolExecutor(max_workers=len(todo)) as ex:
            list(ex.map(lambda s: _compile(s, verbose), todo))
    if todo or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [_nvcc(), "-shared"] + ARCH + objs + ["-o", tmp, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
        os.replace(tmp, LIB)
        if verbose:
            sys.stdout.write(f"linked {LIB}\n")
    return LIB


if __name__ == "__main__":
    build(verbose=True, force="--force" in sys.argv)
