"""Build the CUDA library libmcsteklov.so in-tree for sm_103a (B300).

The library is plain C ABI (include/mcsteklov.h); nvcc compiles every .cu
file under csrc/ (in parallel, objects under _build/) and links them into one
shared object next to this file.  Walk-deciding
arithmetic needs IEEE operations in the written order, so the library is
compiled without FMA contraction (-fmad=false) and with IEEE division and
square root (nvcc's defaults without --use_fast_math).
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmcsteklov.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-fmad=false", "-Xcompiler", "-fPIC", "-shared",
         "-diag-suppress", "549"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    deps.append(os.path.join(os.path.dirname(HERE), "include", "mcsteklov.h"))
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every csrc/*.cu to an object in parallel (one nvcc each) under
    _build/, then link them into the shared library."""
    if not force and not stale():
        return LIB
    from concurrent.futures import ThreadPoolExecutor
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    compile_flags = [f for f in FLAGS if f != "-shared"]

    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    headers.append(os.path.join(os.path.dirname(HERE), "include", "mcsteklov.h"))
    newest_header = max(os.path.getmtime(h) for h in headers)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        if (not force and os.path.exists(obj) and os.path.getmtime(obj) > os.path.getmtime(src)
                and os.path.getmtime(obj) > newest_header and os.path.getmtime(obj) > os.path.getmtime(__file__)):
            return obj, subprocess.CompletedProcess([], 0, "", "")
        cmd = [nvcc, *ARCH, *compile_flags, "-c", "-o", obj, src]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return obj, r

    with ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 1))) as ex:
        results = list(ex.map(compile_one, sources()))
    for obj, r in results:
        if r.stderr:
            print(r.stderr, file=sys.stderr, end="")
        if r.returncode != 0:
            raise subprocess.CalledProcessError(r.returncode, r.args)
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *[o for o, _ in results], "-lcudart"])
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
