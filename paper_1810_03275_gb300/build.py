"""Build libctrecon.so (the CUDA library behind include/ctrecon.h) in-tree with nvcc
for sm_103a.  Translation units compile in parallel; the result lands in
``paper_1810_03275_gb300/_build/libctrecon.so``."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libctrecon.so")
ROOT = os.path.dirname(HERE)
HEADERS = [os.path.join(ROOT, "include", "ctrecon.h"), os.path.join(SRC, "ctr_internal.cuh")]
# kernels.cu includes radon.cu and fft.cu (one translation unit, see its header)
INCLUDED = {"kernels.cu": ["radon.cu", "fft.cu"]}
UNITS = ["kernels.cu", "solver.cu", "capi.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libctrecon")
    return exe


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, out_dir: str = None) -> str:
    """Compile libctrecon.so (into out_dir, default _build/) and return its path."""
    out = out_dir or OUT
    lib = os.path.join(out, "libctrecon.so")
    os.makedirs(out, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
                    "-I" + os.path.join(ROOT, "include")] + list(extra_flags or [])
    objs = []
    jobs = []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(out, u.replace(".cu", ".o"))
        objs.append(obj)
        deps = [src] + HEADERS + [os.path.join(SRC, x) for x in INCLUDED.get(u, [])]
        if force or _stale(obj, deps):
            jobs.append([nvcc()] + flags + ["-c", src, "-o", obj])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed ({' '.join(cmd)}):\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, flush=True)

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
