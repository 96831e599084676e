"""Builds liblbm.so in-tree for sm_103a with nvcc (no CMake, no torch extension).

The translation units are compiled in parallel, then linked into
``paper_2112_05258_gb300/_build/liblbm.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "liblbm.so")
SOURCES = ["lbm_api.cu", "lbm_stream_collide.cu", "lbm_kernels.cu", "lbm_axi.cu", "lbm_ib.cu", "lbm_layout.cu", "lbm_noalloc.cu", "lbm_mlp.cu"]
HEADERS = ["lbm_internal.h", "lbm_kernels.h", "lbm_device.cuh", "lbm_zero_d.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra=None, out_dir: str = BUILD) -> str:
    """Compiles into ``out_dir`` (default: the in-tree _build) and returns the .so path."""
    os.makedirs(out_dir, exist_ok=True)
    so = os.path.join(out_dir, "liblbm.so")
    inc = os.path.join(os.path.dirname(HERE), "include")
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(inc, f) for f in os.listdir(inc)] + [__file__]
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc()] + ARCH + FLAGS + (extra or []) + ["-I", inc, "-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    if jobs or force or _stale(so, objs):
        tmp = so + f".{os.getpid()}.tmp"
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, so)
    return so


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas", action="store_true", help="print register and spill counts")
    ap.add_argument("--define", action="append", default=[], help="NAME=VALUE preprocessor definition")
    ap.add_argument("--out", default=BUILD, help="output directory")
    a = ap.parse_args()
    extra = (["-Xptxas", "-v"] if a.ptxas else []) + [f"-D{d}" for d in a.define]
    print(build(force=a.force, verbose=True, extra=extra, out_dir=os.path.abspath(a.out)))
