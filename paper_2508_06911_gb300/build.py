"""Build liblelbm.so in-tree with nvcc for sm_103a (GB300)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblelbm.so")
# (source, object, defines): the heavy kernels are compiled once per variant so that
# the variants build in parallel
UNITS = [
    ("lelbm_step.cu", "lelbm_step.o", []),
    ("lelbm_api.cu", "lelbm_api.o", []),
    ("lelbm_noalloc.cu", "lelbm_noalloc.o", []),
    ("lelbm_mlp.cu", "lelbm_mlp.o", []),
    ("lelbm_check.cu", "lelbm_check.o", []),
    ("lelbm_3d.cu", "lelbm_3d.o", []),
    ("lelbm_gather.cu", "lelbm_gather.o", []),
    ("lelbm_cell.cu", "lelbm_cell_1d_fp64.o", ["-DLBM_D=1", "-DLBM_PREC=0"]),
    ("lelbm_cell.cu", "lelbm_cell_1d_mixed.o", ["-DLBM_D=1", "-DLBM_PREC=1"]),
    ("lelbm_cell.cu", "lelbm_cell_1d_fp32.o", ["-DLBM_D=1", "-DLBM_PREC=2"]),
    ("lelbm_cell.cu", "lelbm_cell_2d_fp64.o", ["-DLBM_D=2", "-DLBM_PREC=0"]),
    ("lelbm_cell.cu", "lelbm_cell_2d_mixed.o", ["-DLBM_D=2", "-DLBM_PREC=1"]),
    ("lelbm_cell.cu", "lelbm_cell_2d_fp32.o", ["-DLBM_D=2", "-DLBM_PREC=2"]),
    ("lelbm_batch.cu", "lelbm_batch_fp64.o", ["-DLBM_PREC=0"]),
    ("lelbm_batch.cu", "lelbm_batch_mixed.o", ["-DLBM_PREC=1"]),
    ("lelbm_batch.cu", "lelbm_batch_fp32.o", ["-DLBM_PREC=2"]),
]
HEADERS = ["lelbm_internal.h", "lelbm_device.cuh", "lelbm_df.cuh", "lelbm_land.cuh", "lelbm_mlp.cuh", "lelbm_step.cuh",
           os.path.join("..", "..", "include", "lelbm.h")]

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA source (in parallel) and link the shared library; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    for s, o, defs in UNITS:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, o)
        if force or _stale(obj, src):
            cmd = [NVCC, *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        for r in ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
            if verbose:
                print(r.stderr)
    objs = [os.path.join(BUILD, o) for _, o, _ in UNITS]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
