"""Build libsmnn.so in-tree with nvcc for sm_103a (B300).

smnn.cu (plans, C ABI) and one object per step shape of smnn_shape.cu (the kernels and
launch sequences of that shape) compile in parallel, then link into one shared library."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "build")
LIB = os.path.join(HERE, "libsmnn.so")
MAIN = os.path.join(CSRC, "smnn.cu")
SHAPE = os.path.join(CSRC, "smnn_shape.cu")
# (n_b, R+1, Q) of every built step shape: the SMNN_SHAPES list of smnn_impl.cuh
SHAPES = [(9, 3, 3), (2, 2, 1), (3, 3, 1), (4, 4, 1), (4, 2, 1), (4, 2, 2), (6, 2, 3), (6, 3, 2)]
DEPS = [MAIN, SHAPE] + [os.path.join(CSRC, f) for f in ("smnn_impl.cuh", "smnn_chunk.cuh", "smnn_num.cuh")] + \
    [os.path.join(os.path.dirname(HERE), "include", "smnn.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _units():
    """(source, object, extra flags) of every translation unit."""
    units = [(MAIN, os.path.join(OBJ, "smnn.o"), [])]
    for nb, r1, q in SHAPES:
        units.append((SHAPE, os.path.join(OBJ, f"shape_{nb}_{r1}_{q}.o"),
                      [f"-DSMNN_SHAPE_NB={nb}", f"-DSMNN_SHAPE_R1={r1}", f"-DSMNN_SHAPE_Q={q}"]))
    return units


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile the CUDA sources into libsmnn.so unless it is newer than every source."""
    if not force and os.path.exists(LIB):
        mt = os.path.getmtime(LIB)
        if all(os.path.getmtime(p) <= mt for p in DEPS):
            return LIB
    os.makedirs(OBJ, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose else []

    def compile_one(unit):
        src, obj, flags = unit
        tmp = obj + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc(), *NVCC_FLAGS, *extra, *flags, "-c", "-o", tmp, src])
        os.replace(tmp, obj)
        return obj

    units = _units()
    with ThreadPoolExecutor(max_workers=jobs or min(len(units), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
