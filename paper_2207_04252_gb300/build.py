"""In-tree build of librossbi.so for sm_103a (GB300).

The host runtime and each kernel family are separate translation units,
compiled in parallel to objects under _build/ and linked into one shared
library next to this file.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librossbi.so")
SOURCES = [os.path.join(CSRC, f) for f in
           ("k_stage_full.cu", "k_stage_full_prim.cu", "k_stage_pert_f32.cu", "k_stage_pert_f32_prim.cu",
            "k_stage_pert_f32_gen.cu", "k_stage_pert_f32_gen_prim.cu", "k_stage_pert_f64.cu",
            "k_stage_pert_f64_prim.cu", "k_adjoint.cu", "rossbi.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".cu"))] + \
    [os.path.join(ROOT, "include", "rossbi.h"), os.path.abspath(__file__)]

COMPILE_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-O3", "-lineinfo", "-std=c++17",
    # single-precision division and square root by the hardware approximations
    # (2 ulp); only the FP32 perturbation kernels use float arithmetic
    "-prec-div=false", "-prec-sqrt=false",
    "-Xcompiler", "-fPIC,-ffp-contract=off",
]
LINK_FLAGS = [
    "-gencode", "arch=compute_103a,code=sm_103a",
    "-cudart", "shared",
    "-Xlinker", "-rpath,/usr/local/cuda/lib64",
    "-shared",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in DEPS)


def _obj(src: str) -> str:
    return os.path.join(OBJ, os.path.splitext(os.path.basename(src))[0] + ".o")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    pid = os.getpid()

    def compile_one(src):
        tmp = f"{_obj(src)}.{pid}.tmp.o"
        cmd = [nvcc()] + COMPILE_FLAGS + ["-c", "-o", tmp, src]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.check_call(cmd)
        os.replace(tmp, _obj(src))

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        list(ex.map(compile_one, SOURCES))
    tmp = f"{LIB}.{pid}.tmp"
    cmd = [nvcc()] + LINK_FLAGS + ["-o", tmp] + [_obj(s) for s in SOURCES]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
