"""Build libhcao.so in-tree for sm_103a with nvcc.

hcao_f64.cu is compiled with -fmad=false (FP64 parity mode: no FMA
contraction); host code with -ffp-contract=off.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libhcao.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off,-O2",
          "-I", INC, "--expt-relaxed-constexpr"]
UNITS = {
    "hcao_f64.cu": ["-fmad=false"],
    "hcao_f32.cu": [],
    "hcao_sort.cu": [],
    "hcao_api.cu": [],
    "hcao_rates.cu": [],
}
HEADERS = ["hcao_internal.h", "hcao_kernels.cuh", "hcao_fused.cuh", "hcao_sort.h", "hcao_rates.h"]


def _nvcc() -> str:
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False, extra: list | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INC, "hcao.h")]
    dep_t = max(os.path.getmtime(d) for d in deps)
    objs = []
    nv = _nvcc()
    for src, flags in UNITS.items():
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), dep_t):
            cmd = [nv, *ARCH, *COMMON, *flags, *(extra or []), "-c", s, "-o", o]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
    if force or not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(o) for o in objs):
        cmd = [nv, *ARCH, "-shared", "-o", OUT, *objs, "-Xcompiler", "-fPIC"]
        subprocess.check_call(cmd)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True,
                extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None))
