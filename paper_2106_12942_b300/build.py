"""Build the CUDA library in-tree (sm_103a only).

    python -m paper_2106_12942_b300.build

produces paper_2106_12942_b300/librhseg_b300.so from csrc/*.cu with nvcc.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "librhseg_b300.so")
SRC_MAIN = os.path.join(HERE, "csrc", "rhseg_api.cu")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "--use_fast_math=false"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")) + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
                  + [os.path.join(os.path.dirname(HERE), "include", "rhseg.h")])


def stale() -> bool:
    if not os.path.exists(SO):
        return True
    t = os.path.getmtime(SO)
    return any(os.path.getmtime(s) > t for s in sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return SO
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = SO + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, *[f for f in FLAGS if not f.startswith("--use_fast_math")], "-o", tmp, SRC_MAIN]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
