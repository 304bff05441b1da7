"""Builds libipgc.so (CUDA, sm_103a) in-tree with nvcc; no torch extension."""
from __future__ import annotations

import glob
import os
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libipgc.so")
BUILD_DIR = os.path.join(HERE, "_build")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I", INCLUDE]

_lock = threading.Lock()


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(
        os.path.join(CSRC, "*.cuh")
    ) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every .cu under csrc/ in parallel and link libipgc.so."""
    with _lock:
        if not force and up_to_date():
            return LIB
        os.makedirs(BUILD_DIR, exist_ok=True)
        procs, objs = [], []
        for src in sources():
            obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
            objs.append(obj)
            cmd = [NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        failed = []
        for cmd, pr in procs:
            out, _ = pr.communicate()
            if verbose or pr.returncode != 0:
                print(out.decode(errors="replace"))
            if pr.returncode != 0:
                failed.append(" ".join(cmd))
        if failed:
            raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(
            [NVCC, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lpthread"], check=True
        )
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys

    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
