"""Build libsr.so (the sm_103a kernels and the C-ABI of include/sr.h) in-tree.

The translation units are compiled in parallel with nvcc for sm_103a only,
then linked into paper_2003_12693_gb300/libsr.so.  No PyTorch headers are
involved: the library exposes plain C entry points.
"""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsr.so")
SOURCES = ["sr_kernels.cu", "sr_fft.cu", "sr_fftgen.cu", "sr_api.cu", "sr_noalloc.cu", "sr_net.cu",
           "sr_wfix.cu", "sr_inner.cu", "sr_colrec.cu", "sr_aos.cu", "sr3.cu", "sr_small.cu", "sr_resident.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc() -> str:
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    cand = os.path.join(cuda, "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, s) for s in SOURCES]
    # every header the sources may include
    files += [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".h", ".cuh"))]
    files += [os.path.join(INCLUDE, f) for f in sorted(os.listdir(INCLUDE)) if f.endswith(".h")]
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    with tempfile.TemporaryDirectory(prefix="srbuild") as tmp:
        objs, procs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, src.replace(".cu", ".o"))
            cmd = [nvcc, *ARCH, *FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append(subprocess.Popen(cmd))
            objs.append(obj)
        codes = [p.wait() for p in procs]
        if any(codes):
            raise RuntimeError("nvcc failed while building libsr.so")
        out_tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc, *ARCH, "-shared", "-o", out_tmp, *objs]
        subprocess.run(cmd, check=True)
        os.replace(out_tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
