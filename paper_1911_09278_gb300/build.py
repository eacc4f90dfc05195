"""Build the CUDA library libmace.so in-tree for sm_103a (GB300) with nvcc."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "mace.cu")
HDR = os.path.join(os.path.dirname(HERE), "include", "mace.h")
LIB = os.path.join(HERE, "libmace.so")

NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--split-compile", "0",
              "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC", "-shared"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + NVCC_FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-o", tmp, SRC]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
