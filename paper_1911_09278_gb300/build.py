"""Build the CUDA library libmace.so in-tree for sm_103a (GB300) with nvcc.

The device code is split over a few translation units (the host side with
the builder and the small kernels, and the ICD sweep kernels once per stored
value type), compiled in parallel and linked into one shared library.
build(debug=True) makes libmace_debug.so with -DMACE_DEBUG: the kernels
check the indices they read from stored data against the buffers they
address and report a failed check as an error instead of making the access
(the binding loads it when MACE_DEBUG=1 is set in the environment)."""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
HDR = os.path.join(os.path.dirname(HERE), "include", "mace.h")
UNITS = ["mace.cu", "sweep_f32.cu", "sweep_bf16.cu", "sweep_f16.cu"]
HEADERS = ["common.cuh", "sweep.cuh"]
LIB = os.path.join(HERE, "libmace.so")
LIB_DEBUG = os.path.join(HERE, "libmace_debug.so")
OBJDIR = os.path.join(HERE, "_build")

NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo",
              "-gencode", "arch=compute_103a,code=sm_103a",
              "-Xcompiler", "-fPIC"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _sources():
    return [os.path.join(CSRC, u) for u in UNITS] + [os.path.join(CSRC, h) for h in HEADERS] + [HDR, __file__]


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    lib = LIB_DEBUG if debug else LIB
    newest = max(os.path.getmtime(p) for p in _sources())
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    os.makedirs(OBJDIR, exist_ok=True)
    tag = "%s%d" % ("d" if debug else "", os.getpid())

    def compile_unit(u):
        obj = os.path.join(OBJDIR, u.replace(".cu", ".%s.o" % tag))
        cmd = [nvcc()] + NVCC_FLAGS + (["-DMACE_DEBUG"] if debug else []) + \
            (["-Xptxas", "-v"] if verbose else []) + ["-c", "-o", obj, os.path.join(CSRC, u)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s" % u)
        return obj

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp." + tag
    subprocess.check_call([nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs)
    for o in objs:
        os.remove(o)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
