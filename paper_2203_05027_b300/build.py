"""Build libmfs.so (the CUDA path behind include/mfs.h) in-tree for sm_103a with nvcc."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmfs.so")
SOURCES = ["mfs_solver.cu", "mfs_batch.cu", "mfs_shared.cu", "mfs_mlp.cu", "mfs_static.cu", "mfs_ruiz.cu"]
HEADERS = ["mfs_device.cuh", "mfs_kernels.cuh", "mfs_staged.cuh", "mfs_gemm.cuh", "mfs_alloc.h", "mfs_literal.cuh", "mfs_infeas.cuh", "mfs_host.h", "mfs_measures.h", "mfs_trace.h", "mfs_setup.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


LIB_BOUNDS = os.path.join(HERE, "libmfs_bounds.so")


def build(force=False, verbose=False, extra=(), bounds=False):
    """Compile libmfs.so, or with bounds=True the bounds-checked libmfs_bounds.so (MFS_DEBUG_BOUNDS:
    the single-instance sweep and residual kernels check every gather and padded-entry index)."""
    lib = LIB_BOUNDS if bounds else LIB
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "mfs.h"))
    if not force and not _stale(lib, deps):
        return lib
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    tmp = lib + ".tmp"
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "-Xcompiler", "-pthread", "--expt-relaxed-constexpr",
           *(["-DMFS_DEBUG_BOUNDS"] if bounds else []), *extra,
           "-o", tmp, *[os.path.join(CSRC, f) for f in SOURCES], "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv, bounds="--bounds" in sys.argv)
    print(LIB_BOUNDS if "--bounds" in sys.argv else LIB)
