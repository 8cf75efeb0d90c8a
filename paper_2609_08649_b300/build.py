"""Builds the CUDA library in-tree for sm_103a: paper_2609_08649_b300/liblf.so."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "liblf.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo", "-ftz=true",
         "-Xcompiler", "-fPIC", "-shared"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)
                  if f.endswith((".cu", ".cuh", ".h"))) + [os.path.join(HERE, "..", "include", "lf.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


CHECK_LIB = os.path.join(HERE, "liblf_check.so")


def build(force=False, verbose=False, check_bounds=False):
    """Builds liblf.so, or with check_bounds the LF_CHECK_BOUNDS build liblf_check.so (device
    index checks that record LF_DEVERR_BOUNDS; load it with LF_LIBRARY=<path>)."""
    lib = CHECK_LIB if check_bounds else LIB
    if not force and not check_bounds and up_to_date():
        return LIB
    cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose else []) + \
        (["-DLF_CHECK_BOUNDS=1"] if check_bounds else []) + ["-o", lib + ".tmp", os.path.join(CSRC, "lf.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + r.stdout + r.stderr)
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, check_bounds="--check-bounds" in sys.argv))
