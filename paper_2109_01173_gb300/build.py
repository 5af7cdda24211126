"""Build libmofem.so in-tree: nvcc for sm_103a, one object per source, compiled in parallel.

Usage: ``python -m paper_2109_01173_gb300.build`` (also called by ``__graft_entry__.build()``).
Objects go to ``paper_2109_01173_gb300/_build/``; the shared library to
``paper_2109_01173_gb300/libmofem.so``.  Rebuilds only what changed.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmofem.so")
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = shutil.which("nvcc") or os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
          "-diag-suppress", "177"]
SOURCES = ["apply_f32.cu", "apply_f64.cu", "apply_df.cu", "blas1.cu", "gemm_tc.cu", "solver.cu", "noalloc.cu", "dib.cu", "setup.cpp", "capi.cpp", "group.cpp"]
HEADERS = ["internal.h", "apply_impl.cuh", "apply_pcg_f2.cuh", "apply_pcg_push.cuh", os.path.join("..", "..", "include", "mofem.h")]


def _newest_header():
    return max(os.path.getmtime(os.path.join(CSRC, h)) for h in HEADERS)


def _compile(src):
    s = os.path.join(CSRC, src)
    o = os.path.join(BUILD, src + ".o")
    if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), _newest_header()):
        return o, None
    cmd = [NVCC] + ARCH + COMMON + ["-c", s, "-o", o]
    if src.endswith(".cpp"):
        cmd = [NVCC, "-x", "c++"] + COMMON + ["-c", s, "-o", o]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        return o, f"{' '.join(cmd)}\n{r.stdout}\n{r.stderr}"
    return o, None


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        results = list(ex.map(_compile, SOURCES))
    errs = [e for _, e in results if e]
    if errs:
        raise RuntimeError("libmofem build failed:\n" + "\n".join(errs))
    objs = [o for o, _ in results]
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(o) for o in objs):
        return LIB
    cmd = [NVCC] + ARCH + ["-shared", "-o", LIB] + objs + [
        "-L", os.path.join(CUDA, "lib64"), "-lcublas", "-lcusolver",
        "-Xlinker", "-rpath," + os.path.join(CUDA, "lib64"), "-Xlinker", "--no-undefined"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"libmofem link failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
