"""Build libader.so in-tree with nvcc for sm_103a (no cmake, parallel TUs).

    python -m paper_1806_07984_gb300.build
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libader.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["k_euler3d.cu", "k_euler2d.cu", "k_acoustics3d.cu", "k_acoustics2d.cu", "k_limiter3d.cu", "k_limiter2d.cu",
           "partition.cpp",
           "k_common.cu", "k_noalloc.cu", "k_batch.cu", "api_batch.cpp", "k_adjoint.cu", "k_tc.cu", "api.cpp", "mesh.cpp", "basis.cpp"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libader.so")
    return exe


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if os.path.exists(obj) and os.path.getmtime(obj) >= _newest_input(path):
        return obj
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "-I", CSRC, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _newest_input(path):
    newest = os.path.getmtime(path)
    for f in os.listdir(CSRC):
        if f.endswith((".h", ".cuh")):
            newest = max(newest, os.path.getmtime(os.path.join(CSRC, f)))
    inc = os.path.join(os.path.dirname(HERE), "include", "ader.h")
    if os.path.exists(inc):
        newest = max(newest, os.path.getmtime(inc))
    return newest


def build(verbose=False):
    os.makedirs(BUILD, exist_ok=True)
    workers = min(len(SOURCES), os.cpu_count() or 4)
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(_compile, SOURCES))
    if os.path.exists(OUT) and os.path.getmtime(OUT) >= max(os.path.getmtime(o) for o in objs):
        return OUT
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", OUT + ".tmp", *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(OUT + ".tmp", OUT)
    if verbose:
        print("built", OUT)
    return OUT


if __name__ == "__main__":
    build(verbose=True)
    sys.exit(0)
