"""Build liblbm.so in-tree for sm_103a (nvcc, one translation unit per file,
compiled in parallel).  Usage: python -m paper_1206_0389_gb300.build"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "liblbm.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["update.cu", "update_d3q19_f64.cu", "update_d3q19_f32.cu", "update_d3q19_f16.cu",
           "update_d3q27_f64.cu", "update_d3q27_f32.cu", "update_d3q27_f16.cu",
           "update_walls_d3q19_f64.cu", "update_walls_d3q19_f32.cu", "update_walls_d3q19_f16.cu",
           "update_walls_d3q27_f64.cu", "update_walls_d3q27_f32.cu", "update_walls_d3q27_f16.cu",
           "interface.cu", "util.cu", "api.cu", "plan.cpp", "noalloc.cu", "adjoint.cu", "shard.cu"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found")
    return exe


def _compile(src):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [nvcc(), "-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
               "-Xptxas", "-v", "-c", path, "-o", obj]

    else:
        # no contraction of a*b + c: the planner's geometry (nozzle cells and
        # link fractions) rounds the same on every host
        cmd = [nvcc(), "-std=c++17", "-O2", "-x", "c++", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
               "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose=False):
    """Compile every source and link liblbm.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = OUT + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
