"""In-tree build of librox.so (CUDA, sm_103a) and of the host test library.

`python -m paper_2510_20870_gb300.build` or `build()` compiles every translation unit
in parallel with nvcc (one -gencode, no cmake) and links them next to this file. The
FP32 Faddeeva constant tables are regenerated first and must match the committed
header (the generator uses only exact arithmetic and numpy's FFT).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "librox.so")
HOST_LIB = os.path.join(HERE, "librox_fadd_host.so")
SOURCES = ["rox_api.cu", "rox_params.cu", "rox_geometry.cu", "rox_voigt.cu", "rox_static.cu", "rox_cia.cu", "rox_probe.cu"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]


def check_tables():
    gen = subprocess.run([sys.executable, os.path.join(CSRC, "gen_faddeeva_tables.py")],
                         check=True, capture_output=True, text=True).stdout
    with open(os.path.join(CSRC, "rox_faddeeva_tables.h")) as f:
        if f.read().strip() != gen.strip():
            raise RuntimeError("rox_faddeeva_tables.h is stale: rerun gen_faddeeva_tables.py")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build_host_lib():
    """CPU build of the FP32 Faddeeva code (for accuracy tests without a GPU)."""
    _run(["g++", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-o", HOST_LIB,
          os.path.join(CSRC, "faddeeva_host.cpp")])
    return HOST_LIB


def build(verbose=False):
    check_tables()
    os.makedirs(BUILD, exist_ok=True)
    objs = []
    cmds = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmds.append([NVCC] + ARCH + FLAGS + ["-Xptxas", "-v", "-c", os.path.join(CSRC, src), "-o", obj])
    with ThreadPoolExecutor(len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    _run([NVCC, "-shared"] + ARCH + ["-o", LIB] + objs)
    build_host_lib()
    if verbose:
        for log in logs:
            sys.stdout.write(log)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
