"""Build the zotfs CUDA library (libzotfs.so) in-tree for sm_103a with nvcc.

Translation units compile in parallel: the C ABI, the plain form, the kernel table and one
object per frame-kernel instantiation (frame_variant.cu compiled with -DZOTFS_VARIANT=i).
The result lands in ``paper_2604_02266_gb300/_build/libzotfs.so``.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(BUILD, "libzotfs.so")

N_VARIANTS = 11
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _units():
    units = [("capi.cu", [], "capi.o"), ("plain.cu", [], "plain.o"), ("frame_table.cu", [], "frame_table.o"),
             ("batch.cu", [], "batch.o"), ("big_variant.cu", [], "big_variant.o"),
             ("server.cu", [], "server.o"), ("tune.cu", [], "tune.o"),
             ("cluster_variant.cu", [], "cluster_variant.o"),
             ("big_cluster_variant.cu", [], "big_cluster_variant.o"), ("grid_variant.cu", [], "grid_variant.o"),
             ("mrc.cu", [], "mrc.o")]
    for i in range(N_VARIANTS):
        units.append(("frame_variant.cu", [f"-DZOTFS_VARIANT={i}"], f"frame_v{i}.o"))
    return units


def _sources():
    out = [os.path.join(INCLUDE, "zotfs.h")]
    for f in os.listdir(CSRC):
        if f.endswith((".cu", ".cuh", ".h")):
            out.append(os.path.join(CSRC, f))
    return out


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False, ptxas_info=False, jobs=None):
    """Compile and link libzotfs.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    extra = ["-Xptxas", "-v"] if ptxas_info else []

    def compile_one(u):
        src, defs, obj = u
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, *extra, *defs, "-c", os.path.join(CSRC, src), "-o",
               os.path.join(BUILD, obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    jobs = jobs or min(len(_units()), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, _units()))
    log = []
    for cmd, r in results:
        if verbose or ptxas_info:
            log.append(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    objs = [os.path.join(BUILD, u[2]) for u in _units()]
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]  # cudart linked statically (nvcc default)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    if log:
        sys.stderr.write("\n".join(log))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
