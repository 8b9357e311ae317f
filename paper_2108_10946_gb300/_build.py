"""Builds the CUDA library libfwi_gb300.so in-tree (paper_2108_10946_gb300/_build/) with
nvcc for sm_103a: every translation unit compiled in parallel, then one link."""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libfwi_gb300.so")
# (source, object name, extra flags): the element kernels are one source compiled once per
# KMV element (triangles k = 2..5, tetrahedra k = 2, 3)
UNITS = [("kmv_tab.cpp", "kmv_tab", []), ("api.cu", "api", []), ("kernels.cu", "kernels", [])] + [
    ("inst.cu", f"inst_{d}_{k}", [f"-DKMV_DIM={d}", f"-DKMV_K={k}"])
    for d, k in ((2, 2), (2, 3), (2, 4), (2, 5), (3, 2), (3, 3))]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "fwi.h"))
    return any(os.path.getmtime(p) > t for p in deps)


def build(force=False, verbose=False):
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()

    def compile_unit(unit):
        src, name, extra = unit
        obj = os.path.join(OUT, name + ".o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", os.path.join(SRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{p.stdout}\n{p.stderr}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"link failed:\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB, file=sys.stderr)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
