"""Build the sharpy CUDA library in-tree (nvcc, sm_103a only).

Each translation unit is compiled in parallel, then linked into
_build/libsharpy.so against the shared CUDA runtime.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libsharpy.so")
# (source, extra nvcc flags, object tag): nuts_inst.cu is compiled once per
# (precision, detector count) and loglike_inst.cu once per precision, so the
# kernel variants build in parallel; loglike_staged.cu and
# loglike_staged_split.cu hold the staged likelihood kernel's two paths.
UNITS = [("context.cu", [], "context"), ("loglike.cu", [], "loglike"), ("smc.cu", [], "smc"),
         ("nuts.cu", [], "nuts"), ("run.cu", [], "run"), ("probe.cu", [], "probe"),
         ("batch.cu", [], "batch"), ("recycle.cu", [], "recycle"),
         ("metric.cu", [], "metric"), ("loglike_staged.cu", [], "loglike_staged"),
         ("loglike_staged_split.cu", [], "loglike_staged_split")] + [
    ("nuts_inst.cu", [f"-DSHARPY_NUTS_PREC={p}", f"-DSHARPY_NUTS_NDET={d}"], f"nuts_p{p}_{d}")
    for p in (0, 1, 2) for d in (1, 2, 3)] + [
    ("loglike_inst.cu", [f"-DSHARPY_LL_PREC={p}"], f"loglike_p{p}") for p in (0, 1, 2)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-O3"]


def _nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the sharpy CUDA library cannot be built")
    return p


def _sources():
    return sorted({os.path.join(CSRC, u[0]) for u in UNITS})


def _deps():
    hdr = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return _sources() + hdr + [os.path.join(HERE, "..", "include", "sharpy.h"), __file__]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    objs = []

    def compile_one(unit):
        src, extra, tag = os.path.join(CSRC, unit[0]), unit[1], unit[2]
        obj = os.path.join(OUT, f"{tag}.{os.getpid()}.o")
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + f".tmp{os.getpid()}"
    cudalib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + \
        ["-Xlinker", f"-rpath,{cudalib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
