"""Build libmfs.so in-tree with nvcc for sm_103a (one -gencode, translation units
compiled in parallel).  Usage: python -m paper_2506_04157_gb300.build"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib")
SOURCES = ["capi.cpp", "mesh_host.cpp", "apply_f32.cu", "apply_f64.cu", "tables.cu", "vec.cu", "noalloc.cu", "mg.cu", "solver.cpp", "wbfbt.cu", "temperature.cu", "batch.cu", "autotune.cpp", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(HERE, "..", "include")]


def nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _compile(src, objdir, verbose, defines=()):
    obj = os.path.join(objdir, os.path.basename(src) + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *[f"-D{d}" for d in defines]]
    if src.endswith(".cpp"):
        cmd += ["-x", "cu"]
    cmd += ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, out_dir=OUT, defines=()):
    """Compile every translation unit and link <out_dir>/libmfs.so; returns its path.
    `defines` are extra preprocessor definitions (tuning knobs such as
    MFS_SWEEP_MINBLOCKS)."""
    objdir = os.path.join(out_dir, "obj")
    os.makedirs(objdir, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        res = list(ex.map(lambda s: _compile(s, objdir, verbose, defines), SOURCES))
    if verbose:
        for _, log in res:
            sys.stderr.write(log)
    so = os.path.join(out_dir, "libmfs.so")
    tmp = so + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *[o for o, _ in res]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, so)
    return so


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
