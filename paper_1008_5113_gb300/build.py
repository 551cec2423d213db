"""In-tree build of the CUDA library ``libvmc.so`` for sm_103a (nvcc, no cmake).

The translation units (the engine's kernels in FP64 and in FP32, the precision-independent
launch entry points; C ABI + host layout; the allocation-free entry point; the dense
reference engine) compile in parallel and are linked into
``paper_1008_5113_gb300/libvmc.so`` next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libvmc.so")
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["vmc_engine_f64.cu", "vmc_engine_f32.cu", "vmc_engine.cu", "vmc_capi.cu", "vmc_noalloc.cu", "vmc_dense.cu"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvmc.so")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "vmc.h"))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def build_library(force: bool = False, verbose: bool = False) -> str:
    """Compile libvmc.so if any source is newer; returns its path."""
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *GENCODE, "-I", os.path.join(ROOT, "include")]
    with tempfile.TemporaryDirectory(prefix="vmcbuild") as tmp:
        procs, objs = [], []
        for src in SOURCES:
            obj = os.path.join(tmp, src + ".o")
            objs.append(obj)
            cmd = [nvcc, *common, "-c", os.path.join(CSRC, src), "-o", obj]
            if verbose:
                print(" ".join(cmd), flush=True)
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        for src, p in procs:
            out, _ = p.communicate()
            if p.returncode != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{out.decode(errors='replace')}")
        tmp_lib = os.path.join(tmp, "libvmc.so")
        subprocess.run([nvcc, "-shared", *GENCODE, *objs, "-o", tmp_lib], check=True)
        shutil.copy2(tmp_lib, LIB + ".tmp")
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force=True, verbose=True))
