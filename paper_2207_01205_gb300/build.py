"""Builds the CUDA libraries for sm_103a (in-tree, into ``_build/``):
``libfofse.so``, the product, exporting the C ABI of ``include/fofse.h``, and
``libfofse_probes.so``, the measurement probes of ``include/fofse_probes.h``
that the benchmark uses (no part of the method).

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into its library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libfofse.so")
PROBES_LIB = os.path.join(BUILD, "libfofse_probes.so")
SOURCES = ["fofse_api.cu", "fofse_fwd.cu", "fofse_fwd3.cu", "fofse_ofse.cu", "fofse_bwd.cu",
           "fofse_curve.cu", "fofse_dct.cu", "fofse_volume.cu"]
PROBE_SOURCES = ["fofse_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libfofse.so")
    return exe


def _deps():
    inc = os.path.join(HERE, "..", "include")
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(inc, f) for f in os.listdir(inc)] + [__file__]


def up_to_date() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(PROBES_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBES_LIB))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    extra = extra or []

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [exe, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + len(PROBE_SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES + PROBE_SOURCES))

    def link(lib, parts):
        tmp = lib + f".{os.getpid()}.tmp"
        r = subprocess.run([exe, *ARCH, "-shared", "-o", tmp, *parts], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)

    link(LIB, objs[:len(SOURCES)])
    link(PROBES_LIB, objs[len(SOURCES):])
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "-v" in sys.argv else None))
