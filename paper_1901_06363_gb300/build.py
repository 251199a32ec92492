"""Build libgeodock.so in-tree: every .cu under csrc/ compiled for sm_103a in parallel, then linked.

Also builds libgeodock_checked.so, the same library compiled with GEODOCK_CHECKED: its kernels test the
indices they derive from their inputs and report the first failure as an error of the call instead of
touching memory out of bounds (the binding loads it when GEODOCK_CHECKED=1 is set).

Usage: python -m paper_1901_06363_gb300.build [--verbose-ptxas]
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libgeodock.so")
OUT_CHECKED = os.path.join(HERE, "libgeodock_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off"]


def nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgeodock.so")


# geodock_sweep_inst.cu holds the sweep kernel's launchers for one angle-chunk size; it is compiled once
# per size (one object each, in parallel)
INST = os.path.join(CSRC, "geodock_sweep_inst.cu")
CHUNK_SIZES = (8, 12, 18, 36)


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object name, extra nvcc flags) of every translation unit."""
    out = []
    for src in _sources():
        if src == INST:
            out += [(src, f"geodock_sweep_kc{kc}.o", [f"-DGD_KC={kc}"]) for kc in CHUNK_SIZES]
        else:
            out.append((src, os.path.basename(src) + ".o", []))
    return out


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "geodock.h")]


def up_to_date() -> bool:
    if not (os.path.exists(OUT) and os.path.exists(OUT_CHECKED)):
        return False
    t = min(os.path.getmtime(OUT), os.path.getmtime(OUT_CHECKED))
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, ptxas_verbose: bool = False, jobs: int | None = None) -> str:
    if not force and up_to_date():
        return OUT
    cc = nvcc()
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    # every unit twice: the library and its checked build
    units = [(src, name, flags, "") for src, name, flags in _units()] + \
            [(src, name, flags + ["-DGEODOCK_CHECKED"], "checked_") for src, name, flags in _units()]
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(unit):
        src, name, flags, pre = unit
        obj = os.path.join(objdir, pre + name)
        cmd = [cc, *ARCH, *FLAGS, *flags, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {' '.join(flags)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(jobs) as ex:
        results = list(ex.map(compile_one, units))
    if ptxas_verbose:
        for (_, _, _, pre), (_, log) in zip(units, results):
            if not pre:
                sys.stderr.write(log)
    for out, pre in ((OUT, ""), (OUT_CHECKED, "checked_")):
        objs = [o for (_, _, _, p), (o, _) in zip(units, results) if p == pre]
        tmp = out + f".{os.getpid()}.tmp"
        cmd = [cc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(force=True, ptxas_verbose="--verbose-ptxas" in sys.argv))
