"""Build of the in-tree DoGIP shared library for sm_103a (GB300).

Steps: compile and run the host table generator (exact rational B and w tables
-> ``_build/tables_gen.h``), compile every CUDA translation unit with nvcc in
parallel, link ``paper_1710_09913_gb300/libdogip.so``.  Rebuilds only when a
source is newer than the library.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libdogip.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-std=c++17", "--expt-relaxed-constexpr", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden"]
UNITS = ["host.cpp", "setup_kernels.cu", "setup_d2.cu", "setup_d3.cu", "vec.cu", "apply_d2.cu",
         "apply_d3a.cu", "apply_d3b.cu", "apply_qp2.cu", "apply_qp3.cu", "apply_gw.cu",
         "apply_hi.cu", "apply_tc.cu", "noalloc.cu", "batch.cu", "cg_small.cu"]

PMAX2, PMAX3 = 4, 3  # orders with compile-time tables (unrolled kernels)
PHI2, PHI3 = 8, 4  # highest orders, served by the run-time-table kernels


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    out = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".cpp"))]
    return out + [os.path.join(INCLUDE, "dogip.h"), os.path.abspath(__file__)]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, force: bool = False) -> str:
    """Build libdogip.so if needed; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    gen = os.path.join(BUILD, "gen_tables")
    _run(["g++", "-O2", "-std=c++17", "-o", gen, os.path.join(CSRC, "gen_tables.cpp")])
    hdr = _run([gen, str(PMAX2), str(PMAX3)])
    with open(os.path.join(BUILD, "tables_gen.h"), "w") as f:
        f.write(hdr)
    hdr = _run([gen, "--hi", str(PMAX2 + 1), str(PHI2), str(PMAX3 + 1), str(PHI3)])
    with open(os.path.join(BUILD, "tables_hi.h"), "w") as f:
        f.write(hdr)
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-I", INCLUDE, "-I", BUILD, "-I", CSRC, "-c",
               os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        log = _run(cmd)
        return obj, log

    workers = min(len(UNITS), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        for obj, log in ex.map(compile_one, UNITS):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    t = __import__("time").time()
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv), f"{__import__('time').time() - t:.1f}s")
