"""Builds libnavixgb.so in-tree for sm_103a (nvcc, one -gencode, -lineinfo).

The translation units compile in parallel and link into
``paper_2407_19396_gb300/_build/libnavixgb.so``; nothing is installed.  The
same sources built with ``-DNX_DEBUG`` (explicit bounds checks before grid
writes and output stores, recorded in the device error word) link into
``_build/libnavixgb_debug.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnavixgb.so")
DEBUG_LIB = os.path.join(BUILD, "libnavixgb_debug.so")
SOURCES = ["nx_kernels.cu", "nx_kernels_full.cu", "nx_capi.cu", "nx_static.cu", "nx_server.cu", "nx_lean_g1.cu",
           "nx_lean_g4.cu", "nx_lean_g8.cu", "nx_lean_g16.cu", "nx_lean_g32.cu", "nx_lean_pol.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libnavixgb")
    return p


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "navixgb.h")]
    return max(os.path.getmtime(f) for f in files)


def _variants(debug: bool):
    out = [(LIB, os.path.join(BUILD, "release"), [])]
    if debug:
        out.append((DEBUG_LIB, os.path.join(BUILD, "debug"), ["-DNX_DEBUG"]))
    return out


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compiles and links the library (and, with debug=True, its NX_DEBUG
    variant); up-to-date libraries are left alone.  Returns the release path."""
    os.makedirs(BUILD, exist_ok=True)
    newest = _deps()
    todo = [v for v in _variants(debug) if force or not os.path.exists(v[0]) or os.path.getmtime(v[0]) < newest]
    if not todo:
        return LIB
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                     "-I", CSRC]
    jobs = []
    for lib, odir, defs in todo:
        os.makedirs(odir, exist_ok=True)
        for src in SOURCES:
            jobs.append((src, [cc] + common + defs + ["-c", os.path.join(CSRC, src), "-o",
                                                      os.path.join(odir, src.replace(".cu", ".o"))]))

    def compile_one(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)

    with cf.ThreadPoolExecutor(min(len(jobs), max(os.cpu_count() or 1, len(SOURCES)))) as ex:
        list(ex.map(compile_one, jobs))
    for lib, odir, _ in todo:
        tmp = lib + f".tmp{os.getpid()}"
        objs = [os.path.join(odir, s.replace(".cu", ".o")) for s in SOURCES]
        r = subprocess.run([cc] + ARCH + ["-shared", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True, debug=True))
