"""Compiles the CUDA sources of csrc/ into the in-tree shared library
``paper_2105_00110_gb300/_build/libtc_gb300.so`` for sm_103a (GB300).

nvcc cross-compiles without a GPU.  Translation units are compiled in
parallel and linked with the CUDA runtime statically; the library links
no other CUDA library (CUB is header-only and compiled in).
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libtc_gb300.so")
BUILD_INFO = os.path.join(BUILD, "build_info.json")
# the bounds-checked variant (-DTC_DEBUG_BOUNDS), built on request for tests
DEBUG_BUILD = os.path.join(HERE, "_build_debug")
DEBUG_LIB = os.path.join(DEBUG_BUILD, "libtc_gb300.so")
SOURCES = ["tc_api.cu", "tc_build.cu", "tc_count.cu", "tc_core.cu", "tc_gather.cu", "tc_batch.cu", "tc_noalloc.cu",
           "tc_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]



def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tc.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds the library (debug=True: the bounds-checked variant, in its own
    folder) if a source changed since; returns its path."""
    out_dir, lib = (DEBUG_BUILD, DEBUG_LIB) if debug else (BUILD, LIB)
    defs = ["-DTC_DEBUG_BOUNDS"] if debug else []
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = lib + ".tmp%d" % os.getpid()
    link = [nvcc, *ARCH, "-shared", *objs, "-o", tmp]
    subprocess.check_call(link)
    os.replace(tmp, lib)
    if not debug:
        # the commands this library was made with (read by the build checks)
        with open(BUILD_INFO, "w") as fh:
            json.dump({"compile": [[nvcc, *ARCH, *FLAGS, "-c", src] for src in SOURCES], "link": link[:-2]}, fh)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
