"""Build libfempic_env.so in-tree for sm_103a (nvcc + g++, no cmake).

The CUDA translation units and the host mesh builder compile in parallel, then
nvcc links the shared library next to this file.  The same sources compiled
with FEMPIC_BOUNDS_CHECK give the debug build, libfempic_env_debug.so
(every mesh-table index checked before it addresses memory), built
alongside in the same parallel job set.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libfempic_env.so")
DEBUG_LIB = os.path.join(HERE, "libfempic_env_debug.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES_CU = ["fempic_env.cu", "fempic_downshift.cu"]
SOURCES_CPP = ["fempic_mesh.cpp"]
HEADERS = [os.path.join(CSRC, "fempic_internal.h"), os.path.join(INCLUDE, "fempic_env.h"),
           os.path.join(INCLUDE, "fempic_downshift.h")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def _stale() -> bool:
    if not (os.path.exists(LIB) and os.path.exists(DEBUG_LIB)):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(DEBUG_LIB))
    srcs = [os.path.join(CSRC, s) for s in SOURCES_CU + SOURCES_CPP] + HEADERS
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link the library if any source is newer than it."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
    host_flags = ["-fPIC", "-ffp-contract=off", "-fno-fast-math"]
    jobs, objs, dobjs = [], [], []
    for s in SOURCES_CU:
        for flags, suffix, lst in (([], ".o", objs), (["-DFEMPIC_BOUNDS_CHECK"], ".debug.o", dobjs)):
            o = os.path.join(BUILD_DIR, s + suffix)
            cmd = [nvcc, *ARCH, "-lineinfo", *common, *flags, "-Xcompiler", ",".join(host_flags), "-c",
                   os.path.join(CSRC, s), "-o", o]
            jobs.append(cmd)
            lst.append(o)
    for s in SOURCES_CPP:
        o = os.path.join(BUILD_DIR, s + ".o")
        cmd = ["g++", *common, *host_flags, "-c", os.path.join(CSRC, s), "-o", o]
        jobs.append(cmd)
        objs.append(o)
        dobjs.append(o)
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in jobs]
    for c, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(c) + "\n" + out.decode(errors="replace"))
        if verbose and out:
            sys.stdout.write(out.decode(errors="replace"))
    for lib, ob in ((LIB, objs), (DEBUG_LIB, dobjs)):
        tmp = lib + f".tmp{os.getpid()}"
        link = [nvcc, *ARCH, "-shared", "-o", tmp, *ob]
        r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed: " + " ".join(link) + "\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
