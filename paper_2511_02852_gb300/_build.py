"""In-tree build of the CUDA library (libscwp.so) for sm_103a.

nvcc compiles each CUDA translation unit (in parallel) with
``-gencode arch=compute_103a,code=sm_103a``; the float64 host table code is
compiled by g++; everything is linked into ``_lib/libscwp.so``.  Host code is
compiled with ``-ffp-contract=off`` so the float64 operations that decide
integers are not fused into multiply-adds.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libscwp.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
CU_SOURCES = ["api.cu", "k_particles.cu", "k_fft.cu", "k_synth.cu", "k_synth_tc.cu", "k_layered.cu",
              "noalloc.cu", "k_normals.cu", "k_synth_sat.cu", "k_synth_sat3.cu"]
CXX_SOURCES = ["host_spectrum.cpp"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _digest():
    h = hashlib.sha256()
    for name in sorted(os.listdir(CSRC)) + ["../../include/scwp.h", "../_build.py"]:
        path = os.path.join(CSRC, name)
        if os.path.isfile(path):
            h.update(name.encode())
            with open(path, "rb") as f:
                h.update(f.read())
    import platform
    h.update(platform.machine().encode())
    return h.hexdigest()[:16]


def build(force=False, verbose=False):
    """Compile the library if its sources changed; returns the .so path."""
    os.makedirs(LIBDIR, exist_ok=True)
    stamp = os.path.join(LIBDIR, "libscwp.stamp")
    dig = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == dig:
                return LIB
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in CU_SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
               "-I", INCLUDE, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in CXX_SOURCES:
        obj = os.path.join(objdir, src.replace(".cpp", ".o"))
        cmd = ["g++", "-O2", "-fPIC", "-std=c++17", "-ffp-contract=off", "-I", INCLUDE,
               "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(" ".join(cmd) + "\n" + out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(cmd[-3])
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-lcudart"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(dig)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
