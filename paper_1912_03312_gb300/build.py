"""Build the in-tree shared libraries ``librexi.so`` and ``librexi_debug.so``
(sm_103a).

    python -m paper_1912_03312_gb300.build [--force]

The translation units are compiled in parallel (the CUDA engine, the
shared-basis Lanczos kernel, the C ABI, the allocation-free entry point, and the
host-side FCF construction in double-double arithmetic, which needs
floating-point contraction disabled) and linked with the shared CUDA runtime.
``librexi_debug.so`` is the same library with the Lanczos kernel and the C ABI
compiled with REXI_DEBUG (index checks on every access of the kernel; the
binding loads it when the environment sets REXI_DEBUG=1).
"""

from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librexi.so")
DEBUG_LIB = os.path.join(HERE, "librexi_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc():
    p = shutil.which("nvcc") or os.path.join(CUDA_HOME, "bin", "nvcc")
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found (set CUDA_HOME)")
    return p


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "rexi.h")]


def up_to_date():
    if not (os.path.exists(LIB) and os.path.exists(DEBUG_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(DEBUG_LIB))
    return all(os.path.getmtime(s) <= t for s in _sources())


def _link(nvcc, lib, objs):
    tmp = lib + ".tmp"
    link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + [os.path.join(BUILD, o) for o in objs] + \
        ["-Xlinker", "-rpath," + os.path.join(CUDA_HOME, "lib64")]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("librexi link failed:\n" + " ".join(link) + "\n" + r.stdout)
    os.replace(tmp, lib)


def build(force=False, verbose=False):
    """Compile and link both libraries unless they are newer than every source;
    returns the path of librexi.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
    jobs = [
        [nvcc] + ARCH + common + ["-lineinfo", "-c", os.path.join(CSRC, "engine.cu"),
                                  "-o", os.path.join(BUILD, "engine.o")],
        [nvcc] + ARCH + common + ["-c", os.path.join(CSRC, "api.cu"), "-o", os.path.join(BUILD, "api.o")],
        [nvcc] + ARCH + common + ["-c", os.path.join(CSRC, "static_step.cu"),
                                  "-o", os.path.join(BUILD, "static_step.o")],
        [nvcc] + ARCH + common + ["-lineinfo", "-c", os.path.join(CSRC, "lanczos.cu"),
                                  "-o", os.path.join(BUILD, "lanczos.o")],
        [nvcc] + ARCH + common + ["-DREXI_DEBUG", "-c", os.path.join(CSRC, "api.cu"),
                                  "-o", os.path.join(BUILD, "api_dbg.o")],
        [nvcc] + ARCH + common + ["-DREXI_DEBUG", "-lineinfo", "-c", os.path.join(CSRC, "lanczos.cu"),
                                  "-o", os.path.join(BUILD, "lanczos_dbg.o")],
        ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-c", os.path.join(CSRC, "fcf.cpp"),
         "-o", os.path.join(BUILD, "fcf.o")],
    ]
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for j in jobs]
    errors = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append(" ".join(j) + "\n" + out)
        elif verbose and out:
            print(out)
    if errors:
        raise RuntimeError("librexi build failed:\n" + "\n".join(errors))
    _link(nvcc, LIB, ["engine.o", "api.o", "fcf.o", "static_step.o", "lanczos.o"])
    _link(nvcc, DEBUG_LIB, ["engine.o", "api_dbg.o", "fcf.o", "static_step.o", "lanczos_dbg.o"])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
