"""Builds the in-tree shared library ``libstfem.so`` (C ABI of include/stfem.h).

Host setup (C++) is compiled with g++, the CUDA translation unit with nvcc for
sm_103a only; the three objects are compiled in parallel and linked with nvcc
(static CUDA runtime).  Objects go to ``_build/`` next to this file.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstfem.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def commands():
    nvcc = _nvcc()
    inc = "-I" + os.path.join(ROOT, "include")
    cxx = ["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", "-Wall", "-Wno-unused-function", inc, "-c"]
    objs = []
    cmds = []
    cuda_inc = "-I" + os.path.join(os.path.dirname(os.path.dirname(nvcc)), "include")
    for src in ("fem.cpp", "host_api.cpp", "server.cpp"):
        o = os.path.join(OUT, src + ".o")
        cmds.append(cxx[:-1] + [cuda_inc, "-c", os.path.join(CSRC, src), "-o", o])
        objs.append(o)
    o = os.path.join(OUT, "stfem.cu.o")
    cmds.append([nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp", inc,
                 "-c", os.path.join(CSRC, "stfem.cu"), "-o", o])
    objs.append(o)
    link = [nvcc, ARCH, "-shared", "-o", LIB] + objs + ["-lpthread", "-lgomp"]
    return cmds, link


def build(verbose=False):
    os.makedirs(OUT, exist_ok=True)
    cmds, link = commands()
    procs = [subprocess.Popen(c, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for c in cmds]
    failed = []
    for c, p in zip(cmds, procs):
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(c))
    if failed:
        raise RuntimeError("compilation failed:\n" + "\n".join(failed))
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if verbose or r.returncode != 0:
        sys.stdout.write(r.stdout.decode(errors="replace"))
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(link))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
