"""Build the sm_103a shared library ``lib/libmgrid.so`` in the source tree.

Each translation unit is compiled by its own nvcc process (in parallel) and
then linked; the CUDA runtime is linked statically.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "libmgrid.so")
SOURCES = ["mg_kernels.cu", "mg_short.cu", "mg_regrid.cu", "mg_adjoint.cu", "mg_batch.cu", "mg_capi.cu",
           "mg_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                "-I" + os.path.join(ROOT, "include"), "-I" + SRC]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(cuda, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def compile_commands():
    objs, cmds = [], []
    for s in SOURCES:
        o = os.path.join(LIB_DIR, s.replace(".cu", ".o"))
        objs.append(o)
        cmds.append([_nvcc()] + FLAGS + ["-c", os.path.join(SRC, s), "-o", o])
    link = [_nvcc()] + ARCH + ["-shared", "-o", LIB] + objs
    return cmds, link


def start():
    """Launch the compile processes; returns (procs, link command)."""
    os.makedirs(LIB_DIR, exist_ok=True)
    cmds, link = compile_commands()
    return [subprocess.Popen(c) for c in cmds], link


def finish(procs, link):
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("nvcc failed: " + " ".join(p.args))
    subprocess.run(link, check=True)
    for s in SOURCES:
        o = os.path.join(LIB_DIR, s.replace(".cu", ".o"))
        if os.path.exists(o):
            os.remove(o)


def build():
    finish(*start())
    return LIB
