"""Build libstmg.so in-tree for sm_103a (nvcc for the kernels, g++ for the host setup).

    python -m paper_2502_09159_gb300.builder          # build if sources changed
    python -m paper_2502_09159_gb300.builder --force  # rebuild

Objects go to paper_2502_09159_gb300/_build/, the library to
paper_2502_09159_gb300/libstmg.so.  Translation units compile in parallel; a stamp
of the sources and flags skips up-to-date builds.
"""
from __future__ import annotations

import hashlib
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libstmg.so")

SOURCES = ["setup.cpp", "levels.cpp", "host_api.cpp", "net_api.cpp",
           "k_apply.cu", "k_apply2d.cu", "k_apply2d_reg.cu", "k_mg_persist.cu", "k_vanka.cu", "k_transfer.cu", "k_vec.cu", "k_cells.cu", "k_net.cu", "api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def _flags(cuda):
    inc = ["-I", CSRC, "-I", INCLUDE, "-I", os.path.join(cuda, "include")]
    nv = [os.path.join(cuda, "bin", "nvcc"), "-std=c++17", "-O3", *ARCH, "-lineinfo",
          "-Xcompiler", "-fPIC", "-diag-suppress", "177", *inc]
    cxx = [os.environ.get("CXX", "g++"), "-std=c++17", "-O3", "-fPIC", "-Wall", *inc]
    return nv, cxx


def _stamp(nv, cxx):
    h = hashlib.sha256()
    for f in sorted(os.listdir(CSRC)):
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    for f in sorted(os.listdir(INCLUDE)):
        with open(os.path.join(INCLUDE, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    h.update(" ".join(nv + cxx).encode())
    return h.hexdigest()


def build(force: bool = False, verbose: bool = False) -> str:
    cuda = _cuda_home()
    nv, cxx = _flags(cuda)
    stamp = _stamp(nv, cxx)
    stamp_file = os.path.join(BUILD, "stamp")
    if not force and os.path.exists(LIB) and os.path.exists(stamp_file):
        with open(stamp_file) as f:
            if f.read() == stamp:
                return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = (nv if src.endswith(".cu") else cxx) + ["-c", os.path.join(CSRC, src), "-o", obj]
        p = subprocess.run(cmd, capture_output=True, text=True)
        if p.returncode != 0:
            raise RuntimeError(f"compiling {src} failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
        if verbose and (p.stdout or p.stderr):
            print(p.stdout + p.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nv[0], "-shared", *ARCH, "-o", tmp, *objs, "-lpthread"]
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError(f"linking failed:\n{' '.join(cmd)}\n{p.stdout}\n{p.stderr}")
    os.replace(tmp, LIB)
    with open(stamp_file, "w") as f:
        f.write(stamp)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
