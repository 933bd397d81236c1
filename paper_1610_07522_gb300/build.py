"""In-tree build of libsky.so for sm_103a (nvcc, one translation unit per
kernel family, compiled in parallel, then linked as one shared library)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsky.so")
SOURCES = ["sky_api.cu", "hamiltonian.cu", "fields.cu", "gemm.cu", "eigen.cu", "eigen_tridiag.cu", "overlap_noalloc.cu", "tc_ops.cu", "oz_ops.cu", "oz_deriv.cu", "precond.cu", "probe.cu", "td.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _flags(verbose_ptxas=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _compile(src, obj, verbose_ptxas):
    cmd = [nvcc_path(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(verbose_ptxas)
    r = subprocess.run(cmd, capture_output=True, text=True)
    return src, r.returncode, r.stdout + r.stderr


def build(force=False, verbose_ptxas=False, jobs=None):
    """Compile every CUDA source and link ``_lib/libsky.so``.  Skips the work
    when the library is newer than every source and header."""
    os.makedirs(OUT_DIR, exist_ok=True)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "sky.h"), __file__]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    objs = [os.path.join(OUT_DIR, s.replace(".cu", ".o")) for s in SOURCES]
    jobs = jobs or min(len(SOURCES), os.cpu_count() or 1)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for src, rc, log in ex.map(lambda so: _compile(so[0], so[1], verbose_ptxas), zip(SOURCES, objs)):
            logs.append((src, log))
            if rc != 0:
                raise RuntimeError(f"nvcc failed on {src}:\n{log}")
    tmp = LIB + ".tmp"
    cmd = [nvcc_path(), "-shared", "-o", tmp] + objs + ARCH + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB)
    if verbose_ptxas:
        for src, log in logs:
            sys.stdout.write(f"== {src}\n{log}")
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv)
    print(LIB)
