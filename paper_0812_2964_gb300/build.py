"""Build libmcgpu.so in-tree for sm_103a (nvcc; no cmake).

Each translation unit is compiled in parallel, then linked into one shared
library next to this file.  Host code is compiled with -ffp-contract=off.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmcgpu.so")
SOURCES = ["mc_kernels.cu", "mc_api.cu", "mc_inst_reg_a.cu", "mc_inst_reg_b.cu", "mc_inst_reg_c.cu",
           "mc_inst_smem_1.cu", "mc_inst_smem_2.cu", "mc_inst_smem_3.cu", "mc_inst_smem_4.cu",
           "mc_inst_smem_16.cu", "mc_inst_smem_32.cu", "mc_inst_smem_48.cu", "mc_inst_smem_64.cu", "mc_inst_smem_96.cu", "mc_inst_smem_100.cu",
           "mc_inst_smem_128.cu", "mc_inst_rec.cu", "mc_noalloc.cu", "mc_batch.cu", "mc_server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def flags(verbose_ptxas: bool = False) -> list[str]:
    f = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "-I", os.path.join(ROOT, "include")]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _deps() -> list[str]:
    out = [os.path.join(ROOT, "include", n) for n in os.listdir(os.path.join(ROOT, "include"))] + [__file__]
    for n in os.listdir(CSRC):
        out.append(os.path.join(CSRC, n))
    return out


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose_ptxas: bool = False, quiet: bool = True) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nv, *flags(verbose_ptxas), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        for obj, log in ex.map(compile_one, SOURCES):
            objs.append(obj)
            if log.strip() and (verbose_ptxas or not quiet):
                print(log, file=sys.stderr)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv, quiet=False)
    print(LIB)
