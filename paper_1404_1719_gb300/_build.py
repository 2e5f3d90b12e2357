"""Compiles libvx_rates.so in-tree with nvcc for sm_103a (one -gencode, translation units in parallel)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libvx_rates.so")
SOURCES = ["vx_rates.cu", "vx_mixed_fwd_b2.cu", "vx_mixed_fwd_b3.cu", "vx_mixed_adj_b2.cu", "vx_mixed_adj_b3.cu",
           "vx_mixed_fwd_b2p.cu", "vx_mixed_fwd_b3p.cu", "vx_mixed_adj_b2p.cu", "vx_mixed_adj_b3p.cu",
           "vx_fp64.cu", "vx_btd.cu", "vx_probe.cu", "vx_nes.cu", "vx_abs.cu"]
HEADERS = ["vx_internal.h", "vx_kernel_mixed.cuh", "vx_mixed_inst.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]
# Extra nvcc flags (e.g. -DVX_ADJ_PAIR=1) for tuning experiments; part of the staleness check.
EXTRA = os.environ.get("VX_NVCC_FLAGS", "").split()


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    stamp = LIB + ".flags"
    if not os.path.exists(stamp) or open(stamp).read() != " ".join(EXTRA):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, h)
                                                                  for h in ("vx_rates.h", "vx_btd.h", "vx_probe.h", "vx_nes.h", "vx_eos.h", "vx_abs.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        nvcc = "nvcc"

    def compile_one(src):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [nvcc] + ARCH + FLAGS + EXTRA + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(LIB + ".flags", "w") as f:
        f.write(" ".join(EXTRA))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
