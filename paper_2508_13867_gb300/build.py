"""Build libuqlb.so in-tree for sm_103a with nvcc (no cmake; translation units in parallel).

The library is written to ``paper_2508_13867_gb300/_build/libuqlb.so``.  A rebuild happens only
when a source or header is newer than the library (or ``force=True``).
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libuqlb.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["lbm_f64.cu", "lbm_f32.cu", "lbm_f16.cu", "lbm_bf16.cu", "lbm_fx16.cu", "lbm_launch.cu", "plain_f64.cu",
              "project_kernels.cu", "w1_kernels.cu"]
CPP_SOURCES = ["uqlb_host.cpp"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libuqlb")
    return path


def _inputs() -> list[str]:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(INCLUDE, "uqlb.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(src: str, extra: list[str]) -> str:
    obj = os.path.join(OUT_DIR, os.path.basename(src) + f".{os.getpid()}.o")
    cmd = [nvcc(), "-std=c++17", "-O3", "-Xcompiler", "-fPIC", "-I", INCLUDE, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    if "-Xptxas=-v" in extra:
        print(r.stderr)
    return obj


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    """Compile every translation unit and link libuqlb.so; returns its path."""
    if not force and not ptxas_info and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cu_flags = [*ARCH, "-lineinfo", "--expt-relaxed-constexpr"]
    if ptxas_info:
        cu_flags.append("-Xptxas=-v")
    jobs = [(os.path.join(CSRC, f), cu_flags) for f in CU_SOURCES]
    jobs += [(os.path.join(CSRC, f), []) for f in CPP_SOURCES]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        objs = list(ex.map(lambda j: _compile(*j), jobs))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        try:
            os.remove(o)
        except OSError:
            pass
    if r.returncode != 0:
        raise RuntimeError(f"link of libuqlb.so failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


if __name__ == "__main__":
    import sys

    build(force=True, verbose=True, ptxas_info="--ptxas" in sys.argv)
