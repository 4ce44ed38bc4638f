"""Build libmpt.so in-tree with nvcc for sm_103a (GB300).

Translation units are compiled in parallel and linked into
``paper_1908_09301_gb300/libmpt.so``; the build is skipped when the library is
newer than every source.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmpt.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["mpt_step.cu", "mpt_pipe.cu", "mpt_host.cu", "mpt_static.cu", "mpt_adjoint.cu", "int_peak.cu"]
CPP_SOURCES = ["host_parse.cpp"]
HEADERS = ["mpt_kernel.cuh", "mpt_common.cuh", "mpt_divisor.cuh", "host_parse.h"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmpt")
    return p


def _inputs():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "mpt.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"build failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}"]
    jobs, objs = [], []
    for f in CU_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([nv, *ARCH, "-lineinfo", *common, "-Xptxas", "-v", "-c",
                     os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    for f in CPP_SOURCES:
        o = os.path.join(BUILD, f + ".o")
        jobs.append([nv, *common, "-c", os.path.join(CSRC, f), "-o", o])
        objs.append(o)
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_compile, jobs))
    if verbose:
        for lg in logs:
            print(lg)
    tmp = LIB + f".{os.getpid()}.tmp"
    _compile([nv, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
