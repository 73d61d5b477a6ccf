"""Builds ``libmeshletcodec.so`` in-tree: host encoder (g++) and sm_103a
kernels (nvcc), compiled in parallel and linked with nvcc.

Usage: ``python -m paper_2404_06359_gb300.build [--force]``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
INCLUDE = os.path.join(ROOT, "include")
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libmeshletcodec.so")

HOST_SOURCES = ["host/meshletize.cpp", "host/strip.cpp", "host/encode.cpp"]
DEVICE_SOURCES = ["device/kernels.cu", "device/cull.cu", "device/cull_views.cu", "device/api_device.cu"]
HEADERS = ["host/host_internal.h", "device/decode_warp.cuh", "device/grab_loop.cuh", "device/cull_common.cuh", "device/kernels.h"]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the codec")


def _cmds():
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in HOST_SOURCES:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        jobs.append(["g++", "-O3", "-std=c++17", "-fPIC", "-ffp-contract=off", "-pthread",
                     "-Wall", "-Wno-unused-function", "-I", INCLUDE, "-c", os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    for s in DEVICE_SOURCES:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        jobs.append([nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "--fmad=false",
                     "-Xcompiler", "-fPIC", "-Xptxas", "-v", "-I", INCLUDE, "-c",
                     os.path.join(CSRC, s), "-o", o])
        objs.append(o)
    link = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs, "-lpthread"]
    return jobs, link


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, s) for s in HOST_SOURCES + DEVICE_SOURCES + HEADERS]
    srcs.append(os.path.join(INCLUDE, "meshlet_codec.h"))
    srcs.append(os.path.abspath(__file__))
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    jobs, link = _cmds()
    log = []

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        for cmd, r in ex.map(run, jobs):
            log.append(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(LIB + ".tmp", LIB)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("\n".join(log))
    if verbose:
        print("\n".join(log))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
