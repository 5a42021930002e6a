"""Builds the in-tree CUDA library libpond.so for sm_103a with nvcc.

The translation units compile in parallel (the step-kernel variants live in their own
units), then one nvcc link makes the shared library."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpond.so")
OBJ = os.path.join(HERE, "_build")
SOURCES = ["pond_api.cu", "pond_v2f.cu", "pond_v2f_learned.cu", "pond_v2d.cu", "pond_v1.cu", "pond_vtube.cu",
           "pond_v3f.cu", "pond_v3d.cu", "pond_veq.cu", "pond_vfused.cu"]
HEADERS = ["pond_core.cuh", "pond_kernels.cuh", "pond_batch.cuh", "pond_launch.cuh", "pond_variants.cuh",
           "pond_tc.cuh", "pond_mlp.cuh", "pond_mlp_train.cuh", "pond_reduce.cuh", "pond_sl.cuh", "pond_sl2.cuh",
           "pond3.cuh", "pond3_launch.cuh", "pond_v3_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC"]


def _newest_input():
    paths = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    paths.append(os.path.join(os.path.dirname(HERE), "include", "pond.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths if os.path.exists(p))


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    tag = "%d" % os.getpid()

    def compile_one(src):
        obj = os.path.join(OBJ, os.path.splitext(src)[0] + "." + tag + ".o")
        cmd = [nvcc, *FLAGS, "-c", "-o", obj, os.path.join(CSRC, src)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, obj, r

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as pool:
        results = list(pool.map(compile_one, SOURCES))
    failed = [(src, r) for src, _, r in results if r.returncode != 0]
    for src, obj, r in results:
        if verbose or r.returncode != 0:
            print(r.stdout, end="")
            print(r.stderr, end="")
    if failed:
        raise subprocess.CalledProcessError(failed[0][1].returncode, "nvcc " + failed[0][0])
    tmp = LIB + "." + tag + ".tmp"
    objs = [obj for _, obj, _ in results]
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    for o in objs:
        os.remove(o)
    os.replace(tmp, LIB)
    return LIB
