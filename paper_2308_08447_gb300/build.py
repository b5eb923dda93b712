"""Builds libgbdemag.so in-tree for sm_103a (nvcc + g++, translation units in parallel).

    python -m paper_2308_08447_gb300.build          # or: python paper_2308_08447_gb300/build.py

Objects go to paper_2308_08447_gb300/_build/, the library next to this file. A unit is
rebuilt when its source or any header under csrc/ or include/ is newer than its object.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbdemag.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_UNITS = ["gbd_api.cu", "gbd_row.cu", "gbd_row_io.cu", "gbd_row_rk.cu", "gbd_row_bf16.cu", "gbd_row_fp16.cu",
              "gbd_conv.cu", "gbd_conv_bf16.cu", "gbd_conv_fp16.cu", "gbd_ypass.cu", "gbd_mixed_row.cu",
              "gbd_mixed_conv.cu"]
CXX_UNITS = ["gbd_tensor.cpp"]


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _cuda_home(nvcc):
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _headers():
    out = []
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".h", ".cuh")):
                out.append(os.path.join(d, f))
    return out


def _stale(src, obj, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + headers)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout)
    return r.stdout


def build(verbose=False, ptxas_info=False):
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    headers = _headers()
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
    jobs = []
    for u in CUDA_UNITS:
        src, obj = os.path.join(CSRC, u), os.path.join(BUILD, u + ".o")
        if _stale(src, obj, headers) or ptxas_info:
            cmd = [nvcc, "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", *ARCH, *inc,
                   "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp"]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    for u in CXX_UNITS:
        src, obj = os.path.join(CSRC, u), os.path.join(BUILD, u + ".o")
        if _stale(src, obj, headers):
            jobs.append(["g++", "-c", src, "-o", obj, "-O2", "-std=c++17", "-fPIC", "-fopenmp", *inc,
                         "-I" + os.path.join(_cuda_home(nvcc), "include")])
    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        logs = list(ex.map(_run, jobs))
    if verbose or ptxas_info:
        for log in logs:
            if log.strip():
                print(log)
    objs = [os.path.join(BUILD, u + ".o") for u in CUDA_UNITS + CXX_UNITS]
    if jobs or not os.path.exists(LIB):
        _run([nvcc, "-shared", *ARCH, "-o", LIB, *objs, "-Xcompiler", "-fopenmp", "-lgomp", "-lcudart", "-ldl"])
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
