"""Builds libqx in place (nvcc for sm_103a); no cmake, two translation units in parallel."""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "libqx.so")
# measured FMA rates of the GPU (the roofline of FP64-bound kernels); not libqx
PEAK_LIB = os.path.join(OUT_DIR, "libqxpeak.so")
PEAK_SRC = "qx_peak.cu"
INCLUDE = os.path.join(ROOT, "include")
SOURCES = ["qx_host.cpp", "qx_device.cu", "qx_noalloc.cu", "qx_server.cpp", "qx_adjoint.cpp",
           "qx_kak.cpp"]
HEADERS = ["qx_common.h", "qx_kernels.cuh", "qx_expand_fused.cuh", "qx_clifford_tiles.cuh", "qx_merge_fast.cuh",
           "qx_merge_inplace.cuh", "qx_merge_blocks.cuh", "qx_pauli_rot.cuh", "qx_batch.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    path = os.path.join(cuda, "bin", "nvcc")
    return path if os.path.exists(path) else "nvcc"


def _stale():
    if not os.path.exists(LIB) or not os.path.exists(PEAK_LIB):
        return True
    if os.path.getmtime(PEAK_LIB) < os.path.getmtime(os.path.join(CSRC, PEAK_SRC)):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "qx.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libqx.so if a source is newer than the library; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-I", INCLUDE, "-I", CSRC,
                     "-Xcompiler", "-fPIC,-ffp-contract=off", "-Xptxas", "-v" if verbose else "-O3"]
    objs = []

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + f".{os.getpid()}.o")
        cmd = [nvcc] + common + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    def build_peak():
        if not force and os.path.exists(PEAK_LIB) and (
                os.path.getmtime(PEAK_LIB) >= os.path.getmtime(os.path.join(CSRC, PEAK_SRC))):
            return
        tmp = PEAK_LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared",
                               os.path.join(CSRC, PEAK_SRC), "-o", tmp, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {PEAK_SRC}:\n{r.stderr}")
        os.replace(tmp, PEAK_LIB)

    with ThreadPoolExecutor(len(SOURCES) + 1) as ex:
        peak = ex.submit(build_peak)
        objs = list(ex.map(compile_one, SOURCES))
        peak.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
