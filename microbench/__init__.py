"""Measured compute peaks of the GPU (denominators of the benchmark's ALU and tensor rooflines).

``build()`` compiles ``peaks.cu`` (nvcc, sm_103a) into ``_build/libpeaks.so``; ``measure()``
runs its compute-only kernels on the current CUDA device and returns the rates:
FFMA, FFMA2 (packed FP32) and DFMA flop/s, MUFU rsqrt / sin / cos per second, and the tcgen05
TF32 and BF16 MMA rates.  ``python -m microbench`` prints them as JSON.
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "peaks.cu")
_LIB = os.path.join(_HERE, "_build", "libpeaks.so")
KEYS = ("ffma_flops", "ffma2_flops", "dfma_flops", "rsqrt_per_s", "sin_per_s", "cos_per_s", "tcgen05_tf32_flops",
        "tcgen05_bf16_flops", "sm_count", "mma_wait_error")


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def build() -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    cmd = [_nvcc(), "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC", "-o", _LIB, _SRC]
    subprocess.run(cmd, check=True)
    return _LIB


def measure() -> dict:
    """Rates on the current CUDA device (requires a GPU and the built library)."""
    if not os.path.exists(_LIB):
        raise RuntimeError(f"peak microbenchmark not built: {_LIB}")
    L = ctypes.CDLL(_LIB)
    L.peaks_measure.restype = ctypes.c_int
    L.peaks_measure.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    out = (ctypes.c_double * len(KEYS))()
    rc = L.peaks_measure(out, len(KEYS))
    if rc != 0:
        raise RuntimeError("peak microbenchmark failed")
    return {k: float(v) for k, v in zip(KEYS, out)}

