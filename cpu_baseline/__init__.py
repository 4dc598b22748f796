"""Multithreaded FP32 CPU correlator (Section 4.1's design: 2x2 station
tiles, the time loop vectorised, threads over the work), a comparison
baseline for the benchmark. Not the product path and not the oracle.

``build()`` compiles ``corr_cpu.c`` with gcc (-O3, OpenMP; no
machine-specific flags, so it builds the same on x86 and Arm hosts)."""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corr_cpu.c")
_LIB = os.path.join(_HERE, "libcorr_cpu.so")
_lib = None


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        fp = ctypes.POINTER(ctypes.c_float)
        lib.cpu_correlate.argtypes = [fp, ctypes.c_long, ctypes.c_int, ctypes.c_long, fp,
                                      ctypes.c_int]
        lib.cpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    return int(_load().cpu_threads())


def correlate(x: np.ndarray, n_threads: int = 0) -> np.ndarray:
    """Visibilities ``(units, B, 2, 2)`` complex64 of complex64 samples
    ``(..., S, T, 2)`` (leading axes flattened into units)."""
    x = np.ascontiguousarray(x, dtype=np.complex64)
    S, T, P = x.shape[-3:]
    if P != 2:
        raise ValueError("two polarisations expected")
    lead = x.shape[:-3]
    units = int(np.prod(lead)) if lead else 1
    B = S * (S + 1) // 2
    out = np.zeros((units, B, 2, 2), dtype=np.complex64)
    if units and S and T:
        fp = ctypes.POINTER(ctypes.c_float)
        _load().cpu_correlate(x.ctypes.data_as(fp), units, S, T, out.ctypes.data_as(fp), n_threads)
    return out.reshape(lead + (B, 2, 2))
