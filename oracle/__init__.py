"""FP64 CPU oracle of the correlator (Python side).

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use it; the product path never imports it.

The arithmetic lives in ``corr_oracle.c`` (plain double-precision loops, see
that file for the definitions each function follows, all from Section 2 of
the paper: the correlation formula and the loop nest of Fig. 2). This module
compiles it with gcc, widens inputs exactly to complex128 and reshapes the
outputs. It shares no code with the CUDA path.

Functions with a pin (tests under ``tests/test_oracle_pins.py``):
  * ``correlate``   - brute force on tiny inputs with exact rationals, closed
                      forms, invariants (Hermitian, real non-negative
                      autocorrelations, identical stations, linearity in T,
                      channel independence), exact integers;
  * ``gain_loss``   - brute-force definition on tiny inputs;
  * ``gain_grad``   - central finite differences of ``gain_loss``;
  * ``input_grad``  - central finite differences through ``correlate``;
  * ``reorder``     - element placement built by plain loops from each
                      layout's definition, round trips, composition.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corr_oracle.c")
_LIB = os.path.join(_HERE, "libcorr_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over channels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_correlate.argtypes = [dp, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, dp]
        lib.oracle_gain_loss.argtypes = [dp, dp, dp, ctypes.c_long, ctypes.c_int,
                                         ctypes.c_int, dp, dp]
        lib.oracle_gain_grad.argtypes = [dp, dp, dp, ctypes.c_long, ctypes.c_int,
                                         ctypes.c_int, dp]
        lib.oracle_input_grad.argtypes = [dp, dp, dp, dp, ctypes.c_long, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_int, dp]
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags.c_contiguous and a.dtype in (np.float64, np.complex128)
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def widen(x: np.ndarray, dtype: str) -> np.ndarray:
    """Exact widening to complex128. ``cf32``: complex array ``(...,S,T,P)``;
    ``cf16``/``ci8``: real pairs ``(...,S,T,P,2)``."""
    if dtype == "cf32":
        return np.ascontiguousarray(x, dtype=np.complex128)
    if dtype in ("cf16", "ci8"):
        parts = np.asarray(x).astype(np.float64)
        return np.ascontiguousarray(parts[..., 0] + 1j * parts[..., 1])
    raise ValueError(dtype)


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_threads())


def correlate(x: np.ndarray, dtype: str = "cf32") -> np.ndarray:
    """Visibilities ``(units, B, P, P)`` complex128 of samples
    ``(units, S, T, P)`` (leading axes are flattened into units)."""
    z = widen(x, dtype)
    S, T, P = z.shape[-3:]
    lead = z.shape[:-3]
    units = int(np.prod(lead)) if lead else 1
    B = S * (S + 1) // 2
    out = np.zeros((units, B, P, P), dtype=np.complex128)
    if units and S and T:
        _load().oracle_correlate(_ptr(z), units, S, T, P, _ptr(out))
    return out.reshape(lead + (B, P, P))


def gain_loss(R: np.ndarray, g: np.ndarray, M: np.ndarray):
    """Loss and gain-corrupted visibilities. ``R, M``: ``(units, B, P, P)``;
    ``g``: ``(units, S, P)``. Returns ``(L, V)``."""
    R = np.ascontiguousarray(R, dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    units, S, P = g.shape
    V = np.zeros_like(R)
    L = np.zeros(1)
    _load().oracle_gain_loss(_ptr(R), _ptr(g), _ptr(M), units, S, P, _ptr(V), _ptr(L))
    return float(L[0]), V


def gain_grad(R: np.ndarray, g: np.ndarray, M: np.ndarray) -> np.ndarray:
    """``2 dL/d(conj g)``, shape of ``g``."""
    R = np.ascontiguousarray(R, dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    units, S, P = g.shape
    out = np.zeros_like(g)
    _load().oracle_gain_grad(_ptr(R), _ptr(g), _ptr(M), units, S, P, _ptr(out))
    return out


def input_grad(x: np.ndarray, R: np.ndarray, g: np.ndarray, M: np.ndarray) -> np.ndarray:
    """``2 dL/d(conj x)``, shape of ``x`` (complex ``(units, S, T, P)``)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    R = np.ascontiguousarray(R, dtype=np.complex128)
    M = np.ascontiguousarray(M, dtype=np.complex128)
    g = np.ascontiguousarray(g, dtype=np.complex128)
    units, S, T, P = x.shape
    out = np.zeros_like(x)
    _load().oracle_input_grad(_ptr(x), _ptr(R), _ptr(g), _ptr(M), units, S, T, P, _ptr(out))
    return out


# Axes of one integration in each sample layout (Section 4.4's transposed
# layout keeps all stations of a time step together; Section 7's corner turn
# starts from one receiver's stream of all channels).
LAYOUT_AXES = {"cst": ("c", "s", "t"), "cts": ("c", "t", "s"), "sct": ("s", "c", "t")}


def reorder(x: np.ndarray, from_layout: str, to_layout: str) -> np.ndarray:
    """Samples x[I][three axes of from_layout][...element] rearranged into
    to_layout: element (i, c, s, t) keeps its value and moves to its place in
    the new axis order (a numpy transpose of the three layout axes)."""
    src = LAYOUT_AXES[from_layout]
    dst = LAYOUT_AXES[to_layout]
    perm = [0] + [1 + src.index(a) for a in dst] + list(range(4, x.ndim))
    return np.ascontiguousarray(np.transpose(x, perm))
