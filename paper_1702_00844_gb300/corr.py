"""Thin Python binding of libcorr.so (ctypes), with the same entry points as
include/corr.h. Arguments are marshalled from torch tensors; every step of
the computation runs in the library's CUDA kernels. There is no fallback: if
the library is missing or fails to load, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import torch

from . import build as _build

DTYPES = {"cf32": 0, "cf16": 1, "ci8": 2}
PATHS = {"auto": 0, "fp32": 1, "tensor": 2}
FLAG_GAINS = 0x1
FLAG_NO_AUTOTUNE = 0x2
FLAG_HOST_IO = 0x4
LAYOUTS = {"cst": 0, "cts": 1, "sct": 2}
STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported", 3: "out of memory",
          4: "CUDA error", 5: "timeout"}

_LIB = None


class CorrError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} (status {status})")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int), ("n_pols", ctypes.c_int),
                ("n_channels", ctypes.c_int), ("n_samples", ctypes.c_int),
                ("n_integrations", ctypes.c_int), ("dtype", ctypes.c_int),
                ("path", ctypes.c_int), ("flags", ctypes.c_uint)]


class Subarray(ctypes.Structure):
    _fields_ = [("n_stations", ctypes.c_int), ("n_channels", ctypes.c_int),
                ("n_samples", ctypes.c_int), ("reserved", ctypes.c_int),
                ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p)]


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads the in-tree libcorr.so (building it first if needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run build() first")
        _build.build()
    L = ctypes.CDLL(path)
    vp, ip = ctypes.c_void_p, ctypes.c_int
    L.corr_create.argtypes = [ctypes.POINTER(Desc), ctypes.POINTER(vp)]
    L.corr_correlate.argtypes = [vp, vp, vp, vp]
    L.corr_correlate_batched.argtypes = [vp, ip, ctypes.POINTER(Subarray), vp]
    L.corr_correlate_host.argtypes = [vp, vp, vp, vp]
    L.corr_gain_loss.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.corr_gain_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.corr_destroy.argtypes = [vp]
    L.corr_get_error.argtypes = [vp]
    L.corr_status_string.argtypes = [ip]
    L.corr_status_string.restype = ctypes.c_char_p
    L.corr_last_error_message.argtypes = []
    L.corr_last_error_message.restype = ctypes.c_char_p
    L.corr_tile_cost.argtypes = [ip, ip, ctypes.POINTER(ctypes.c_long),
                                 ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_long)]
    L.corr_tile_variant.argtypes = [vp]
    L.corr_tile_variant.restype = ip
    L.corr_batch_tile_variant.argtypes = [vp]
    L.corr_batch_tile_variant.restype = ip
    L.corr_tile_config.argtypes = [vp, ctypes.POINTER(ip), ctypes.POINTER(ip), ctypes.POINTER(ip),
                                   ctypes.POINTER(ip)]
    L.corr_tile_config.restype = ip
    L.corr_tune_results.argtypes = [vp, ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ctypes.c_float)]
    L.corr_tune_results.restype = ip
    L.corr_set_kernel_events.argtypes = [vp, vp, vp]
    L.corr_set_kernel_events.restype = ip
    L.corr_tc_tiles.argtypes = [ip]
    L.corr_tc_tile_decode.argtypes = [ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.corr_tc_schedule.argtypes = [ip, ip, ip, ip, ctypes.POINTER(ip)]
    L.corr_tc_schedule.restype = ip
    L.corr_fp32_subtiles.argtypes = [ip]
    L.corr_fp32_subtile_decode.argtypes = [ip, ip, ctypes.POINTER(ip), ctypes.POINTER(ip)]
    L.corr_gain_backward_noalloc.argtypes = [ip, ip, ip, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.corr_gain_backward_noalloc.restype = ip
    L.corr_reorder.argtypes = [ip, ip, ip, ip, ip, ip, ip, vp, vp, vp]
    L.corr_reorder.restype = ip
    L.corr_noalloc_scratch_bytes.argtypes = []
    L.corr_noalloc_scratch_bytes.restype = ctypes.c_size_t
    for name in ("corr_create", "corr_correlate", "corr_correlate_host", "corr_correlate_batched", "corr_gain_loss",
                 "corr_gain_backward", "corr_destroy", "corr_get_error"):
        getattr(L, name).restype = ip
    _LIB = L
    return L


def _check(status: int, where: str):
    if status != 0:
        msg = ""
        if _LIB is not None:
            msg = (_LIB.corr_last_error_message() or b"").decode(errors="replace")
        raise CorrError(status, where + (f" [{msg}]" if msg else ""))


def _stream_handle(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    if not t.is_contiguous():
        raise ValueError("contiguous tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def layout_shape(S: int, C: int, T: int, I: int, dtype: str, layout: str):
    """Tensor shape of samples in a layout: [I] + the layout's three axes +
    [2 pols] (+ [re, im] for the f16 and int8 types)."""
    axes = {"cst": (C, S, T), "cts": (C, T, S), "sct": (S, C, T)}[layout]
    base = (I,) + axes + (2,)
    return base if dtype == "cf32" else base + (2,)


def reorder(x: torch.Tensor, S: int, C: int, T: int, I: int, dtype: str, from_layout: str,
            to_layout: str, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """``corr_reorder``: samples ``x`` in layout ``from_layout`` ("cst", "cts" or
    "sct") permuted into ``to_layout`` on the device."""
    L = lib()
    if out is None:
        out = torch.empty(layout_shape(S, C, T, I, dtype, to_layout), dtype=torch_dtype(dtype),
                          device=x.device)
    want = I * C * S * T * 2 * (1 if dtype == "cf32" else 2)
    for t, what in ((x, "samples"), (out, "out")):
        if t.numel() != want or t.dtype != torch_dtype(dtype):
            raise ValueError(f"{what}: expected {want} elements of {torch_dtype(dtype)}")
    _check(L.corr_reorder(S, C, T, I, DTYPES[dtype], LAYOUTS[from_layout], LAYOUTS[to_layout],
                          _ptr(x), _ptr(out), ctypes.c_void_p(_stream_handle(stream))),
           "corr_reorder")
    return out


def n_baselines(S: int) -> int:
    return S * (S + 1) // 2


def input_shape(S: int, C: int, T: int, I: int, dtype: str, n_pols: int = 2):
    """Device tensor shape for samples [I][C][S][T][P pols] of a dtype."""
    base = (I, C, S, T, n_pols)
    return base if dtype == "cf32" else base + (2,)


def torch_dtype(dtype: str):
    return {"cf32": torch.complex64, "cf16": torch.float16, "ci8": torch.int8}[dtype]


class Plan:
    """A correlation plan (``corr_create``) for S stations, C channels, T samples
    per integration and I integrations of samples of type ``dtype``."""

    def __init__(self, n_stations: int, n_channels: int, n_samples: int, n_integrations: int = 1,
                 dtype: str = "cf32", path: str = "auto", flags: int = 0, n_pols: int = 2):
        self.L = lib()
        self.S, self.C, self.T, self.I = n_stations, n_channels, n_samples, n_integrations
        self.dtype = dtype
        self.P = n_pols
        d = Desc(n_stations, n_pols, n_channels, n_samples, n_integrations, DTYPES[dtype],
                 PATHS[path], flags)
        h = ctypes.c_void_p()
        _check(self.L.corr_create(ctypes.byref(d), ctypes.byref(h)), "corr_create")
        self.h = h

    # ------------------------------------------------------------- forward
    def out_shape(self):
        return (self.I, self.C, n_baselines(self.S), self.P, self.P)

    def empty_out(self, device="cuda"):
        if self.dtype == "ci8":
            return torch.empty(self.out_shape() + (2,), dtype=torch.int32, device=device)
        return torch.empty(self.out_shape(), dtype=torch.complex64, device=device)

    def correlate(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
        """Visibilities of samples ``x`` (``corr_correlate``)."""
        if out is None:
            out = self.empty_out(x.device)
        want = self.I * self.C * self.S * self.T * self.P * (1 if self.dtype == "cf32" else 2)
        if x.numel() != want or x.dtype != torch_dtype(self.dtype):
            raise ValueError(f"samples: expected {want} elements of {torch_dtype(self.dtype)}")
        _check(self.L.corr_correlate(self.h, _ptr(x), _ptr(out), _stream_handle(stream)),
               "corr_correlate")
        return out

    def correlate_host(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
        """``corr_correlate_host``: ``x`` and ``out`` are CPU tensors (pin them
        for overlapped copies). Returns ``out``; synchronize the stream before
        reading it."""
        if out is None:
            out = self.empty_out("cpu")
        if x.is_cuda or out.is_cuda or not x.is_contiguous() or not out.is_contiguous():
            raise ValueError("contiguous host tensors expected")
        _check(self.L.corr_correlate_host(self.h, ctypes.c_void_p(x.data_ptr() or None),
                                          ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "corr_correlate_host")
        return out

    def correlate_batched(self, pairs: Sequence[Tuple[torch.Tensor, torch.Tensor]],
                          shapes: Sequence[Tuple[int, int, int]], stream=None):
        """Ragged batch (``corr_correlate_batched``): ``pairs[i] = (x_i, out_i)``
        with ``shapes[i] = (S_i, C_i, T_i)``."""
        arr = (Subarray * len(pairs))()
        for k, ((x, o), (S, C, T)) in enumerate(zip(pairs, shapes)):
            arr[k] = Subarray(S, C, T, 0, x.data_ptr(), o.data_ptr())
        _check(self.L.corr_correlate_batched(self.h, len(pairs), arr, _stream_handle(stream)),
               "corr_correlate_batched")

    # ------------------------------------------------------------- gains
    def gain_loss(self, R, g, M, V=None, loss=None, stream=None):
        if loss is None:
            loss = torch.empty((), dtype=torch.float32, device=R.device)
        _check(self.L.corr_gain_loss(self.h, _ptr(R), _ptr(g), _ptr(M), _ptr(V), _ptr(loss),
                                     _stream_handle(stream)), "corr_gain_loss")
        return loss

    def gain_backward(self, x, g, M, R=None, grad_scale=None, input_grad=True, loss=None,
                      stream=None):
        grad_g = torch.empty_like(g)
        grad_x = torch.empty_like(x) if input_grad else None
        _check(self.L.corr_gain_backward(self.h, _ptr(x), _ptr(g), _ptr(M), _ptr(R),
                                         _ptr(grad_g), _ptr(grad_x), _ptr(loss),
                                         _ptr(grad_scale), _stream_handle(stream)),
               "corr_gain_backward")
        return grad_g, grad_x

    # ------------------------------------------------------------- misc
    def tile_variant(self) -> str:
        v = self.L.corr_tile_variant(self.h)
        return {0: "narrow", 1: "wide", 2: "pair"}.get(v, "fp32")

    def set_kernel_events(self, start=None, stop=None):
        """``corr_set_kernel_events``: record ``start``/``stop``
        (torch.cuda.Event, already created on the device) around the plan's
        main kernel launch in later calls; no arguments turn it off."""
        a = start._as_parameter_ if start is not None else None
        b = stop._as_parameter_ if stop is not None else None
        _check(self.L.corr_set_kernel_events(self.h, a, b), "corr_set_kernel_events")

    def tile_config(self) -> dict:
        """``corr_tile_config``: the tensor-path tile configuration and how it
        was chosen."""
        v, t, l, src = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.L.corr_tile_config(self.h, ctypes.byref(v), ctypes.byref(t), ctypes.byref(l),
                                       ctypes.byref(src)), "corr_tile_config")
        names = {0: "narrow", 1: "wide", 2: "pair"}
        sources = {0: "forced", 1: "rule", 2: "timed", 3: "memory", 4: "file"}
        return {"variant": names[v.value], "tail": names[t.value], "layout": l.value,
                "source": sources[src.value]}

    def tune_results(self, batch: bool = False):
        """``corr_tune_results``: [(variant, tail, layout), ms] of the
        candidates the autotuner timed."""
        n = self.L.corr_tune_results(self.h, int(batch), 0, None, None)
        cfg = (ctypes.c_int * (3 * max(n, 1)))()
        ms = (ctypes.c_float * max(n, 1))()
        self.L.corr_tune_results(self.h, int(batch), n, cfg, ms)
        names = {0: "narrow", 1: "wide", 2: "pair"}
        return [((names[cfg[3 * i]], names[cfg[3 * i + 1]], cfg[3 * i + 2]), ms[i]) for i in range(n)]

    def batch_tile_variant(self) -> Optional[str]:
        """Tile variant of the current ragged batch (None before any)."""
        v = self.L.corr_batch_tile_variant(self.h)
        return {0: "narrow", 1: "wide", 2: "pair"}.get(v)

    def check_error(self):
        _check(self.L.corr_get_error(self.h), "corr_get_error")

    def close(self):
        if getattr(self, "h", None):
            self.L.corr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GainCalibrationLoss(torch.autograd.Function):
    """L(x, g) = sum |g_a conj(g_b) corr(x)_ab - M_ab|^2 with the forward
    correlation and the hand-written adjoint of libcorr (FP32).

    ``x``: complex64 [I][C][S][T][2]; ``g``: complex64 [I][C][S][2];
    ``M``: complex64 [I][C][B][2][2]; ``plan``: a cf32 Plan made with
    FLAG_GAINS. Returns a float32 scalar."""

    @staticmethod
    def forward(ctx, x, g, M, plan):
        x = x.contiguous()
        g = g.contiguous()
        M = M.contiguous()
        R = plan.correlate(x)
        loss = plan.gain_loss(R, g, M)
        ctx.save_for_backward(x, g, M, R)
        ctx.plan = plan
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        x, g, M, R = ctx.saved_tensors
        scale = grad_out.detach().to(torch.float32).contiguous()
        grad_g, grad_x = ctx.plan.gain_backward(
            x, g, M, R=R, grad_scale=scale, input_grad=ctx.needs_input_grad[0])
        return grad_x, (grad_g if ctx.needs_input_grad[1] else None), None, None
