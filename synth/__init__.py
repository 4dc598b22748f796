"""Seeded synthetic inputs for the correlator workloads.

This module is shared by the FP64 oracle tests and by the CUDA path's tests
and benchmark. It only draws and lays out samples; it holds none of the
correlator's arithmetic (no products, sums or conjugates of samples).

Layouts follow the problem statement of Section 2 (Fig. 2): samples are
indexed ``[channel][station][time][polarisation]`` with real and imaginary
parts interleaved. Several integrations are stacked in front of the channel
axis, ``[integration][channel][station][time][pol]``.

Representations (numpy, host side):
  * ``cf32`` -> ``np.complex64`` array of shape ``(..., S, T, P)``;
  * ``cf16`` -> ``np.float16`` array of shape ``(..., S, T, P, 2)``;
  * ``ci8``  -> ``np.int8`` array of shape ``(..., S, T, P, 2)``.

The workloads (base seed 1702844, workload k uses seed 1702844 + k):
  1. tiny FP32: S=8, P=2, C=16, T=256, N(0,1) parts;
  2. production FP32: S=64, C=256, T=768, 10 integrations, N(0,1) noise plus a
     point source common to all stations (amplitude 0.1, a per-station phase
     ramp across channels);
  3. precision: S=256, C=480, T=1024, complex int8 from N(0, 32^2) rounded and
     clipped to [-127, 127]; the same values cast to FP16 for the FP16 path;
  4. batching: 32 sub-arrays, S ~ U{16..576}, C ~ U{64..512},
     T ~ U{256..4096} in steps of 128, complex FP16 N(0,1);
  5. differentiation: S=64, C=64, T=1024, complex64 N(0,1), gains
     1 + N(0, 0.1^2) (complex), model visibilities of a 3-point-source sky.
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1702844
P = 2  # X and Y polarisations (Section 2)


def rng(k: int, sub: int = 0) -> np.random.Generator:
    """PCG64 generator for workload ``k`` (and an optional sub-stream)."""
    return np.random.Generator(np.random.PCG64([BASE_SEED + k, sub]))


# ---------------------------------------------------------------- primitives
def complex_normal(g: np.random.Generator, shape, sigma: float = 1.0) -> np.ndarray:
    """complex64 array whose real and imaginary parts are i.i.d. N(0, sigma^2)."""
    re = g.standard_normal(shape, dtype=np.float32)
    im = g.standard_normal(shape, dtype=np.float32)
    out = np.empty(shape, dtype=np.complex64)
    out.real = re * sigma
    out.imag = im * sigma
    return out


def to_cf16(z: np.ndarray) -> np.ndarray:
    """complex -> float16 pairs ``(..., 2)`` (round to nearest)."""
    out = np.empty(z.shape + (2,), dtype=np.float16)
    out[..., 0] = z.real.astype(np.float16)
    out[..., 1] = z.imag.astype(np.float16)
    return out


def int8_normal(g: np.random.Generator, shape, sigma: float = 32.0) -> np.ndarray:
    """int8 pairs ``(..., 2)`` from N(0, sigma^2), rounded and clipped to +-127."""
    v = g.standard_normal(shape + (2,), dtype=np.float32) * np.float32(sigma)
    return np.clip(np.rint(v), -127, 127).astype(np.int8)


def int8_as_cf16(x: np.ndarray) -> np.ndarray:
    """Exact cast of int8 pairs to float16 pairs (|v| <= 128 is representable)."""
    return x.astype(np.float16)


# ------------------------------------------------------------------ workloads
def tiny(seed_offset: int = 1):
    """Workload 1: S=8, P=2, C=16, T=256, complex64 N(0,1)."""
    S, C, T = 8, 16, 256
    x = complex_normal(rng(seed_offset), (C, S, T, P))
    return dict(x=x, S=S, C=C, T=T, I=1, dtype="cf32")


def point_source_signal(g: np.random.Generator, C: int, S: int, T: int,
                        amp: float = 0.1) -> np.ndarray:
    """A sky signal seen by every station and both polarisations.

    ``a[c, t]`` is complex N(0,1) (one draw shared by all stations) and each
    station sees it with a phase ``2*pi*c*d_s/C`` that ramps across channels
    (``d_s`` uniform in [0, S)). Returns complex64 ``(C, S, T, P)``.
    """
    a = complex_normal(g, (C, 1, T, 1))
    d = g.uniform(0.0, float(S), size=S)
    c = np.arange(C, dtype=np.float64)[:, None]
    phase = np.exp(2j * np.pi * c * d[None, :] / C).astype(np.complex64)  # (C,S)
    return (amp * a * phase[:, :, None, None]).astype(np.complex64)


def production(n_integrations: int = 10, C: int = 256, S: int = 64, T: int = 768,
               seed_offset: int = 2):
    """Workload 2: noise plus a common point source, several integrations."""
    out = np.empty((n_integrations, C, S, T, P), dtype=np.complex64)
    for i in range(n_integrations):
        g = rng(seed_offset, i)
        out[i] = complex_normal(g, (C, S, T, P)) + point_source_signal(g, C, S, T)
    return dict(x=out, S=S, C=C, T=T, I=n_integrations, dtype="cf32")


def precision(C: int = 480, S: int = 256, T: int = 1024, seed_offset: int = 3,
              channels=None):
    """Workload 3: complex int8 from N(0, 32^2), shape ``(C, S, T, P, 2)``.

    The FP16 path of this workload correlates the same values cast to FP16
    (``int8_as_cf16``), which is exact.

    ``channels`` selects a subset of channel indices; each channel is drawn
    from its own sub-stream, so a subset equals the matching slice of the
    full array.
    """
    chans = range(C) if channels is None else channels
    x = np.empty((len(chans), S, T, P, 2), dtype=np.int8)
    for k, c in enumerate(chans):
        x[k] = int8_normal(rng(seed_offset, c), (S, T, P))
    return dict(x=x, S=S, C=len(chans), T=T, I=1, dtype="ci8")


def batching_shapes(n_sub: int = 32, seed_offset: int = 4):
    """Workload 4 shapes: list of (S, C, T)."""
    g = rng(seed_offset)
    S = g.integers(16, 576, size=n_sub, endpoint=True)
    C = g.integers(64, 512, size=n_sub, endpoint=True)
    T = 128 * g.integers(2, 32, size=n_sub, endpoint=True)
    return [(int(s), int(c), int(t)) for s, c, t in zip(S, C, T)]


def batching_subarray(S: int, C: int, T: int, index: int, seed_offset: int = 4):
    """Host data of one ragged sub-array: complex FP16 N(0,1), ``(C,S,T,P,2)``."""
    g = rng(seed_offset, 1000 + index)
    return to_cf16(complex_normal(g, (C, S, T, P)))


def batching_subarray_device(S: int, C: int, T: int, index: int, device,
                             seed_offset: int = 4):
    """Device data of one ragged sub-array (torch Philox stream), float16
    ``(C,S,T,P,2)``. Used where the host generator would be too slow."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed((BASE_SEED + seed_offset) * 1_000_003 + index)
    return torch.randn((C, S, T, P, 2), generator=gen, device=device,
                       dtype=torch.float32).to(torch.float16)


def station_positions(g: np.random.Generator, S: int) -> np.ndarray:
    """Station positions uniform in the unit disk, shape (S, 2)."""
    r = np.sqrt(g.uniform(0.0, 1.0, S))
    th = g.uniform(0.0, 2 * np.pi, S)
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def sky_model(C: int, S: int, T: int, g: np.random.Generator,
              fluxes=(1.0, 0.5, 0.25)) -> np.ndarray:
    """Model visibilities of a point-source sky on the baseline triangle.

    Returns complex128 ``(C, B, P, P)`` with ``B = S(S+1)/2`` baselines
    ordered ``s2*(s2+1)/2 + s1`` (s1 <= s2). For source k with flux A_k at
    direction (l_k, m_k) and channel frequency f_c = 1 + c/C the model is
    ``delta_pq * T * sum_k A_k exp(-2 pi i f_c (b_s1 - b_s2).(l_k, m_k))``.
    """
    pos = station_positions(g, S)
    lm = g.uniform(-0.1, 0.1, size=(len(fluxes), 2))
    B = S * (S + 1) // 2
    s2 = np.concatenate([np.full(j + 1, j) for j in range(S)])
    s1 = np.concatenate([np.arange(j + 1) for j in range(S)])
    d = pos[s1] - pos[s2]                                 # (B, 2)
    proj = d @ lm.T                                        # (B, K)
    out = np.zeros((C, B, P, P), dtype=np.complex128)
    for c in range(C):
        f = 1.0 + c / C
        vis = (np.exp(-2j * np.pi * f * proj) * np.asarray(fluxes)[None, :]).sum(1) * T
        out[c, :, 0, 0] = vis
        out[c, :, 1, 1] = vis
    return out


def differentiation(C: int = 64, S: int = 64, T: int = 1024, seed_offset: int = 5):
    """Workload 5: samples, gains 1+N(0,0.1^2) and a 3-source model."""
    g = rng(seed_offset)
    x = complex_normal(g, (C, S, T, P))
    gains = (1.0 + complex_normal(g, (C, S, P), sigma=0.1)).astype(np.complex64)
    model = sky_model(C, S, T, g).astype(np.complex64)
    return dict(x=x, g=gains, M=model, S=S, C=C, T=T, I=1, dtype="cf32")


def precision_device(C: int = 480, S: int = 256, T: int = 1024, device="cuda",
                     seed_offset: int = 3, rank: int = 0, first_channel: int = 0):
    """Workload 3 drawn on the device (torch Philox stream): complex int8 from
    N(0, 32^2), rounded and clipped to +-127, shape ``(C, S, T, P, 2)``.
    Same recipe as ``precision`` (different stream), for full-size runs.
    Each channel has its own seed, so channels ``first_channel ..
    first_channel + C - 1`` are the same values whoever draws them (a rank's
    share of a workload split over ranks); ``rank`` gives a rank a workload
    of its own instead."""
    import torch
    gen = torch.Generator(device=device)
    base = ((BASE_SEED + seed_offset) * 7919 + rank) * 65536
    out = torch.empty((C, S, T, P, 2), dtype=torch.int8, device=device)
    for c in range(C):
        gen.manual_seed(base + first_channel + c)
        v = torch.randn((S, T, P, 2), generator=gen, device=device) * 32.0
        out[c] = v.round_().clamp_(-127, 127).to(torch.int8)
    return out
