"""Throughput accounting of the correlator (Sections 2 and 4)."""
from __future__ import annotations


def n_baselines(S: int) -> int:
    """Station pairs s1 <= s2, autocorrelations included: S(S+1)/2 (Section 2)."""
    return S * (S + 1) // 2


def correlator_ops(S: int, T: int, units: int) -> float:
    """Correlator operations: 8 per complex multiply-add (four FMAs), four
    polarisation pairs per baseline, i.e. 32 per baseline per sample."""
    return 32.0 * n_baselines(S) * T * units


def ai_global(S: int) -> float:
    """Global arithmetic intensity of FP32 input (Section 3.6): 32 flops per
    baseline over 16 bytes per station per sample = S + 1."""
    return 32.0 * n_baselines(S) / (16.0 * S)


def perf_max(peak: float, ai: float, bandwidth: float) -> float:
    """Bound-and-bottleneck model (Section 3.6): min(peak, AI x bandwidth)."""
    return min(peak, ai * bandwidth)


def io_bytes(S: int, T: int, units: int, in_bytes_per_sample: int, out_bytes_per_value: int) -> float:
    """Algorithmic bytes of one correlation: every input sample read once
    (2 pols per station and time) and every visibility written once."""
    return float(units) * (S * T * in_bytes_per_sample + n_baselines(S) * 4 * out_bytes_per_value)


# bytes per (station, time) holding both polarisations, and per output value
IN_BYTES = {"cf32": 16, "cf16": 8, "ci8": 4}
OUT_BYTES = {"cf32": 8, "cf16": 8, "ci8": 8}
