"""The multithreaded FP32 CPU correlator (Section 4.1's design, the
benchmark's comparison baseline) against the FP64 oracle: odd station counts
(partial 2x2 tiles), time axes that are not a multiple of the vector length,
one and several units, and thread counts."""
import numpy as np
import pytest

import cpu_baseline
import oracle
import synth
from helpers import TOL_FP32, coef_error, rel_frobenius_per_unit


@pytest.mark.parametrize("S,C,T", [(1, 1, 1), (2, 1, 9), (3, 2, 7), (8, 16, 256), (17, 3, 100),
                                   (64, 4, 768), (65, 2, 1031)])
def test_cpu_fp32_correlator_matches_oracle(S, C, T):
    x = synth.complex_normal(synth.rng(95, S * 7 + T), (C, S, T, 2))
    got = cpu_baseline.correlate(x).astype(np.complex128)
    ref = oracle.correlate(x)
    assert got.shape == ref.shape
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP32
    assert coef_error(got, ref, S) < 1e-5


def test_cpu_fp32_correlator_threads_and_integrations_agree():
    """Thread count and leading axes do not change the result (each tile is
    summed in a fixed order by one thread)."""
    x = synth.complex_normal(synth.rng(96), (2, 3, 20, 50, 2))
    a = cpu_baseline.correlate(x, n_threads=1)
    b = cpu_baseline.correlate(x, n_threads=4)
    c = cpu_baseline.correlate(x.reshape(6, 20, 50, 2))
    assert np.array_equal(a, b)
    assert np.array_equal(a.reshape(c.shape), c)


def test_cpu_fp32_correlator_integer_samples_exact():
    """Small integer samples: every partial sum is an exact FP32 integer."""
    g = synth.rng(97)
    x = (g.integers(-8, 9, (2, 9, 64, 2)) + 1j * g.integers(-8, 9, (2, 9, 64, 2))).astype(np.complex64)
    np.testing.assert_array_equal(cpu_baseline.correlate(x).astype(np.complex128), oracle.correlate(x))
