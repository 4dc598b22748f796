"""Host-side checks (no GPU): the seeded input recipes are deterministic and
have the stated shapes, ranges and distributions, and the benchmark's
operation count, profile-summary link and peak fallback behave as stated."""
import os
import sys

import numpy as np

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def test_recipes_are_deterministic():
    a = synth.tiny()["x"]
    b = synth.tiny()["x"]
    assert np.array_equal(a, b)
    s1 = synth.batching_shapes()
    s2 = synth.batching_shapes()
    assert s1 == s2 and len(s1) == 32


def test_int8_recipe_range_and_scale():
    x = synth.int8_normal(synth.rng(5), (2, 16, 4096, 2))
    assert x.dtype == np.int8 and x.shape == (2, 16, 4096, 2, 2)
    assert x.min() >= -127 and x.max() <= 127        # clipped to +-127, never -128
    assert 30.0 < x.astype(np.float64).std() < 34.0  # N(0, 32^2) before rounding


def test_int8_as_cf16_is_exact():
    x = synth.int8_normal(synth.rng(6), (1, 4, 64, 2))
    h = synth.int8_as_cf16(x)
    assert h.dtype == np.float16
    assert np.array_equal(h.astype(np.int64), x.astype(np.int64))


def test_batching_shapes_follow_the_workload():
    for S, C, T in synth.batching_shapes():
        assert 16 <= S <= 576 and 64 <= C <= 512
        assert 256 <= T <= 4096 and T % 128 == 0


def test_differentiation_recipe():
    d = synth.differentiation(C=3, S=5, T=16)
    assert d["x"].shape == (3, 5, 16, 2) and d["x"].dtype == np.complex64
    assert d["g"].shape == (3, 5, 2)
    assert np.abs(d["g"] - 1).max() < 1.0          # 1 + N(0, 0.1^2)
    B = 5 * 6 // 2
    assert d["M"].shape == (3, B, 2, 2)
    # the model is pol-diagonal (delta_pq) and Hermitian on autocorrelations
    assert np.all(d["M"][..., 0, 1] == 0) and np.all(d["M"][..., 1, 0] == 0)


def test_bench_ops_count_and_profile_link():
    import bench
    # 8 ops per complex multiply-add x 4 pol pairs x S(S+1)/2 baselines x T x units
    assert bench.ops_of(256, 1024, 480) == 32.0 * 32896 * 1024 * 480
    # the committed ncu summary carries the keys the roofline reads
    keys = {}
    for ln in open(bench.PROFILE_SUMMARY):
        if ":" in ln and not ln.startswith("#"):
            k, v = ln.split(":", 1)
            keys[k.strip()] = v.strip()
    assert len(keys["source_sha256_16"]) == 16
    assert float(keys["dram_bytes_per_launch_full"]) > 0
    peaks, src = bench.measured_peaks()
    assert src in ("measured", "fallback") and peaks["hbm_gbs"] > 0


def test_bench_ragged_mode_and_error_metrics():
    """--workload ragged with --ragged-scale keeps every sub-array and
    scales its channels (at least one each); the error metrics the bench
    reports against the oracle are the plain definitions."""
    import numpy as np

    import bench
    import synth
    a = bench.parse(["--workload", "ragged", "--ragged-scale", "0.05"])
    assert a.workload == "ragged" and a.ragged_scale == 0.05
    full = synth.batching_shapes()
    small = bench.ragged_shapes(0.05)
    assert [(s, t) for s, _, t in small] == [(s, t) for s, _, t in full]
    assert all(c == max(1, round(C * 0.05)) for (_, c, _), (_, C, _) in zip(small, full))
    assert bench.ragged_shapes(1.0) == full
    # relative Frobenius error per unit, the largest over units
    ref = np.ones((2, 3, 2, 2), dtype=np.complex128)
    got = ref.copy()
    got[1, 0, 0, 0] += 0.5
    assert abs(bench._rel_frob(got, ref) - 0.5 / np.sqrt(12)) < 1e-12
    # correlation-coefficient error: |dV_ab| / sqrt(V_aa V_bb); 2 stations
    S = 2
    ref = np.zeros((1, 3, 2, 2), dtype=np.complex128)
    ref[0, 0, 0, 0] = ref[0, 0, 1, 1] = 4.0     # station 0 autocorrelations
    ref[0, 2, 0, 0] = ref[0, 2, 1, 1] = 9.0     # station 1
    got = ref.copy()
    got[0, 1, 0, 1] += 1.2                      # baseline (0, 1), X x Y
    assert abs(bench._coef_err(got, ref, S) - 1.2 / 6.0) < 1e-12
