"""tcgen05 tensor-core path against the FP64 oracle.

INT8 inputs: bit-exact INT32 visibilities. FP16 inputs: the oracle is fed the
same FP16 values widened exactly, so the only difference is FP32
accumulation (tolerance TOL_FP16, per channel, relative Frobenius norm).
"""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP16, coef_error, rel_frobenius_per_unit, to_numpy_int, to_numpy_vis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


VARIANTS = ["narrow", "wide", "pair"]
# Tile configurations (variant, tail kind of the pair variant's second list,
# kernel layout): the autotuner chooses among these.
CONFIGS = {"narrow": ("narrow", None, None), "wide": ("wide", None, None),
           "pair": ("pair", None, None), "pair-narrow-tail": ("pair", "narrow", None),
           "pair-wide-tail": ("pair", "wide", None), "pair-layout1": ("pair", None, "1")}


def force_config(monkeypatch, name):
    v, tail, layout = CONFIGS[name]
    monkeypatch.setenv("CORR_TC_VARIANT", v)
    for key, val in (("CORR_TC_TAIL", tail), ("CORR_TC_LAYOUT", layout)):
        if val is None:
            monkeypatch.delenv(key, raising=False)
        else:
            monkeypatch.setenv(key, val)
    return v


@pytest.fixture(params=list(CONFIGS))
def variant(request, monkeypatch):
    """Forces the tile configuration of the plans a test creates; returns its
    variant."""
    return force_config(monkeypatch, request.param)


def run_tc(x: np.ndarray, S, C, T, dtype, I=1, expect_variant=None):
    from paper_1702_00844_gb300 import Plan
    plan = Plan(S, C, T, I, dtype=dtype, path="tensor")
    if expect_variant:
        assert plan.tile_variant() == expect_variant
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = plan.empty_out()
    if dtype == "ci8":
        out.fill_(0x7FFFFFFF)
    else:
        out.fill_(float("nan"))
    plan.correlate(xd, out)
    torch.cuda.synchronize()
    plan.check_error()
    return out


def exact_int(got_t, x8):
    """INT32 result equals the exact integer result of the oracle."""
    ref = oracle.correlate(x8, "ci8")
    got = to_numpy_int(got_t)
    ref_re = np.rint(ref.real).astype(np.int64)
    ref_im = np.rint(ref.imag).astype(np.int64)
    assert np.array_equal(ref.real, ref_re) and np.array_equal(ref.imag, ref_im)
    np.testing.assert_array_equal(got[..., 0], ref_re.reshape(got[..., 0].shape))
    np.testing.assert_array_equal(got[..., 1], ref_im.reshape(got[..., 1].shape))


SHAPES = [(1, 1, 1), (2, 3, 2), (5, 8, 1), (64, 32, 2), (65, 33, 2), (150, 100, 3),
          (128, 64, 1), (130, 30, 2), (200, 257, 1)]


@pytest.mark.parametrize("S,T,C", SHAPES)
def test_int8_exact(S, T, C, variant):
    g = synth.rng(60, S * 1000 + T)
    x8 = synth.int8_normal(g, (C, S, T, 2))
    out = run_tc(x8, S, C, T, "ci8", expect_variant=variant)
    exact_int(out, x8)


@pytest.mark.parametrize("S,T,C", SHAPES)
def test_fp16_matches_oracle(S, T, C, variant):
    g = synth.rng(61, S * 1000 + T)
    x16 = synth.to_cf16(synth.complex_normal(g, (C, S, T, 2)))
    got = to_numpy_vis(run_tc(x16, S, C, T, "cf16", expect_variant=variant), "cf16")
    ref = oracle.correlate(x16, "cf16")
    assert np.isfinite(got).all()
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP16
    assert coef_error(got, ref, S) < 1e-4


@pytest.mark.parametrize("T", [512, 1024, 1500])
def test_int8_adversarial_extremes_chunk_fold(T, variant):
    """All-(+-127) samples drive every partial sum to its bound; the 512-sample
    chunks keep each FP32 partial below 2^24 and the INT32 fold is exact."""
    S, C = 70, 1
    g = synth.rng(62, T)
    signs = np.where(g.random((C, S, T, 2, 2)) < 0.5, -127, 127).astype(np.int8)
    signs[0, 3] = 127  # a station with all +127 (largest autocorrelation)
    signs[0, 4] = -127
    out = run_tc(signs, S, C, T, "ci8")
    exact_int(out, signs)


@pytest.mark.parametrize("variant", ["pair-narrow-tail", "pair-wide-tail", "pair-layout1"], indirect=True)
def test_int8_extremes_odd_block_count_pair_and_tail(variant):
    """Three 64-station blocks with the pair variant: pair tiles over two
    blocks and the third block's tiles in a second list (narrow tiles for
    the last block column, or wide tiles for block 0's row), in two launches
    with their own redo lists. All-(+-127) samples over 1500 samples make
    every tile of both lists fail the power check and take its chunked redo."""
    S, C, T = 150, 2, 1500
    g = synth.rng(63, T)
    x = np.where(g.random((C, S, T, 2, 2)) < 0.5, -127, 127).astype(np.int8)
    out = run_tc(x, S, C, T, "ci8", expect_variant="pair")
    exact_int(out, x)


def test_fp16_int_valued_exact_below_2pow24():
    """FP16 copies of int8 samples with T <= 512: exact integers in FP32."""
    S, T, C = 96, 512, 2
    g = synth.rng(63)
    x8 = synth.int8_normal(g, (C, S, T, 2))
    got = to_numpy_vis(run_tc(synth.int8_as_cf16(x8), S, C, T, "cf16"), "cf16")
    ref = oracle.correlate(x8, "ci8")
    np.testing.assert_array_equal(got, ref)


def test_autotuner_picks_a_variant_and_variants_agree(monkeypatch):
    """The autotuned plan reports one of the variants, and every variant gives
    the same (exact) INT8 result on a 3-block station count (odd: the pair
    variant's last tile has a block with no stations)."""
    from paper_1702_00844_gb300 import Plan
    S, T, C = 190, 96, 3
    x8 = synth.int8_normal(synth.rng(64), (C, S, T, 2))
    for key in ("CORR_TC_VARIANT", "CORR_TC_TAIL", "CORR_TC_LAYOUT"):
        monkeypatch.delenv(key, raising=False)
    plan = Plan(S, C, T, dtype="ci8", path="tensor")
    assert plan.tile_variant() in VARIANTS
    outs = []
    for name in CONFIGS:
        v = force_config(monkeypatch, name)
        outs.append(to_numpy_int(run_tc(x8, S, C, T, "ci8", expect_variant=v)))
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)


def test_zero_samples_gives_zeros():
    from paper_1702_00844_gb300 import Plan
    for dt in ("cf16", "ci8"):
        plan = Plan(70, 2, 0, dtype=dt, path="tensor")
        out = plan.empty_out()
        out.fill_(7)
        x = torch.zeros(16, dtype=torch.float16 if dt == "cf16" else torch.int8, device="cuda")[:0]
        plan.correlate(x, out)
        torch.cuda.synchronize()
        assert (out == 0).all()


@pytest.mark.parametrize("variant", VARIANTS, indirect=True)
def test_precision_workload_full_size_sampled(variant):
    """The 256-station, 480-channel, 1024-sample INT8 workload in the launch
    configuration the benchmark times; sampled channels are compared with the
    oracle bit for bit (INT8) and within tolerance (FP16 of the same values),
    and every channel's XX/YY autocorrelations must be real and positive."""
    d = synth.precision()
    S, C, T = d["S"], d["C"], d["T"]
    x8 = d["x"]
    out8 = run_tc(x8, S, C, T, "ci8")
    out16 = run_tc(synth.int8_as_cf16(x8), S, C, T, "cf16")
    picks = [0, 137, 479]
    got8 = to_numpy_int(out8)
    got16 = to_numpy_vis(out16, "cf16")
    for c in picks:
        ref = oracle.correlate(x8[c][None], "ci8")
        np.testing.assert_array_equal(got8[c][None][..., 0], ref.real.astype(np.int64))
        np.testing.assert_array_equal(got8[c][None][..., 1], ref.imag.astype(np.int64))
        assert rel_frobenius_per_unit(got16[c][None], ref).max() < TOL_FP16
    autos = [s * (s + 1) // 2 + s for s in range(S)]
    for p in range(2):
        assert (got8[:, autos, p, p, 1] == 0).all()
        assert (got8[:, autos, p, p, 0] > 0).all()


def test_several_integrations_one_launch(variant):
    """Integrations are stacked in front of the channels: [I][C][S][T][pol]."""
    S, C, T, I = 100, 3, 96, 4
    x8 = synth.int8_normal(synth.rng(65), (I, C, S, T, 2))
    out = run_tc(x8, S, C, T, "ci8", I=I, expect_variant=variant)
    got = to_numpy_int(out)
    ref = oracle.correlate(x8.reshape(I * C, S, T, 2, 2), "ci8")
    np.testing.assert_array_equal(got[..., 0], ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1], ref.imag.astype(np.int64))


def test_int8_largest_output_sampled():
    """16384 stations, one channel, 64 samples: 134 M baselines, a 4.3 GB
    output whose byte offsets pass 2^32 and 8256 pair tiles of 128 x 128
    stations. Sampled baselines (corners, block edges, random pairs) equal
    the oracle bit for bit; the oracle correlates each sampled station pair
    as a two-station array."""
    S, C, T = 16384, 1, 64
    g = synth.rng(140)
    x8 = synth.int8_normal(g, (C, S, T, 2))
    out = run_tc(x8, S, C, T, "ci8")
    edges = [0, 1, 63, 64, 127, 128, 8191, 8192, S - 2, S - 1]
    pairs = {(a, b) for a in edges for b in edges if a <= b}
    r = g.integers(0, S, size=(400, 2))
    pairs |= {(int(min(a, b)), int(max(a, b))) for a, b in r}
    pairs = sorted(pairs)
    idx = torch.tensor([s2 * (s2 + 1) // 2 + s1 for s1, s2 in pairs], dtype=torch.long, device="cuda")
    got = out[0, 0].index_select(0, idx).cpu().numpy().astype(np.int64)   # [n][p1][p2][re, im]
    for k, (s1, s2) in enumerate(pairs):
        sub = x8[:, [s1, s2]] if s1 != s2 else x8[:, [s1]]
        ref = oracle.correlate(np.ascontiguousarray(sub), "ci8")[0]
        v = ref[1] if s1 != s2 else ref[0]                            # baseline (0, 1) or (0, 0)
        np.testing.assert_array_equal(got[k][..., 0], v.real.astype(np.int64))
        np.testing.assert_array_equal(got[k][..., 1], v.imag.astype(np.int64))
