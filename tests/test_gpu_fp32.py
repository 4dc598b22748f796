"""FP32 CUDA-core path against the FP64 oracle (element by element)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP32, coef_error, rel_frobenius_per_unit, to_numpy_vis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_fp32(x: np.ndarray, S, C, T, I=1):
    from paper_1702_00844_gb300 import Plan
    plan = Plan(S, C, T, I, dtype="cf32", path="fp32")
    xd = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).cuda()
    out = plan.empty_out()
    out.fill_(float("nan"))
    plan.correlate(xd, out)
    torch.cuda.synchronize()
    plan.check_error()
    return to_numpy_vis(out, "cf32")


def check(got, ref, S):
    assert np.isfinite(got).all(), "unwritten or non-finite outputs"
    err = rel_frobenius_per_unit(got, ref)
    assert err.max() < TOL_FP32, err.max()
    assert coef_error(got, ref, S) < 1e-4


def test_tiny_workload_full():
    d = synth.tiny()
    got = run_fp32(d["x"], d["S"], d["C"], d["T"])
    ref = oracle.correlate(d["x"])
    check(got, ref, d["S"])


@pytest.mark.parametrize("S,T,C", [(1, 1, 1), (2, 3, 2), (3, 7, 1), (5, 16, 2), (9, 33, 2),
                                   (150, 100, 3), (64, 70, 2), (37, 65, 3), (200, 17, 1)])
def test_edge_and_ragged_shapes(S, T, C):
    g = synth.rng(50, S * 1000 + T)
    x = synth.complex_normal(g, (C, S, T, 2))
    got = run_fp32(x, S, C, T)
    ref = oracle.correlate(x)
    check(got, ref, S)


def test_zero_samples_gives_zeros():
    from paper_1702_00844_gb300 import Plan
    plan = Plan(4, 2, 0, dtype="cf32", path="fp32")
    out = plan.empty_out()
    out.fill_(float("nan"))
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")[:0]
    plan.correlate(x, out)
    torch.cuda.synchronize()
    assert (out == 0).all()


def test_production_workload_sampled_channels():
    """Full 64-station, 256-channel, 768-sample, 10-integration workload in one
    launch; every channel of a few sampled integration/channel pairs is
    compared with the oracle, and all channels are checked for invariants."""
    d = synth.production()
    S, C, T, I = d["S"], d["C"], d["T"], d["I"]
    got = run_fp32(d["x"], S, C, T, I).reshape(I, C, -1, 2, 2)
    picks = [(0, 0), (3, 17), (9, 255), (5, 128)]
    for i, c in picks:
        ref = oracle.correlate(d["x"][i, c][None])
        check(got[i, c][None], ref, S)
    autos = [s * (s + 1) // 2 + s for s in range(S)]
    xx = got[:, :, autos, 0, 0]
    assert (xx.real > 0).all()
    # the XY and YX autocorrelations are conjugates
    xy = got[:, :, autos, 0, 1]
    yx = got[:, :, autos, 1, 0]
    assert np.abs(xy - np.conj(yx)).max() < 1e-5 * np.abs(xx).max()


@pytest.mark.parametrize("ks", ["1", "2", "3", "7"])
@pytest.mark.parametrize("npol", [2, 1])
def test_split_sample_axis_matches_oracle(monkeypatch, ks, npol):
    """Few units split the sample axis over CTAs (partial sums, then an
    ordered reduction); forced split counts with a ragged sample count and
    several integrations give the oracle's result within the FP32
    tolerance."""
    from paper_1702_00844_gb300 import Plan
    monkeypatch.setenv("CORR_FP32_KSPLIT", ks)
    S, C, T, I = 37, 3, 250, 2
    g = synth.rng(90 + int(ks), npol)
    x = (g.standard_normal((I, C, S, T, npol)) + 1j * g.standard_normal((I, C, S, T, npol))).astype(np.complex64)
    plan = Plan(S, C, T, I, dtype="cf32", path="fp32", n_pols=npol)
    out = plan.empty_out()
    out.fill_(float("nan"))
    plan.correlate(torch.from_numpy(x).cuda(), out)
    torch.cuda.synchronize()
    plan.check_error()
    ref = oracle.correlate(x.reshape((I * C, S, T, npol)))
    got = out.cpu().numpy().reshape(ref.shape)
    assert np.isfinite(got).all()
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP32


@pytest.mark.parametrize("S,npol", [(8, 2), (37, 2), (64, 2), (65, 2), (130, 2), (61, 1), (200, 1)])
def test_subtile_widths_bit_identical(monkeypatch, S, npol):
    """4 x 4- and 4 x 2-station sub-tiles run each accumulator's FMAs in the
    same order, so both give the same bits (station counts on and off the
    sub-tile grid, both pol counts), and both match the oracle."""
    from paper_1702_00844_gb300 import Plan
    monkeypatch.setenv("CORR_FP32_KSPLIT", "1")
    C, T = 3, 200
    g = synth.rng(120 + S, npol)
    x = (g.standard_normal((C, S, T, npol)) + 1j * g.standard_normal((C, S, T, npol))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    outs = {}
    for tw in ("4", "2"):
        monkeypatch.setenv("CORR_FP32_TW", tw)
        plan = Plan(S, C, T, dtype="cf32", path="fp32", n_pols=npol)
        out = plan.empty_out()
        out.fill_(float("nan"))
        plan.correlate(xd, out)
        torch.cuda.synchronize()
        plan.check_error()
        outs[tw] = out
    assert torch.equal(outs["4"], outs["2"])
    ref = oracle.correlate(x)
    got = outs["2"].cpu().numpy().reshape(ref.shape)
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP32
