"""FP32 samples on the tensor cores (path "tensor", dtype cf32): every sample
split into a tf32 value and a tf32 remainder, three tf32 products per
product term, FP32 accumulation. Checked against the FP64 oracle with the
FP32 path's tolerance (per-channel relative Frobenius error below 1e-5) and
element-wise through the correlation-coefficient error, on shapes that
span several 64-station blocks with a partial last one, sample counts that
are not multiples of the 16-sample K-block, diagonal-only problems, both
ways of summing 256-sample accumulator chunks, and the production workload
(sampled channels)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import coef_error, rel_frobenius_per_unit

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run(x, S, C, T, I=1):
    from paper_1702_00844_gb300 import Plan
    plan = Plan(S, C, T, I, dtype="cf32", path="tensor")
    out = plan.empty_out()
    out.fill_(float("nan"))
    plan.correlate(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out)
    torch.cuda.synchronize()
    plan.check_error()
    assert plan.tile_variant() == "fp32"   # not one of the f16/int8 tile variants
    got = out.cpu().numpy().astype(np.complex128)
    return got.reshape((-1,) + got.shape[-3:])


@pytest.mark.parametrize("S,C,T", [(8, 16, 256), (1, 3, 40), (64, 4, 768), (70, 3, 100),
                                   (130, 2, 33), (200, 2, 257)])
def test_tf32_split_correlator_vs_oracle(S, C, T):
    g = synth.rng(120 + S)
    x = synth.complex_normal(g, (C, S, T, 2))
    got = _run(x, S, C, T)
    ref = oracle.correlate(x)
    assert np.isfinite(got).all()
    assert rel_frobenius_per_unit(got, ref).max() < 1e-5
    assert coef_error(got, ref, S) < 1e-5


def test_tf32_split_correlator_both_chunk_modes():
    """More samples than one 256-sample accumulator chunk, with many tiles
    (320 channels: chunks summed by the epilogue into the output) and with
    few (4 channels: every chunk a work item of its own, partial sums added
    by a second kernel); sampled channels against the oracle."""
    S, T = 64, 600
    for C in (320, 4):
        g = synth.rng(140 + C)
        x = synth.complex_normal(g, (C, S, T, 2))
        got = _run(x, S, C, T)
        for c in sorted({0, C // 2, C - 1}):
            ref = oracle.correlate(x[c][None])
            assert rel_frobenius_per_unit(got[c][None], ref).max() < 1e-5, C
            assert coef_error(got[c][None], ref, S) < 1e-5, C


def test_tf32_split_correlator_integrations_and_exact_integers():
    """Integrations stacked before the channels; small integer samples,
    whose products and sums are exact in FP32 and in the split (the
    remainders are zero), give the oracle's values exactly."""
    S, C, T, I = 90, 2, 48, 3
    g = synth.rng(131)
    x = g.integers(-8, 9, size=(I, C, S, T, 2, 2)).astype(np.float32)
    xc = (x[..., 0] + 1j * x[..., 1]).astype(np.complex64)
    got = _run(xc, S, C, T, I)
    ref = oracle.correlate(xc.reshape(I * C, S, T, 2))
    np.testing.assert_array_equal(got, ref)


def test_tf32_split_correlator_empty_time_axis():
    from paper_1702_00844_gb300 import Plan
    S, C = 20, 2
    plan = Plan(S, C, 0, dtype="cf32", path="tensor")
    out = plan.empty_out()
    out.fill_(float("nan"))
    plan.correlate(torch.empty(0, dtype=torch.complex64, device="cuda"), out)
    torch.cuda.synchronize()
    assert (out == 0).all()


def test_tf32_split_correlator_production_sampled():
    """64 stations, 256 channels, 768 samples, one integration (the
    production recipe): one diagonal tile per channel; sampled channels."""
    d = synth.production(n_integrations=1)
    x = d["x"][0]
    C, S, T = x.shape[0], x.shape[1], x.shape[2]
    got = _run(x, S, C, T)
    for c in (0, 100, 255):
        ref = oracle.correlate(x[c][None])
        assert rel_frobenius_per_unit(got[c][None], ref).max() < 1e-5
        assert coef_error(got[c][None], ref, S) < 1e-5


def test_tf32_split_correlator_single_pol_is_unsupported():
    from paper_1702_00844_gb300 import CorrError, Plan
    with pytest.raises(CorrError) as e:
        Plan(16, 2, 64, dtype="cf32", path="tensor", n_pols=1)
    assert e.value.status == 2
