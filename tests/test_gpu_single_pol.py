"""Single-polarisation plans (n_pols = 1) against the FP64 oracle.

The tensor path pairs stations (2m, 2m+1) as the two pols of one
pseudo-station; these tests cover odd station counts (the last pseudo-station
half empty), ragged sample counts (int8 rows that are not whole 16-byte
chunks take the plain-load copy), every tile variant, the exact INT8 fold
with extreme samples, ragged batches, host streaming, and the FP32 path."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP16, rel_frobenius_per_unit, to_numpy_int, to_numpy_vis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VARIANTS = ["narrow", "wide", "pair"]


@pytest.fixture(params=VARIANTS)
def variant(request, monkeypatch):
    monkeypatch.setenv("CORR_TC_VARIANT", request.param)
    return request.param


def int8_samples(seed, C, S, T, extreme=False):
    g = synth.rng(seed)
    if extreme:
        return np.where(g.random((C, S, T, 1, 2)) < 0.5, -127, 127).astype(np.int8)
    return synth.int8_normal(g, (C, S, T, 1))


def run(x, S, C, T, dtype, path="tensor"):
    from paper_1702_00844_gb300 import Plan
    plan = Plan(S, C, T, dtype=dtype, path=path, n_pols=1)
    out = plan.empty_out()
    if dtype == "ci8":
        out.fill_(0x7FFFFFFF)
    else:
        out.fill_(float("nan"))
    plan.correlate(torch.from_numpy(np.ascontiguousarray(x)).cuda(), out)
    torch.cuda.synchronize()
    plan.check_error()
    return out


SHAPES = [(1, 1, 1), (2, 40, 2), (3, 33, 1), (65, 64, 2), (128, 96, 1), (129, 100, 2),
          (150, 36, 1), (255, 64, 1), (256, 40, 1)]


@pytest.mark.parametrize("S,T,C", SHAPES)
def test_single_pol_int8_exact(S, T, C, variant):
    x = int8_samples(S * 7 + T, C, S, T)
    got = to_numpy_int(run(x, S, C, T, "ci8"))
    ref = oracle.correlate(x, "ci8")
    np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1].reshape(ref.shape), ref.imag.astype(np.int64))


@pytest.mark.parametrize("S,T,C", [(3, 33, 1), (129, 100, 2), (200, 257, 1)])
def test_single_pol_fp16(S, T, C, variant):
    g = synth.rng(S + 5 * T)
    x = g.standard_normal((C, S, T, 1, 2)).astype(np.float16)
    got = to_numpy_vis(run(x, S, C, T, "cf16"), "cf16")
    ref = oracle.correlate(x, "cf16")
    assert np.isfinite(got).all()
    assert rel_frobenius_per_unit(got.reshape(ref.shape), ref).max() < TOL_FP16


@pytest.mark.parametrize("T", [512, 1500])
def test_single_pol_int8_extremes_fold(T, variant):
    """All +-127 samples: every partial sum at its bound; T = 1500 takes the
    checked launch plus the chunked redo of every tile."""
    S, C = 70, 2
    x = int8_samples(T, C, S, T, extreme=True)
    got = to_numpy_int(run(x, S, C, T, "ci8"))
    ref = oracle.correlate(x, "ci8")
    np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1].reshape(ref.shape), ref.imag.astype(np.int64))


def test_single_pol_equals_xx_of_two_pols():
    """The single-pol plan's visibilities are the XX entries of the two-pol
    plan on samples whose X pol is the same data (GPU against GPU, both
    exact), for a station count that spans several blocks."""
    from paper_1702_00844_gb300 import Plan
    S, C, T = 190, 3, 96
    x1 = int8_samples(4, C, S, T)
    x2 = np.concatenate([x1, int8_samples(5, C, S, T)], axis=3)
    p1 = Plan(S, C, T, dtype="ci8", path="tensor", n_pols=1)
    p2 = Plan(S, C, T, dtype="ci8", path="tensor")
    o1 = p1.correlate(torch.from_numpy(x1).cuda())
    o2 = p2.correlate(torch.from_numpy(x2).cuda())
    torch.cuda.synchronize()
    assert torch.equal(o1[..., 0, 0, :], o2[..., 0, 0, :])


def test_single_pol_batched_and_host_streaming():
    from paper_1702_00844_gb300 import FLAG_HOST_IO, Plan
    shapes = [(37, 3, 64), (128, 2, 200), (5, 4, 31), (300, 1, 96)]
    xs, outs, hosts = [], [], []
    for k, (S, C, T) in enumerate(shapes):
        h = int8_samples(100 + k, C, S, T)
        hosts.append(h)
        xs.append(torch.from_numpy(h).cuda())
        outs.append(torch.full((C, S * (S + 1) // 2, 1, 1, 2), 0x7FFFFFFF, dtype=torch.int32,
                               device="cuda"))
    plan = Plan(1, 1, 1, dtype="ci8", path="tensor", n_pols=1)
    plan.correlate_batched(list(zip(xs, outs)), shapes)
    torch.cuda.synchronize()
    plan.check_error()
    for h, o in zip(hosts, outs):
        ref = oracle.correlate(h, "ci8")
        got = to_numpy_int(o)
        np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    S, C, T = 100, 6, 128
    h = int8_samples(9, C, S, T)
    plan = Plan(S, C, T, dtype="ci8", path="tensor", flags=FLAG_HOST_IO, n_pols=1)
    out = plan.correlate_host(torch.from_numpy(h).pin_memory())
    torch.cuda.synchronize()
    ref = oracle.correlate(h, "ci8")
    got = out.numpy().astype(np.int64)
    np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1].reshape(ref.shape), ref.imag.astype(np.int64))


@pytest.mark.parametrize("S,T,C,I", [(1, 5, 1, 1), (3, 33, 2, 1), (17, 100, 3, 2), (64, 768, 4, 1),
                                     (129, 64, 1, 1), (200, 40, 1, 1)])
def test_single_pol_fp32(S, T, C, I):
    """FP32 CUDA-core path with one polarisation (pairs of stations staged as
    the two pols of pseudo-stations by 8-byte asynchronous copies)."""
    from paper_1702_00844_gb300 import Plan
    from helpers import TOL_FP32
    g = synth.rng(S * 3 + T)
    x = (g.standard_normal((I, C, S, T, 1)) + 1j * g.standard_normal((I, C, S, T, 1))).astype(np.complex64)
    plan = Plan(S, C, T, I, dtype="cf32", path="fp32", n_pols=1)
    out = plan.empty_out()
    out.fill_(float("nan"))
    plan.correlate(torch.from_numpy(x).cuda(), out)
    torch.cuda.synchronize()
    plan.check_error()
    got = out.cpu().numpy().reshape((I * C, S * (S + 1) // 2, 1, 1))
    ref = oracle.correlate(x.reshape((I * C, S, T, 1)))
    assert np.isfinite(got).all()
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP32


def test_single_pol_fp32_equals_xx_of_two_pols():
    from paper_1702_00844_gb300 import Plan
    S, C, T = 70, 3, 96
    g = synth.rng(77)
    x2 = (g.standard_normal((C, S, T, 2)) + 1j * g.standard_normal((C, S, T, 2))).astype(np.complex64)
    x1 = np.ascontiguousarray(x2[..., :1])
    o1 = Plan(S, C, T, dtype="cf32", path="fp32", n_pols=1).correlate(torch.from_numpy(x1).cuda())
    o2 = Plan(S, C, T, dtype="cf32", path="fp32").correlate(torch.from_numpy(x2).cuda())
    torch.cuda.synchronize()
    a, b = o1[..., 0, 0].cpu().numpy(), o2[..., 0, 0].cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
