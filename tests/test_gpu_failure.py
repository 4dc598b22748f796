"""Failure detection without a GPU fault: every pipeline wait in the kernels
has a time limit. With the limit set to 1 ns (CORR_WAIT_LIMIT_NS, read when a
plan is created) the tensor kernel gives up on its first wait that does not
complete at once, records the timeout in the plan's error word and returns
after draining its own copies and MMAs and freeing TMEM. The host sees
CORR_ERR_TIMEOUT, and the context stays usable: a plan with the default
limit afterwards gives exact results."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", ["narrow", "pair"])
def test_tensor_wait_timeout_is_reported_and_context_survives(monkeypatch, variant):
    """narrow: one CTA gives up; pair: either CTA of a cluster gives up and
    the other runs into its own limits, both meet at the final cluster
    barrier."""
    from paper_1702_00844_gb300 import CorrError, Plan
    S, C, T = 256, 24, 4096   # each tile's epilogue waits ~100 us for its MMAs
    monkeypatch.setenv("CORR_WAIT_LIMIT_NS", "1")
    monkeypatch.setenv("CORR_TC_VARIANT", variant)
    plan = Plan(S, C, T, dtype="cf16", path="tensor")
    x = torch.zeros((C, S, T, 2, 2), dtype=torch.float16, device="cuda")
    plan.correlate(x)
    torch.cuda.synchronize()          # the kernel ended by itself
    with pytest.raises(CorrError) as e:
        plan.check_error()
    assert e.value.status == 5
    plan.check_error()                # the error word was cleared by the read

    monkeypatch.delenv("CORR_WAIT_LIMIT_NS")
    S2, C2, T2 = 70, 2, 600
    x8 = synth.int8_normal(synth.rng(95), (C2, S2, T2, 2))
    good = Plan(S2, C2, T2, dtype="ci8", path="tensor")
    out = good.correlate(torch.from_numpy(x8).cuda())
    torch.cuda.synchronize()
    good.check_error()
    ref = oracle.correlate(x8, "ci8")
    got = out.cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1].reshape(ref.shape), ref.imag.astype(np.int64))


def test_fp32_tiny_wait_limit_is_safe(monkeypatch):
    """The FP32 kernel only waits for its own TMA loads; with a 1 ns limit it
    either finishes or reports a timeout, and drains its loads either way."""
    from paper_1702_00844_gb300 import CorrError, Plan
    S, C, T = 64, 64, 2048
    monkeypatch.setenv("CORR_WAIT_LIMIT_NS", "1")
    plan = Plan(S, C, T, dtype="cf32", path="fp32")
    x = torch.zeros((C, S, T, 2), dtype=torch.complex64, device="cuda")
    plan.correlate(x)
    torch.cuda.synchronize()
    try:
        plan.check_error()
    except CorrError as e:
        assert e.status == 5
    monkeypatch.delenv("CORR_WAIT_LIMIT_NS")
    d = synth.tiny()
    good = Plan(d["S"], d["C"], d["T"], dtype="cf32", path="fp32")
    out = good.correlate(torch.from_numpy(d["x"]).cuda())
    torch.cuda.synchronize()
    good.check_error()
    ref = oracle.correlate(d["x"])
    got = out.cpu().numpy().reshape(ref.shape)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_input_gradient_wait_timeout_is_reported_and_context_survives(monkeypatch):
    """The tensor-core input gradient with a 1 ns wait limit, on 1024
    stations (128 K-blocks per tile, so that the epilogue waits about 100 us
    for a tile's MMAs): its roles give up on their first wait that does not
    complete at once; the loader waits for its copies in flight and the MMA
    thread for its MMAs before TMEM is freed. The host sees
    CORR_ERR_TIMEOUT, and a plan with the default limit afterwards matches
    the oracle."""
    from paper_1702_00844_gb300 import FLAG_GAINS, CorrError, Plan
    S, C, T = 1024, 2, 256
    B = S * (S + 1) // 2
    x = torch.zeros((C, S, T, 2), dtype=torch.complex64, device="cuda")
    g = torch.ones((C, S, 2), dtype=torch.complex64, device="cuda")
    R = torch.zeros((C, B, 2, 2), dtype=torch.complex64, device="cuda")
    M = torch.zeros_like(R)
    monkeypatch.setenv("CORR_WAIT_LIMIT_NS", "1")
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    plan.gain_backward(x, g, M, R=R)
    torch.cuda.synchronize()          # the kernels ended by themselves
    with pytest.raises(CorrError) as e:
        plan.check_error()
    assert e.value.status == 5
    plan.check_error()

    monkeypatch.delenv("CORR_WAIT_LIMIT_NS")
    S2, C2, T2 = 40, 3, 300
    rg = synth.rng(97)
    xh = synth.complex_normal(rg, (C2, S2, T2, 2))
    gains = (1 + synth.complex_normal(rg, (C2, S2, 2), sigma=0.1)).astype(np.complex64)
    Mh = synth.sky_model(C2, S2, T2, rg).astype(np.complex64)
    xd, gd, Md = (torch.from_numpy(a).cuda() for a in (xh, gains, Mh))
    good = Plan(S2, C2, T2, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    _, gx = good.gain_backward(xd, gd, Md)
    torch.cuda.synchronize()
    good.check_error()
    Rref = oracle.correlate(xh)
    ref = oracle.input_grad(xh, Rref, gains, Mh)
    got = gx.cpu().numpy().astype(np.complex128)
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()
