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
