"""corr_gain_backward_noalloc, the entry point for callers that cannot allocate
device memory (for example a real-time pipeline that forbids cudaMalloc once
observing has started): its results must match corr_gain_backward, which
uses a plan and its own workspace, on two calls in a row (the second call
reuses the library's fixed scratch array as the first left it).

This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def test_noalloc_matches_planned_adjoint_twice():
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan, lib
    L = lib()
    S, C, T = 24, 3, 160
    g = synth.rng(85)
    x = synth.complex_normal(g, (C, S, T, 2))
    gains = (1 + synth.complex_normal(g, (C, S, 2), sigma=0.1)).astype(np.complex64)
    M = synth.sky_model(C, S, T, g).astype(np.complex64)
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    scale = torch.tensor(0.75, dtype=torch.float32, device="cuda")
    ref_loss = torch.empty((), dtype=torch.float32, device="cuda")
    ref_g, ref_x = plan.gain_backward(xd, gd, Md, R=R, grad_scale=scale, loss=ref_loss)
    torch.cuda.synchronize()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        got_g = torch.full_like(gd, float("nan"))
        got_x = torch.full_like(xd, float("nan"))
        got_loss = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
        st = L.corr_gain_backward_noalloc(S, C, T, _vp(xd), _vp(gd), _vp(Md), _vp(R), _vp(got_g),
                                          _vp(got_x), _vp(got_loss), _vp(scale), stream)
        assert st == 0, L.corr_last_error_message()
        torch.cuda.synchronize()
        for got, ref in ((got_g, ref_g), (got_x, ref_x)):
            got = got.cpu().numpy().astype(np.complex128)
            ref = ref.cpu().numpy().astype(np.complex128)
            assert np.isfinite(got).all()
            assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()
        assert abs(float(got_loss) - float(ref_loss)) <= 1e-5 * abs(float(ref_loss))


def test_noalloc_rejects_problems_beyond_the_fixed_array():
    from paper_1702_00844_gb300 import lib
    L = lib()
    cap = L.corr_noalloc_scratch_bytes()
    S = 512                       # W' is (2S)^2 complex64 = 32*S*S bytes per channel = 8 MiB
    C = cap // (32 * S * S) + 1   # one channel more than fits
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = _vp(dummy)
    st = L.corr_gain_backward_noalloc(S, C, 8, p, p, p, p, p, p, None, None, None)
    assert st == 2
    assert b"scratch" in L.corr_last_error_message()
