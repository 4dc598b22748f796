"""corr_gain_backward_noalloc, the entry point for callers that cannot allocate
device memory (for example a real-time pipeline that forbids cudaMalloc once
observing has started): its results must match the FP64 oracle's closed-form
gradients and loss, and corr_gain_backward (which uses a plan and its own
workspace), on two calls in a row (the second call reuses the library's
fixed scratch array as the first left it). Also covered: no input gradient,
loss only, an empty time axis, a loss scalar inside a larger buffer, and the
rejection of problems that do not fit the fixed array.

This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _case(S=24, C=3, T=160, seed=85):
    g = synth.rng(seed)
    x = synth.complex_normal(g, (C, S, T, 2))
    gains = (1 + synth.complex_normal(g, (C, S, 2), sigma=0.1)).astype(np.complex64)
    M = synth.sky_model(C, S, max(T, 1), g).astype(np.complex64)
    return x, gains, M


def _close(got, ref, tol=1e-4):
    got = got.cpu().numpy().astype(np.complex128)
    assert np.isfinite(got).all()
    scale = np.abs(ref).max()
    if scale == 0:
        assert np.abs(got).max() == 0
    else:
        assert np.abs(got - ref).max() < tol * scale


def _call(L, S, C, T, xd, gd, Md, R, grad_g, grad_x, loss, scale):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.corr_gain_backward_noalloc(S, C, T, _vp(xd), _vp(gd), _vp(Md), _vp(R), _vp(grad_g),
                                      _vp(grad_x), _vp(loss), _vp(scale), stream)
    assert st == 0, L.corr_last_error_message()
    torch.cuda.synchronize()


def test_noalloc_matches_oracle_and_planned_adjoint_twice():
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan, lib
    L = lib()
    x, gains, M = _case()
    C, S, T, _ = x.shape
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    scale = torch.tensor(0.75, dtype=torch.float32, device="cuda")
    ref_loss = torch.empty((), dtype=torch.float32, device="cuda")
    ref_g, ref_x = plan.gain_backward(xd, gd, Md, R=R, grad_scale=scale, loss=ref_loss)
    torch.cuda.synchronize()
    # the FP64 oracle's closed forms on the same samples
    Rref = oracle.correlate(x)
    Lref, _ = oracle.gain_loss(Rref, gains, M)
    gref = 0.75 * oracle.gain_grad(Rref, gains, M)
    xref = 0.75 * oracle.input_grad(x, Rref, gains, M)
    for _ in range(2):
        got_g = torch.full_like(gd, float("nan"))
        got_x = torch.full_like(xd, float("nan"))
        got_loss = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
        _call(L, S, C, T, xd, gd, Md, R, got_g, got_x, got_loss, scale)
        _close(got_g, gref)
        _close(got_x, xref)
        assert abs(float(got_loss) - Lref) <= 1e-5 * Lref
        # and the planned entry point, within the same tolerance
        _close(got_g, ref_g.cpu().numpy().astype(np.complex128))
        _close(got_x, ref_x.cpu().numpy().astype(np.complex128))
        assert abs(float(got_loss) - float(ref_loss)) <= 1e-5 * abs(float(ref_loss))


def test_noalloc_without_input_gradient_and_loss_only():
    """d_grad_in = NULL (no W' in the scratch array), then d_loss only next to
    the required gain gradient, with the loss scalar at a 4-byte offset
    inside a larger buffer."""
    from paper_1702_00844_gb300 import Plan, lib
    L = lib()
    x, gains, M = _case(S=40, C=2, T=96, seed=86)
    C, S, T, _ = x.shape
    plan = Plan(S, C, T, dtype="cf32", path="fp32")
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    torch.cuda.synchronize()
    Rref = oracle.correlate(x)
    Lref, _ = oracle.gain_loss(Rref, gains, M)
    gref = oracle.gain_grad(Rref, gains, M)
    got_g = torch.full_like(gd, float("nan"))
    _call(L, S, C, T, xd, gd, Md, R, got_g, None, None, None)
    _close(got_g, gref)
    buf = torch.full((4,), float("nan"), dtype=torch.float32, device="cuda")
    got_g.fill_(float("nan"))
    _call(L, S, C, T, None, gd, Md, R, got_g, None, buf[1:2], None)
    _close(got_g, gref)
    assert abs(float(buf[1]) - Lref) <= 1e-5 * Lref
    assert torch.isnan(buf[0]) and torch.isnan(buf[2])


def test_noalloc_empty_time_axis():
    """T = 0: R is zero, so the gain gradient is zero and the loss is the
    model's norm over the baselines; the sample gradient has no elements."""
    from paper_1702_00844_gb300 import lib
    L = lib()
    S, C = 12, 2
    _, gains, M = _case(S=S, C=C, T=0, seed=87)
    gd, Md = _dev(gains), _dev(M)
    R = torch.zeros((C, S * (S + 1) // 2, 2, 2), dtype=torch.complex64, device="cuda")
    Rref = np.zeros(R.shape, dtype=np.complex128)
    Lref, _ = oracle.gain_loss(Rref, gains, M)
    assert Lref > 0
    got_g = torch.full_like(gd, float("nan"))
    got_x = torch.full((16,), float("nan"), dtype=torch.complex64, device="cuda")  # T = 0: no elements
    loss = torch.full((), float("nan"), dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.corr_gain_backward_noalloc(S, C, 0, None, _vp(gd), _vp(Md), _vp(R), _vp(got_g),
                                      _vp(got_x), _vp(loss), None, stream)
    assert st == 0, L.corr_last_error_message()
    torch.cuda.synchronize()
    _close(got_g, oracle.gain_grad(Rref, gains, M))
    assert abs(float(loss) - Lref) <= 1e-5 * Lref
    assert torch.isnan(got_x).all()


def test_noalloc_rejects_problems_beyond_the_fixed_array():
    """Every buffer is allocated at the size the rejected problem would use,
    so a regression of the size check shows up as a wrong status, not as
    accesses beyond a small buffer."""
    from paper_1702_00844_gb300 import lib
    L = lib()
    cap = L.corr_noalloc_scratch_bytes()
    S, T = 512, 8                 # W' is (2S)^2 complex64 = 32*S*S bytes per channel = 8 MiB
    C = cap // (32 * S * S) + 1   # one channel more than fits
    B = S * (S + 1) // 2
    x = torch.zeros((C, S, T, 2), dtype=torch.complex64, device="cuda")
    g = torch.ones((C, S, 2), dtype=torch.complex64, device="cuda")
    R = torch.zeros((C, B, 2, 2), dtype=torch.complex64, device="cuda")
    M = torch.zeros_like(R)
    grad_g = torch.full_like(g, float("nan"))
    grad_x = torch.full_like(x, float("nan"))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = L.corr_gain_backward_noalloc(S, C, T, _vp(x), _vp(g), _vp(M), _vp(R), _vp(grad_g),
                                      _vp(grad_x), None, None, stream)
    assert st == 2
    assert b"scratch" in L.corr_last_error_message()
    torch.cuda.synchronize()
    assert torch.isnan(grad_g).all() and torch.isnan(grad_x).all()   # nothing was launched
