"""Ragged batches (one persistent launch, CUDA-graph replay) and the gain
adjoint against the FP64 oracle and finite differences."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP16, coef_error, rel_frobenius_per_unit, to_numpy_int, to_numpy_vis, tol_fp16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RAGGED = [(16, 3, 256), (70, 2, 384), (130, 1, 128), (1, 2, 7), (65, 2, 0), (200, 1, 513),
          (33, 4, 1000)]


def make_batch(dtype):
    xs, outs, hosts = [], [], []
    for k, (S, C, T) in enumerate(RAGGED):
        g = synth.rng(70, k)
        if dtype == "ci8":
            h = synth.int8_normal(g, (C, S, T, 2))
            o = torch.full((C, S * (S + 1) // 2, 2, 2, 2), 0x7FFFFFFF, dtype=torch.int32,
                           device="cuda")
        else:
            h = synth.to_cf16(synth.complex_normal(g, (C, S, T, 2)))
            o = torch.full((C, S * (S + 1) // 2, 2, 2), float("nan"), dtype=torch.complex64,
                           device="cuda")
        x = torch.from_numpy(np.ascontiguousarray(h)).cuda()
        if x.numel() == 0:
            x = torch.zeros(16, dtype=x.dtype, device="cuda")
        xs.append(x)
        outs.append(o)
        hosts.append(h)
    return xs, outs, hosts


def check_batch(dtype, outs, hosts):
    for (S, C, T), o, h in zip(RAGGED, outs, hosts):
        ref = oracle.correlate(h, dtype)
        if dtype == "ci8":
            got = to_numpy_int(o)
            np.testing.assert_array_equal(got[..., 0], ref.real.astype(np.int64))
            np.testing.assert_array_equal(got[..., 1], ref.imag.astype(np.int64))
        else:
            got = to_numpy_vis(o, "cf16")
            assert np.isfinite(got).all()
            assert rel_frobenius_per_unit(got, ref).max() < TOL_FP16
            # element-wise too: one wrong baseline cannot hide under the norm
            if T:
                assert coef_error(got, ref, S) < 1e-4


@pytest.mark.parametrize("variant", ["narrow", "wide", "pair"])
@pytest.mark.parametrize("dtype", ["cf16", "ci8"])
def test_ragged_batch_one_launch(dtype, variant, monkeypatch):
    monkeypatch.setenv("CORR_TC_VARIANT", variant)
    from paper_1702_00844_gb300 import Plan
    plan = Plan(1, 1, 1, dtype=dtype, path="tensor")
    xs, outs, hosts = make_batch(dtype)
    plan.correlate_batched(list(zip(xs, outs)), RAGGED)
    torch.cuda.synchronize()
    plan.check_error()
    check_batch(dtype, outs, hosts)


@pytest.mark.parametrize("dtype", ["cf16", "ci8"])
def test_ragged_batch_autotuned_variant(dtype, monkeypatch):
    """Without a forced variant the first call times each tile variant on the
    batch itself, keeps the fastest, and the final run's results are exact;
    with the autotuner off the size rule picks one; a forced one is kept."""
    from paper_1702_00844_gb300 import FLAG_NO_AUTOTUNE, Plan
    monkeypatch.delenv("CORR_TC_VARIANT", raising=False)
    for flags, want in ((0, None), (FLAG_NO_AUTOTUNE, None), (0, "wide")):
        if want:
            monkeypatch.setenv("CORR_TC_VARIANT", want)
        plan = Plan(1, 1, 1, dtype=dtype, path="tensor", flags=flags)
        assert plan.batch_tile_variant() is None
        xs, outs, hosts = make_batch(dtype)
        plan.correlate_batched(list(zip(xs, outs)), RAGGED)
        torch.cuda.synchronize()
        plan.check_error()
        picked = plan.batch_tile_variant()
        assert picked in ("narrow", "wide", "pair")
        if want:
            assert picked == want
        check_batch(dtype, outs, hosts)
        # a second call reuses the choice and the work list
        for o in outs:
            o.fill_(0)
        plan.correlate_batched(list(zip(xs, outs)), RAGGED)
        torch.cuda.synchronize()
        assert plan.batch_tile_variant() == picked
        check_batch(dtype, outs, hosts)


def test_ragged_batch_graph_replay():
    """The work list is built on the first call; later calls are captured in a
    CUDA graph and replayed with identical results."""
    from paper_1702_00844_gb300 import Plan
    plan = Plan(1, 1, 1, dtype="cf16", path="tensor")
    xs, outs, hosts = make_batch("cf16")
    pairs = list(zip(xs, outs))
    plan.correlate_batched(pairs, RAGGED)  # builds the work list (not captured)
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(float("nan"))
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.correlate_batched(pairs, RAGGED, stream=s)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    plan.check_error()
    check_batch("cf16", outs, hosts)


# ------------------------------------------------------------------ gains
def gain_case(S=16, C=3, T=128, seed=80):
    g = synth.rng(seed)
    x = synth.complex_normal(g, (C, S, T, 2))
    gains = (1 + synth.complex_normal(g, (C, S, 2), sigma=0.1)).astype(np.complex64)
    M = synth.sky_model(C, S, T, g).astype(np.complex64)
    return x, gains, M


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_gain_loss_and_gradients_vs_oracle():
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    x, gains, M = gain_case()
    C, S, T, _ = x.shape
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    loss = plan.gain_loss(R, gd, Md)
    grad_g, grad_x = plan.gain_backward(xd, gd, Md, R=R)
    # recompute path (no saved R) must agree
    grad_g2, grad_x2 = plan.gain_backward(xd, gd, Md, R=None)
    torch.cuda.synchronize()
    plan.check_error()
    Rref = oracle.correlate(x)
    Lref, _ = oracle.gain_loss(Rref, gains, M)
    gref = oracle.gain_grad(Rref, gains, M)
    xref = oracle.input_grad(x, Rref, gains, M)
    assert abs(float(loss) - Lref) < 1e-5 * Lref
    for got, ref in ((grad_g, gref), (grad_g2, gref), (grad_x, xref), (grad_x2, xref)):
        got = got.cpu().numpy().astype(np.complex128)
        assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


def test_gain_gradient_vs_finite_differences():
    """GPU dL/dg against FP64 central differences of the oracle's loss."""
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    x, gains, M = gain_case(S=6, C=2, T=64, seed=81)
    C, S, T, _ = x.shape
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    grad_g, _ = plan.gain_backward(xd, gd, Md, input_grad=False)
    torch.cuda.synchronize()
    Rref = oracle.correlate(x)
    g64 = gains.astype(np.complex128)
    fd = np.zeros_like(g64)
    h = 1e-6
    flat = g64.reshape(-1)
    for k in range(flat.size):
        for unit in (1.0, 1j):
            gp = flat.copy(); gm = flat.copy()
            gp[k] += h * unit
            gm[k] -= h * unit
            d = (oracle.gain_loss(Rref, gp.reshape(g64.shape), M)[0]
                 - oracle.gain_loss(Rref, gm.reshape(g64.shape), M)[0]) / (2 * h)
            fd.reshape(-1)[k] += d * unit
    got = grad_g.cpu().numpy().astype(np.complex128)
    assert np.abs(got - fd).max() < 1e-4 * np.abs(fd).max()


def test_autograd_function_matches_oracle():
    from paper_1702_00844_gb300 import FLAG_GAINS, GainCalibrationLoss, Plan
    x, gains, M = gain_case(S=20, C=2, T=96, seed=82)
    C, S, T, _ = x.shape
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd = _dev(x).requires_grad_(True)
    gd = _dev(gains).requires_grad_(True)
    Md = _dev(M)
    L = GainCalibrationLoss.apply(xd, gd, Md, plan)
    (3.0 * L).backward()
    torch.cuda.synchronize()
    Rref = oracle.correlate(x)
    gref = 3.0 * oracle.gain_grad(Rref, gains, M)
    xref = 3.0 * oracle.input_grad(x, Rref, gains, M)
    got_g = gd.grad.cpu().numpy().astype(np.complex128)
    got_x = xd.grad.cpu().numpy().astype(np.complex128)
    assert np.abs(got_g - gref).max() < 1e-4 * np.abs(gref).max()
    assert np.abs(got_x - xref).max() < 1e-4 * np.abs(xref).max()


def test_differentiation_workload_full_size():
    """64 stations, 64 channels, 1024 samples: loss and gradients against the
    oracle's closed form on sampled channels."""
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    d = synth.differentiation()
    x, gains, M = d["x"], d["g"], d["M"]
    C, S, T = d["C"], d["S"], d["T"]
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    grad_g, grad_x = plan.gain_backward(xd, gd, Md, R=R)
    torch.cuda.synchronize()
    for c in (0, 31, 63):
        Rref = oracle.correlate(x[c][None])
        gref = oracle.gain_grad(Rref, gains[c][None], M[c][None])
        xref = oracle.input_grad(x[c][None], Rref, gains[c][None], M[c][None])
        gg = grad_g[c].cpu().numpy().astype(np.complex128)[None]
        gx = grad_x[c].cpu().numpy().astype(np.complex128)[None]
        assert np.abs(gg - gref).max() < 1e-4 * np.abs(gref).max()
        assert np.abs(gx - xref).max() < 1e-4 * np.abs(xref).max()


def _input_grad(plan, xd, gd, Md, R, grad_x):
    """corr_gain_backward into a caller-given grad_x buffer."""
    import ctypes
    grad_g = torch.empty_like(gd)
    st = plan.L.corr_gain_backward(plan.h, ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(gd.data_ptr()),
                                   ctypes.c_void_p(Md.data_ptr()), ctypes.c_void_p(R.data_ptr()),
                                   ctypes.c_void_p(grad_g.data_ptr()), ctypes.c_void_p(grad_x.data_ptr()),
                                   None, None, None)
    assert st == 0, plan.L.corr_last_error_message()
    torch.cuda.synchronize()
    plan.check_error()
    return grad_x.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("S,C,T", [(8, 2, 64), (37, 2, 300), (70, 3, 700)])
def test_input_gradient_tensor_and_cuda_core_paths_vs_oracle(S, C, T, monkeypatch):
    """dL/dx on the tensor cores (the default for 16-byte aligned buffers:
    tf32 with each operand split into value and remainder; CTA pairs from two
    row tiles on), on single CTAs (CORR_IG_PATH=tc1) and on the CUDA cores
    (CORR_IG_PATH=cuda_core), all against the oracle. The shapes span one to
    three 128-row tiles of 4S (three: a pair whose second row tile is
    missing), a K block that 4S fills only in part (S = 37, 70) and a last
    time tile of fewer than 128 or 256 samples. 2e-5 of the largest element
    is FP32-class accuracy: one unsplit tf32 product would miss it by about
    two orders of magnitude."""
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    x, gains, M = gain_case(S, C, T, seed=90 + S)
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    Rref = oracle.correlate(x)
    xref = oracle.input_grad(x, Rref, gains, M)
    scale = np.abs(xref).max()
    got = {}
    for path in ("tensor", "tc1", "cuda_core"):
        if path == "tensor":
            monkeypatch.delenv("CORR_IG_PATH", raising=False)
        else:
            monkeypatch.setenv("CORR_IG_PATH", path)
        got[path] = _input_grad(plan, xd, gd, Md, R, torch.full_like(xd, float("nan")))
        assert np.isfinite(got[path]).all(), path
        assert np.abs(got[path] - xref).max() < 2e-5 * scale, path
    # the two paths round differently: equal bits would mean one did not run
    assert not np.array_equal(got["tensor"], got["cuda_core"])


def test_input_gradient_unaligned_buffers_take_the_cuda_core_path():
    """grad_x (or x) 8 bytes past a 16-byte boundary: the tensor path's TMA
    loads and 16-byte stores do not apply, the CUDA-core path runs and gives
    the same bits as CORR_IG_PATH=cuda_core on aligned buffers."""
    import os
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    S, C, T = 20, 2, 96
    x, gains, M = gain_case(S, C, T, seed=95)
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    xref = oracle.input_grad(x, oracle.correlate(x), gains, M)
    flat = torch.full((xd.numel() + 1,), float("nan"), dtype=torch.complex64, device="cuda")
    out = flat[1:].view(xd.shape)
    assert out.data_ptr() % 16 == 8
    unaligned = _input_grad(plan, xd, gd, Md, R, out)
    assert np.abs(unaligned - xref).max() < 2e-5 * np.abs(xref).max()
    xflat = torch.empty((xd.numel() + 1,), dtype=torch.complex64, device="cuda")
    x_off = xflat[1:].view(xd.shape)
    x_off.copy_(xd)
    unaligned_x = _input_grad(plan, x_off, gd, Md, R, torch.full_like(xd, float("nan")))
    os.environ["CORR_IG_PATH"] = "cuda_core"
    try:
        core = _input_grad(plan, xd, gd, Md, R, torch.full_like(xd, float("nan")))
    finally:
        del os.environ["CORR_IG_PATH"]
    assert np.array_equal(unaligned, core)
    assert np.array_equal(unaligned_x, core)


def test_input_gradient_beyond_65535_units(monkeypatch):
    """65541 channels of 2 stations: more units than a grid's z dimension
    holds, so both paths launch in chunks of 65535 units (sampled channels
    against the oracle, on both sides of the chunk boundary)."""
    from paper_1702_00844_gb300 import FLAG_GAINS, Plan
    S, C, T = 2, 65541, 16
    g = synth.rng(96)
    x = synth.complex_normal(g, (C, S, T, 2))
    gains = (1 + synth.complex_normal(g, (C, S, 2), sigma=0.1)).astype(np.complex64)
    M = synth.complex_normal(g, (C, S * (S + 1) // 2, 2, 2)).astype(np.complex64)
    plan = Plan(S, C, T, dtype="cf32", path="fp32", flags=FLAG_GAINS)
    xd, gd, Md = _dev(x), _dev(gains), _dev(M)
    R = plan.correlate(xd)
    for path in ("tensor", "tc1", "cuda_core"):
        if path == "tensor":
            monkeypatch.delenv("CORR_IG_PATH", raising=False)
        else:
            monkeypatch.setenv("CORR_IG_PATH", path)
        gx = _input_grad(plan, xd, gd, Md, R, torch.full_like(xd, float("nan")))
        assert np.isfinite(gx).all(), path
        for c in (0, 65534, 65535, C - 1):
            Rref = oracle.correlate(x[c][None])
            xref = oracle.input_grad(x[c][None], Rref, gains[c][None], M[c][None])
            assert np.abs(gx[c][None] - xref).max() < 2e-5 * np.abs(xref).max(), (path, c)


def test_ragged_int8_batch_with_extreme_subarray_takes_redo_path(monkeypatch):
    """One sub-array of all +-127 samples (station power above 2^24) in a
    batch with T > 512: its tiles fail the power check and are recomputed in
    exact 512-sample chunks, the others are accepted unchunked; all exact."""
    from paper_1702_00844_gb300 import Plan
    shapes = [(70, 2, 1024), (130, 1, 640), (33, 3, 1500)]
    xs, outs, hosts = [], [], []
    for k, (S, C, T) in enumerate(shapes):
        g = synth.rng(71, k)
        if k == 2:
            h = np.where(g.random((C, S, T, 2, 2)) < 0.5, -127, 127).astype(np.int8)
        else:
            h = synth.int8_normal(g, (C, S, T, 2))
        hosts.append(h)
        xs.append(torch.from_numpy(h).cuda())
        outs.append(torch.full((C, S * (S + 1) // 2, 2, 2, 2), 0x7FFFFFFF, dtype=torch.int32,
                               device="cuda"))
    for variant in ("narrow", "wide", "pair"):
        monkeypatch.setenv("CORR_TC_VARIANT", variant)
        plan = Plan(1, 1, 1, dtype="ci8", path="tensor")
        plan.correlate_batched(list(zip(xs, outs)), shapes)
        torch.cuda.synchronize()
        plan.check_error()
        for (S, C, T), o, h in zip(shapes, outs, hosts):
            ref = oracle.correlate(h, "ci8")
            got = to_numpy_int(o)
            np.testing.assert_array_equal(got[..., 0], ref.real.astype(np.int64))
            np.testing.assert_array_equal(got[..., 1], ref.imag.astype(np.int64))


def test_batching_workload_full_size_sampled():
    """The 32-sub-array ragged batch at full size (about 52 GB of f16
    samples) in the benchmark's launch configuration: one persistent launch,
    captured in a CUDA graph and replayed, with the tile variant the batch
    heuristic picks. One sampled channel of every sub-array is compared with
    the oracle on the same f16 values (relative Frobenius norm and, element
    by element, the correlation-coefficient error), and every
    channel's XX/YY autocorrelations are checked positive with an imaginary
    part at FP32 rounding level (the +a_i a_r and -a_r a_i terms are summed
    in different MMA steps)."""
    from paper_1702_00844_gb300 import Plan
    shapes = synth.batching_shapes()
    xs, outs = [], []
    for k, (S, C, T) in enumerate(shapes):
        xs.append(synth.batching_subarray_device(S, C, T, k, "cuda"))
        outs.append(torch.full((C, S * (S + 1) // 2, 2, 2), float("nan"), dtype=torch.complex64,
                               device="cuda"))
    plan = Plan(1, 1, 1, dtype="cf16", path="tensor")
    pairs = list(zip(xs, outs))
    plan.correlate_batched(pairs, shapes)
    torch.cuda.synchronize()
    for o in outs:
        o.fill_(float("nan"))
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.correlate_batched(pairs, shapes, stream=s)
    graph.replay()
    torch.cuda.synchronize()
    plan.check_error()
    rng = np.random.default_rng(4)
    for k, ((S, C, T), x, o) in enumerate(zip(shapes, xs, outs)):
        c = int(rng.integers(0, C))
        ref = oracle.correlate(x[c:c + 1].cpu().numpy(), "cf16")
        got = o[c:c + 1].cpu().numpy().astype(np.complex128)
        assert np.isfinite(got).all(), k
        assert rel_frobenius_per_unit(got, ref).max() < tol_fp16(T), k
        assert coef_error(got, ref, S) < 1e-4, k
        auto = o[:, [s * (s + 1) // 2 + s for s in range(S)]]        # (C, S, 2, 2)
        xx_yy = torch.stack([auto[..., 0, 0], auto[..., 1, 1]], -1)
        assert bool((xx_yy.real > 0).all()), k
        assert bool((xx_yy.imag.abs() <= 1e-5 * xx_yy.real).all()), k
    del xs, outs, pairs, graph
    torch.cuda.empty_cache()
