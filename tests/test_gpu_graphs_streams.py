"""Capture and concurrency: a single plan's int8 step (power-checked launches
and redo launches of both the pair and the tail lists, with their memsets)
captured in a CUDA graph and replayed, and plans of different paths running
at the same time on separate streams. Results stay exact (int8) or within
tolerance (FP32)."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP32, rel_frobenius_per_unit, to_numpy_int, to_numpy_vis

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def exact(out, x):
    ref = oracle.correlate(x, "ci8")
    got = to_numpy_int(out)
    np.testing.assert_array_equal(got[..., 0].reshape(ref.shape), ref.real.astype(np.int64))
    np.testing.assert_array_equal(got[..., 1].reshape(ref.shape), ref.imag.astype(np.int64))


@pytest.mark.parametrize("extreme", [False, True])
def test_int8_step_graph_capture_replay(monkeypatch, extreme):
    """150 stations (three blocks: pair tiles plus a narrow tail column) and
    1500 samples (power-checked path); with all-(+-127) samples every tile
    of both lists goes through its redo launch inside the graph."""
    from paper_1702_00844_gb300 import Plan
    monkeypatch.setenv("CORR_TC_VARIANT", "pair")
    S, C, T = 150, 3, 1500
    g = synth.rng(71, int(extreme))
    if extreme:
        x = np.where(g.random((C, S, T, 2, 2)) < 0.5, -127, 127).astype(np.int8)
    else:
        x = synth.int8_normal(g, (C, S, T, 2))
    plan = Plan(S, C, T, dtype="ci8", path="tensor")
    xd = torch.from_numpy(x).cuda()
    out = plan.empty_out()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        plan.correlate(xd, out, stream=s)
    for _ in range(2):
        out.fill_(0x7FFFFFFF)
        graph.replay()
        torch.cuda.synchronize()
        plan.check_error()
        exact(out, x)


def test_tensor_and_fp32_plans_on_concurrent_streams():
    from paper_1702_00844_gb300 import Plan
    g = synth.rng(72)
    S1, C1, T1 = 256, 16, 1024
    x8 = synth.int8_normal(g, (C1, S1, T1, 2))
    S2, C2, T2 = 100, 8, 512
    xc = synth.complex_normal(g, (C2, S2, T2, 2)).astype(np.complex64)
    p8 = Plan(S1, C1, T1, dtype="ci8", path="tensor")
    p32 = Plan(S2, C2, T2, dtype="cf32", path="fp32")
    a, b = torch.from_numpy(x8).cuda(), torch.from_numpy(xc).cuda()
    o8, o32 = p8.empty_out(), p32.empty_out()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    s1.wait_stream(torch.cuda.current_stream())
    s2.wait_stream(torch.cuda.current_stream())
    for _ in range(3):
        p8.correlate(a, o8, stream=s1)
        p32.correlate(b, o32, stream=s2)
    torch.cuda.synchronize()
    p8.check_error()
    p32.check_error()
    exact(o8, x8)
    ref = oracle.correlate(xc)
    got = o32.cpu().numpy().reshape(ref.shape)
    assert rel_frobenius_per_unit(got, ref).max() < TOL_FP32


@pytest.mark.parametrize("dtype,path", [("ci8", "tensor"), ("cf32", "fp32")])
def test_kernel_event_hook_brackets_the_main_launch(dtype, path):
    """corr_set_kernel_events: the events bracket the plan's main kernel,
    whose duration is positive and below that of the whole call (int8: the
    redo launch and its memsets stay outside); results are unchanged."""
    from paper_1702_00844_gb300 import Plan
    S, C, T = 256, 32, 1024
    g = synth.rng(73)
    if dtype == "ci8":
        x = synth.int8_normal(g, (C, S, T, 2))
    else:
        x = synth.complex_normal(g, (C, S, T, 2)).astype(np.complex64)
    plan = Plan(S, C, T, dtype=dtype, path=path)
    xd = torch.from_numpy(x).cuda()
    out = plan.empty_out()
    plan.correlate(xd, out)
    ka, kb, ca, cb = (torch.cuda.Event(enable_timing=True) for _ in range(4))
    for e in (ka, kb):
        e.record()
    torch.cuda.synchronize()
    plan.set_kernel_events(ka, kb)
    ca.record()
    plan.correlate(xd, out)
    cb.record()
    plan.set_kernel_events()
    torch.cuda.synchronize()
    plan.check_error()
    k_ms, c_ms = ka.elapsed_time(kb), ca.elapsed_time(cb)
    assert 0 < k_ms <= c_ms
    if dtype == "ci8":
        exact(out, x)
    else:
        ref = oracle.correlate(x)
        assert rel_frobenius_per_unit(out.cpu().numpy().reshape(ref.shape), ref).max() < TOL_FP32


@pytest.mark.parametrize("dtype,S,C,T", [("ci8", 150, 3, 1500), ("ci8", 64, 2, 256), ("cf16", 192, 5, 320)])
def test_back_to_back_calls_read_the_preceding_kernels_writes(monkeypatch, dtype, S, C, T):
    """The tensor path's launches are programmatic dependents of the kernel
    before them on the stream. Each call here follows, with no
    synchronisation, a copy kernel that rewrites its input, and precedes one
    that copies its output away; small grids (2 channels of 64 stations)
    leave most SMs free for an early start. Every call must see its own
    input: int8 exact, f16 against the oracle. 150 and 192 stations (three
    blocks) add the tail list's launches; 1500 int8 samples the power-checked
    launch and its redo launch."""
    from paper_1702_00844_gb300 import Plan
    monkeypatch.setenv("CORR_TC_VARIANT", "pair")
    g = synth.rng(91, S)
    if dtype == "ci8":
        xs = [synth.int8_normal(g, (C, S, T, 2)) for _ in range(3)]
        xs[2] = np.where(g.random((C, S, T, 2, 2)) < 0.5, -127, 127).astype(np.int8)  # every tile redone
    else:
        xs = [synth.to_cf16(synth.complex_normal(g, (C, S, T, 2))) for _ in range(3)]
    plan = Plan(S, C, T, dtype=dtype, path="tensor")
    src = [torch.from_numpy(x).cuda() for x in xs]
    x_dev = torch.empty_like(src[0])
    out = plan.empty_out()
    kept = []
    order = [0, 1, 2, 1, 0, 2, 2, 0]
    torch.cuda.synchronize()
    for k in order:
        x_dev.copy_(src[k])          # a kernel writing the input just before the call
        plan.correlate(x_dev, out)
        kept.append(out.clone())     # a kernel reading the output just after it
    torch.cuda.synchronize()
    plan.check_error()
    for k, o in zip(order, kept):
        if dtype == "ci8":
            exact(o, xs[k])
        else:
            ref = oracle.correlate(xs[k], "cf16")
            got = to_numpy_vis(o, "cf16").reshape(ref.shape)
            assert rel_frobenius_per_unit(got, ref).max() < 1e-5
