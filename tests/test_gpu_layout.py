"""corr_reorder on the GPU against the oracle's permutation: every pair of
layouts, every sample type, ragged sizes (not multiples of the 32 x 32
tile), several integrations, and the full 256-station int8 workload in both
directions the correlator needs (time-major and station-major into the
correlator's layout). Permutations are bit-exact."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

LAYOUTS = ("cst", "cts", "sct")


def host_samples(rng, shape_cst, dtype):
    if dtype == "cf32":
        return (rng.standard_normal(shape_cst) + 1j * rng.standard_normal(shape_cst)).astype(np.complex64)
    if dtype == "cf16":
        return rng.standard_normal(shape_cst + (2,)).astype(np.float16)
    return rng.integers(-128, 128, size=shape_cst + (2,)).astype(np.int8)


@pytest.mark.parametrize("dtype", ["cf32", "cf16", "ci8"])
@pytest.mark.parametrize("S,C,T,I", [(37, 3, 45, 2), (1, 1, 1, 1), (64, 2, 32, 1), (5, 7, 100, 1)])
def test_reorder_all_pairs_bit_exact(dtype, S, C, T, I):
    from paper_1702_00844_gb300 import reorder
    x_cst = host_samples(np.random.default_rng(S * 131 + T), (I, C, S, T, 2), dtype)
    host = {L: oracle.reorder(x_cst, "cst", L) for L in LAYOUTS}
    dev = {L: torch.from_numpy(host[L]).cuda() for L in LAYOUTS}
    for a in LAYOUTS:
        for b in LAYOUTS:
            got = reorder(dev[a], S, C, T, I, dtype, a, b)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), host[b])


def test_reorder_zero_samples_is_a_no_op():
    from paper_1702_00844_gb300 import reorder
    x = torch.zeros((1, 3, 4, 0, 2, 2), dtype=torch.int8, device="cuda")
    out = reorder(x, 4, 3, 0, 1, "ci8", "cst", "cts")
    assert out.numel() == 0


def test_reorder_full_precision_workload_then_correlate():
    """The 256-station x 480-channel x 1024-sample int8 workload: time-major and
    station-major copies reordered into the correlator's layout equal the
    original bit for bit, and the visibilities of the reordered samples equal
    those of the original."""
    from paper_1702_00844_gb300 import Plan, reorder
    S, C, T = 256, 480, 1024
    x = synth.precision_device(C, S, T, "cuda").view(1, C, S, T, 2, 2)
    x_host = x.cpu().numpy()
    for L in ("cts", "sct"):
        other = torch.from_numpy(oracle.reorder(x_host, "cst", L)).cuda()
        back = reorder(other, S, C, T, 1, "ci8", L, "cst")
        torch.cuda.synchronize()
        assert torch.equal(back, x)
        fwd = reorder(x, S, C, T, 1, "ci8", "cst", L)
        torch.cuda.synchronize()
        assert torch.equal(fwd, other)
        del other, back, fwd
    plan = Plan(S, 8, T, dtype="ci8", path="tensor")
    sub = x[0, :8].contiguous()
    via = reorder(reorder(sub.view(1, 8, S, T, 2, 2), S, 8, T, 1, "ci8", "cst", "sct"),
                  S, 8, T, 1, "ci8", "sct", "cst")
    a = plan.correlate(sub)
    b = plan.correlate(via.view_as(sub))
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_corner_turn_single_rank_is_the_local_reorder():
    """Without a process group the corner turn is the station-major ->
    correlator-layout permutation on the device."""
    from paper_1702_00844_gb300.shard import corner_turn
    S, C, T, I = 40, 6, 70, 2
    x_cst = host_samples(np.random.default_rng(3), (I, C, S, T, 2), "ci8")
    sct = torch.from_numpy(oracle.reorder(x_cst, "cst", "sct")).cuda()
    got = corner_turn(sct, S, C, T, I, "ci8")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(got.cpu().numpy(), x_cst)
