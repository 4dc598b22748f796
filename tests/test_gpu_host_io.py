"""corr_correlate_host: host buffers streamed in chunks with the copies
overlapping the kernels must give exactly what corr_correlate gives on
device buffers (every kernel path, FP32 samples on the tensor cores
included; several chunks and a ragged last chunk),
and match the FP64 oracle on sampled channels (the first, one in the middle
and the last, so that the first, a middle and the ragged last chunk are
covered): bit for bit for int8, within the accumulation tolerances for f16
and FP32 samples."""
import numpy as np
import pytest

import oracle
import synth
from helpers import TOL_FP32, coef_error, rel_frobenius_per_unit, to_numpy_int, to_numpy_vis, tol_fp16

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,S,C,T,path", [("ci8", 256, 300, 1024, "auto"), ("cf16", 130, 200, 700, "auto"),
                                               ("cf32", 64, 200, 768, "auto"), ("ci8", 70, 3, 0, "auto"),
                                               ("cf32", 64, 200, 768, "tensor")])
def test_host_streaming_equals_device_call(dtype, S, C, T, path):
    from paper_1702_00844_gb300 import FLAG_HOST_IO, Plan
    g = synth.rng(90, S + C)
    if dtype == "ci8":
        x = torch.from_numpy(synth.int8_normal(g, (C, S, T, 2)))
    elif dtype == "cf16":
        x = torch.from_numpy(synth.to_cf16(synth.complex_normal(g, (C, S, T, 2))))
    else:
        x = torch.from_numpy(synth.complex_normal(g, (C, S, T, 2)))
    plan = Plan(S, C, T, dtype=dtype, path=path, flags=FLAG_HOST_IO)
    xh = x.contiguous().pin_memory()
    oh = plan.empty_out("cpu").pin_memory()
    plan.correlate_host(xh, oh)
    torch.cuda.synchronize()
    plan.check_error()
    ref = plan.correlate(x.cuda()).cpu()
    torch.cuda.synchronize()
    assert torch.equal(oh, ref)
    if T:
        assert bool((oh != 0).any())
    xs = x.numpy()
    for c in sorted({0, C // 2, C - 1}):
        want = oracle.correlate(xs[c][None], dtype)
        if dtype == "ci8":
            got = to_numpy_int(oh[0, c][None])
            np.testing.assert_array_equal(got[..., 0], want.real.astype(np.int64))
            np.testing.assert_array_equal(got[..., 1], want.imag.astype(np.int64))
        elif T:
            got = to_numpy_vis(oh[0, c][None], dtype)
            tol = tol_fp16(T) if dtype == "cf16" else TOL_FP32
            assert rel_frobenius_per_unit(got, want).max() < tol
            assert coef_error(got, want, S) < 1e-4


def test_host_streaming_requires_the_flag():
    from paper_1702_00844_gb300 import CorrError, Plan
    plan = Plan(8, 2, 16, dtype="cf32")
    x = torch.zeros((2, 8, 16, 2), dtype=torch.complex64)
    with pytest.raises(CorrError):
        plan.correlate_host(x)
