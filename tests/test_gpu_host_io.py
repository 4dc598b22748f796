"""corr_correlate_host: host buffers streamed in chunks with the copies
overlapping the kernels must give exactly what corr_correlate gives on
device buffers (both kernel paths, several chunks and a ragged last chunk)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,S,C,T", [("ci8", 256, 300, 1024), ("cf16", 130, 200, 700),
                                          ("cf32", 64, 200, 768), ("ci8", 70, 3, 0)])
def test_host_streaming_equals_device_call(dtype, S, C, T):
    from paper_1702_00844_gb300 import FLAG_HOST_IO, Plan
    g = synth.rng(90, S + C)
    if dtype == "ci8":
        x = torch.from_numpy(synth.int8_normal(g, (C, S, T, 2)))
    elif dtype == "cf16":
        x = torch.from_numpy(synth.to_cf16(synth.complex_normal(g, (C, S, T, 2))))
    else:
        x = torch.from_numpy(synth.complex_normal(g, (C, S, T, 2)))
    plan = Plan(S, C, T, dtype=dtype, flags=FLAG_HOST_IO)
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


def test_host_streaming_requires_the_flag():
    from paper_1702_00844_gb300 import CorrError, Plan
    plan = Plan(8, 2, 16, dtype="cf32")
    x = torch.zeros((2, 8, 16, 2), dtype=torch.complex64)
    with pytest.raises(CorrError):
        plan.correlate_host(x)
