"""sl_norms_static, the allocation-free variant of sl_norms.

Some callers cannot let a library allocate device memory: code running while a
stream is captured into a CUDA graph, and applications whose device memory all
comes from their own pool.  sl_norms_static keeps its scratch in a fixed array
compiled into the library and writes its results to the caller's device buffer.
This file is collected last on purpose so that a run stopping at the first
failure has already run every other test; it also passes on its own.
"""
import numpy as np
import pytest
import torch

from paper_1606_06117_gb300 import _lib as sl

pytestmark = pytest.mark.gpu


def test_static_norms_match_sl_norms_on_consecutive_calls():
    sl.load()
    dev = "cuda"
    out = torch.zeros(3, dtype=torch.float64, device=dev)
    cases = [
        (torch.randn(40, 50, 60, device=dev), torch.randn(40, 50, 60, device=dev), sl.F32),
        (torch.randn(1_000_003, dtype=torch.float64, device=dev),
         torch.randn(1_000_003, dtype=torch.float64, device=dev), sl.F64),
    ]
    for a, b, dt in cases:          # two calls in a row share the one scratch array
        sl.sl_norms_static(a, b, a.numel(), dt, out)
        torch.cuda.synchronize()
        ref = sl.sl_norms(a, b, a.numel(), dt)
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=0)


def test_static_norms_reject_bad_sizes():
    sl.load()
    a = torch.zeros(4, device="cuda")
    out = torch.zeros(3, dtype=torch.float64, device="cuda")
    for n in (0, (1 << 40) + 1):
        with pytest.raises(sl.SLError) as e:
            sl.sl_norms_static(a, a, n, sl.F32, out)
        assert e.value.code == -1 and "2^40" in str(e.value)
