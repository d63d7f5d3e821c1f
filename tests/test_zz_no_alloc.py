"""The allocation-free ordering entry point against the regular one.

vl_causal_order_noalloc serves callers that cannot allocate device memory at
the moment they need the causal order: frameworks and serving runtimes that own
all device memory through their own pooling allocator, and latency-bound loops
that must not pay for the device synchronisation an allocation implies.  It
keeps its scratch in a fixed device array inside the library instead of a
workspace.
Its results must equal those of vl_causal_order.  This file is named so that
pytest collects it last.
"""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _regular(vl, h, D):
    m = D.shape[0]
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    gap = torch.empty(m, dtype=torch.float64, device="cuda")
    vl.vl_causal_order(h, D, order, gap)
    h.sync()
    return order, gap


def test_noalloc_order_matches_regular_entry_on_consecutive_calls(vl):
    h = vl.Handle(0)
    rng = np.random.default_rng(2024)
    # calls in a row on one scratch array: each later one is smaller, so it
    # runs over what the earlier ones left behind; m = 512 fills the array
    # exactly
    for m in (512, 400, 37):
        A = rng.normal(size=(m, m))
        D = torch.from_numpy(A - A.T).cuda()
        ref_order, ref_gap = _regular(vl, h, D)
        order = torch.full((m,), -1, dtype=torch.int32, device="cuda")
        gap = torch.full((m,), math.nan, dtype=torch.float64, device="cuda")
        vl.vl_causal_order_noalloc(D, order, gap)
        torch.cuda.current_stream().synchronize()
        assert torch.equal(order, ref_order)
        fin = torch.isfinite(ref_gap)
        assert torch.equal(torch.isfinite(gap), fin)
        err = (gap[fin] - ref_gap[fin]).abs().max().item() if bool(fin.any()) else 0.0
        assert err <= 1e-12
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(vl):
    m = 513
    D = torch.zeros((m, m), dtype=torch.float64, device="cuda")
    order = torch.empty(m, dtype=torch.int32, device="cuda")
    with pytest.raises(vl.VLError) as ei:
        vl.vl_causal_order_noalloc(D, order)
    assert ei.value.code == 9  # VL_ERR_UNSUPPORTED
