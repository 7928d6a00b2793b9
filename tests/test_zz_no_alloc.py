"""The allocation-free selection entry point, comet_scan_select_noalloc.

It serves callers that cannot allocate device memory (a process whose device memory belongs to a
caching allocator or a fixed budget, or one that cannot create a comet_ctx): it keeps its scratch
in a 1 MiB file-scope device array instead.  Checked here through the C ABI against
comet_scan_select on two calls in a row (the array is shared and keeps the previous call's
contents), plus its size limit.  Selection is index work, so the results must be identical.
This file is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_1911_09340_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _case(S, dtype, seed):
    rng = np.random.default_rng(seed)
    v = rng.integers(0, 64, size=S).astype(np.float64) * 0.25   # many ties
    v[rng.integers(0, S, size=3)] = np.nan
    return torch.as_tensor(v, dtype=dtype, device="cuda")


def test_noalloc_select_matches_select_on_two_calls(ctx):
    cases = [(_case(1 << 18, torch.float32, 1), 10), (_case(70001, torch.float64, 2), 64)]
    for rss, k in cases:
        ref_i = torch.full((k,), -1, dtype=torch.int64, device="cuda")
        ref_v = torch.zeros(k, dtype=rss.dtype, device="cuda")
        B.comet_scan_select(ctx, rss, k, ref_i, ref_v)
        got_i = torch.full((k,), -2, dtype=torch.int64, device="cuda")
        got_v = torch.zeros(k, dtype=rss.dtype, device="cuda")
        B.comet_scan_select_noalloc(rss, k, got_i, got_v)
        torch.cuda.synchronize()
        assert torch.equal(got_i, ref_i)
        assert np.array_equal(got_v.cpu().numpy(), ref_v.cpu().numpy(), equal_nan=True)


def test_noalloc_select_rejects_sizes_beyond_its_scratch():
    rss = torch.zeros(3 << 20, dtype=torch.float64, device="cuda")    # 3.1 M seeds, k = 64
    idx = torch.zeros(64, dtype=torch.int64, device="cuda")
    with pytest.raises(B.CometError, match="static scratch"):
        B.comet_scan_select_noalloc(rss, 64, idx)
