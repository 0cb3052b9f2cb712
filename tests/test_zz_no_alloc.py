"""rr_sort_noalloc: the sort entry point for callers that cannot allocate.

Callers that live inside another system's memory budget (a renderer whose
allocator owns all device memory, a frame loop that forbids cudaMalloc once it
runs) cannot hand rr_sort a workspace.  rr_sort_noalloc sorts with a fixed
scratch array that lives inside librr.so instead.  These tests call it through
the C ABI and check that it returns exactly what rr_sort returns.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_2506_11273_gb300 import rr

pytestmark = pytest.mark.gpu


def _keys(n, bits, seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    if bits < 64:
        k &= np.uint64((1 << bits) - 1)
    k[::7] = k[0]  # plenty of equal keys: stability matters
    if bits > 32:
        return torch.from_numpy(k.view(np.int64)).cuda()
    return torch.from_numpy(k.astype(np.uint32).view(np.int32)).cuda()


def _with_workspace(keys, n, bits, radix_bits):
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    out = torch.empty_like(keys)
    ws = rr.sort_workspace(n, bits, radix_bits)
    rr.rr_sort(keys, out, perm, n, bits, radix_bits, ws)
    torch.cuda.synchronize()
    return rr.u32_to_numpy(perm), rr.keys_to_numpy(out)


def _without_workspace(keys, n, bits, radix_bits):
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    out = torch.empty_like(keys)
    rr.rr_sort_noalloc(keys, out, perm, n, bits, radix_bits)
    torch.cuda.synchronize()
    return rr.u32_to_numpy(perm), rr.keys_to_numpy(out)


def test_noalloc_sort_matches_rr_sort_on_two_calls_in_a_row():
    # the largest accepted size first, then a smaller one with other key and
    # digit widths: the second call must not see the first call's scratch
    cases = [(rr.RR_SORT_NOALLOC_MAX_N, 64, 8, 1), (70001, 32, 4, 2)]
    for n, bits, radix_bits, seed in cases:
        keys = _keys(n, bits, seed)
        p_ref, k_ref = _with_workspace(keys, n, bits, radix_bits)
        p, k = _without_workspace(keys, n, bits, radix_bits)
        assert np.array_equal(p, p_ref)
        assert np.array_equal(k, k_ref)
        assert np.all(k[1:] >= k[:-1])
    # the calls' error word (inside the array) is read by rr_device_error
    assert rr.rr_device_error() == 0


def test_noalloc_sort_rejects_sizes_beyond_its_maximum():
    n = rr.RR_SORT_NOALLOC_MAX_N + 1
    keys = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(rr.RRError) as e:
        rr.rr_sort_noalloc(keys, None, perm, n, 32, 8)
    assert e.value.status == 7  # RR_ERR_TOO_LARGE
