"""Failure detection on the GPU without a fault: bounded waits give up and
report through the device error word; the context stays usable.

The look-back self-test launches the second tile of a sort pass alone, so its
wait on the first tile's published counts runs out (a flag nothing sets).
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr

pytestmark = pytest.mark.gpu


def test_lookback_wait_runs_out_and_is_reported():
    assert rr.rr_device_error() == 0
    t0 = time.time()
    rr.rr_selftest_lookback_timeout()
    dt = time.time() - t0
    assert rr.rr_device_error() == rr.RR_DEVERR_LOOKBACK_TIMEOUT
    assert rr.rr_device_error() == 0  # reading clears the word
    assert dt < 30.0
    # the device still sorts correctly afterwards
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 2**63, size=100000, dtype=np.uint64)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    perm = torch.empty(100000, dtype=torch.int32, device="cuda")
    rr.rr_sort(kt, None, perm, 100000, 64, 8, rr.sort_workspace(100000, 64, 8))
    assert np.array_equal(rr.u32_to_numpy(perm), oracle.stable_sort(keys)[0])
    assert rr.rr_device_error() == 0
