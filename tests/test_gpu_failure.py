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


# ------------------------------------------------------------------ injected host-side failures

def _soup():
    from paper_2506_11273_gb300 import workloads as W
    tris = W.scene_box_soup(seed=9, n_random=256)
    rays = W.rays_box_soup(tris, n=20000, seed=9)
    return W, tris, rays


def test_injected_allocation_failure_then_the_same_call_succeeds():
    W, tris, rays = _soup()
    rr.rr_fault_inject("alloc@1")
    with pytest.raises(rr.RRError) as e:
        rr.BVH(tris)
    assert e.value.status in (2, 3)  # RR_ERR_CUDA / RR_ERR_OOM
    bvh = rr.BVH(tris)  # the spec fired once: the retry builds
    o, d, _ = rr.to_device_rays(rays)
    hits = torch.empty(len(rays), 4, device="cuda")
    rr.rr_trace(bvh, o, d, hits)
    torch.cuda.synchronize()
    oh, _ = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    agree = np.mean(hits.cpu().numpy()[:, 3].view(np.uint32) == oh[:, 3].view(np.uint32))
    assert agree > 0.999
    assert rr.rr_device_error() == 0


def test_injected_launch_failure_leaves_the_pipeline_usable():
    W, tris, rays = _soup()
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    params = rr.key_params(rr.RR_KEY_AILA, 32, lo, hi)
    pipe = rr.Pipeline(bvh, len(rays), params, radix_bits=8)
    o, d, p = rr.to_device_rays(rays)
    hits = torch.empty(len(rays), 4, device="cuda")
    pout = torch.empty_like(p)
    rr.rr_fault_inject("launch@2")  # keys pass their check, the sort's is the second
    with pytest.raises(rr.RRError) as e:
        pipe.run(o, d, p, hits, pout)
    assert e.value.status == 2  # RR_ERR_CUDA
    torch.cuda.synchronize()
    pipe.run(o, d, p, hits, pout)
    torch.cuda.synchronize()
    keys = oracle.compute_keys(oracle.AILA, 32, rays.o_tmin, rays.d_tmax, lo, hi)
    perm, _ = oracle.stable_sort(keys)
    assert np.array_equal(rr.u32_to_numpy(pout), rays.payload[perm])
    pipe.close()
    assert rr.rr_device_error() == 0


def test_injected_wait_timeout_keeps_the_ticket():
    W, tris, rays = _soup()
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    srv = rr.Server(budget_bytes=1 << 28, slots=2)
    sid = srv.add_scene(bvh, lo, hi)
    h = np.zeros((len(rays), 4), np.float32)
    t = srv.submit(sid, rays.o_tmin, rays.d_tmax, h)
    rr.rr_fault_inject("timeout@1")
    with pytest.raises(rr.RRError) as e:
        srv.wait(t)
    assert e.value.status == 4  # RR_ERR_TIMEOUT
    srv.wait(t)  # still valid: the real wait returns the hits
    oh, _ = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    assert np.mean(h[:, 3].view(np.uint32) == oh[:, 3].view(np.uint32)) > 0.999
    srv.close()


def test_injected_group_allocation_failure_fails_only_that_request():
    W, tris, rays = _soup()
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    srv = rr.Server(budget_bytes=1 << 28, slots=1)
    sid = srv.add_scene(bvh, lo, hi)
    h1 = np.zeros((len(rays), 4), np.float32)
    h2 = np.zeros((len(rays), 4), np.float32)
    rr.rr_fault_inject("alloc@1")
    t1 = srv.submit(sid, rays.o_tmin, rays.d_tmax, h1)
    with pytest.raises(rr.RRError) as e:
        srv.wait(t1)
    assert e.value.status == 3  # RR_ERR_OOM
    t2 = srv.submit(sid, rays.o_tmin, rays.d_tmax, h2)
    srv.wait(t2)
    oh, _ = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    assert np.mean(h2[:, 3].view(np.uint32) == oh[:, 3].view(np.uint32)) > 0.999
    srv.close()
    rr.rr_fault_inject(None)


def test_bounds_checked_build_runs_clean():
    """The bounds-checked library (every kernel index checked against its
    buffer) runs the config-1 bounce, a batch and a served request with no
    flag set and the same results as the oracle; an out-of-range permutation
    entry is flagged and skipped there (child process, RR_LIBRARY=checked)."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    out = subprocess.run([sys.executable, os.path.join(here, "checked_run.py")], capture_output=True, text=True,
                         timeout=600, env={**os.environ, "RR_LIBRARY": "checked"})
    assert out.returncode == 0, out.stdout + out.stderr
    assert "checked library loaded" in out.stdout and "clean" in out.stdout, out.stdout
