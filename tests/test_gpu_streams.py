"""Work on several streams at once: device errors are reported per stream,
concurrent trace launches never share a work queue, and a host-buffer wait
covers the payload downloads of earlier submissions.

Failures are made without a GPU fault: the look-back self-test runs a real
bounded wait out on a word nothing publishes.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu


def _flags(stream):
    out = torch.zeros(1, dtype=torch.int32).pin_memory()
    rr.rr_stream_error(out, stream=stream)
    stream.synchronize()
    return int(out.item())


def test_stream_error_words_are_per_stream():
    """The look-back self-test on stream A while a clean sort runs on stream B:
    only A's word carries the time-out flag; B's sort is exact; reading a word
    clears it; a device-memory output works as well as a pinned one."""
    assert rr.rr_device_error() == 0
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    n = 1 << 21
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64)
    kt = torch.from_numpy(keys.view(np.int64)).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = rr.sort_workspace(n, 64, 8)
    torch.cuda.synchronize()
    with torch.cuda.stream(b):
        for _ in range(4):
            rr.rr_sort(kt, None, perm, n, 64, 8, ws, stream=b)
    rr.rr_selftest_lookback_timeout(stream=a)  # synchronises a
    b.synchronize()
    assert _flags(a) == rr.RR_DEVERR_LOOKBACK_TIMEOUT
    assert _flags(a) == 0  # read and cleared
    dev_out = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    rr.rr_stream_error(dev_out, stream=b)
    b.synchronize()
    assert int(dev_out.item()) == 0
    assert np.array_equal(rr.u32_to_numpy(perm), oracle.stable_sort(keys)[0])
    # the device-wide read sees nothing left over
    assert rr.rr_device_error() == 0


def test_stream_error_refuses_pageable_output():
    with pytest.raises(rr.RRError):
        rr.rr_stream_error(torch.zeros(1, dtype=torch.int32))


def test_device_error_collects_every_stream():
    s = torch.cuda.Stream()
    rr.rr_selftest_lookback_timeout(stream=s)
    assert rr.rr_device_error() == rr.RR_DEVERR_LOOKBACK_TIMEOUT
    assert _flags(s) == 0


def test_served_requests_report_no_device_flags():
    tris = W.scene_box_soup(seed=3, n_random=512)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    srv = rr.Server(budget_bytes=1 << 28, slots=2)
    sid = srv.add_scene(bvh, lo, hi)
    # a failure on another stream before the requests does not touch them
    rr.rr_selftest_lookback_timeout(stream=torch.cuda.Stream())
    rays = [W.rays_box_soup(tris, n=m, seed=30 + m) for m in (1000, 5000, 20000)]
    outs = [np.zeros((len(r), 4), np.float32) for r in rays]
    tickets = [srv.submit(sid, r.o_tmin, r.d_tmax, h) for r, h in zip(rays, outs)]
    for t, r, h in zip(tickets, rays, outs):
        tm = srv.wait(t)
        assert tm["device_flags"] == 0
        oh, oi = oracle.trace_brute(tris, r.o_tmin, r.d_tmax)
        compare(tris, r.o_tmin, r.d_tmax, h, oh, oi)
    srv.close()
    assert rr.rr_device_error() == rr.RR_DEVERR_LOOKBACK_TIMEOUT


def test_trace_queues_not_shared_by_concurrent_launches():
    """A long trace on one stream while 4,100 small traces run on another: the
    small launches cycle through every work-queue pair, so one of them takes
    the long trace's pair while it still runs.  Every ray of every launch is
    traced exactly once (no hit left at its sentinel) and the hits match the
    oracle."""
    tris = W.scene_box_soup(seed=6)
    bvh = rr.BVH(tris)
    base = W.rays_box_soup(tris, n=1 << 20, seed=6)
    o1, d1, _ = rr.to_device_rays(base)
    reps = 160  # 168M rays: the long trace outlives the host-side launch loop below
    o_long, d_long = o1.repeat(reps, 1), d1.repeat(reps, 1)
    # sentinel: t = -1 (a hit has t > tmin >= 0 and a miss t = +inf)
    h_long = torch.full((o_long.shape[0], 4), -1.0, device="cuda")
    small = W.rays_box_soup(tris, n=64 * 4100, seed=7)
    os_, ds_, _ = rr.to_device_rays(small)
    h_small = torch.full((os_.shape[0], 4), -1.0, device="cuda")
    a, b = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    L = rr.lib()
    po, pd, ph, sb = os_.data_ptr(), ds_.data_ptr(), h_small.data_ptr(), b.cuda_stream
    rr.rr_trace(bvh, o_long, d_long, h_long, stream=a)
    for k in range(4100):  # the C entry point directly: a short host loop
        assert L.rr_trace(bvh.handle, po + 1024 * k, pd + 1024 * k, 64, ph + 1024 * k, sb) == 0
    torch.cuda.synchronize()
    assert rr.rr_device_error() == 0
    g_long = h_long.cpu().numpy()
    assert not (g_long[:, 0] == -1.0).any()
    g_small = h_small.cpu().numpy()
    assert not (g_small[:, 0] == -1.0).any()
    obvh = oracle.BVH(tris)
    oh, oi = obvh.trace(small.o_tmin, small.d_tmax)
    compare(tris, small.o_tmin, small.d_tmax, g_small, oh, oi)
    # the long trace: every repetition of the base rays gives the same bytes,
    # and a sample of them matches the oracle
    first = g_long[: 1 << 20]
    for r in range(1, reps):
        assert np.array_equal(g_long[r << 20:(r + 1) << 20].view(np.uint32), first.view(np.uint32)), r
    idx = np.sort(np.random.default_rng(1).choice(1 << 20, 30000, replace=False))
    oh, oi = obvh.trace(base.o_tmin[idx], base.d_tmax[idx])
    compare(tris, base.o_tmin[idx], base.d_tmax[idx], first[idx], oh, oi)


def test_pipeline_wait_covers_earlier_payload_downloads():
    """Submissions with and without payloads alternate; waiting only for the
    last one covers the payload downloads of every earlier one."""
    tris = W.scene_box_soup(seed=8, n_random=1024)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    params = rr.key_params(rr.RR_KEY_AILA, 32, lo, hi)
    n = 200000
    pipe = rr.Pipeline(bvh, n, params, radix_bits=8)
    waves = [W.rays_box_soup(tris, n=n, seed=80 + j) for j in range(6)]
    ref = []
    for r in waves:
        h, q = np.zeros((n, 4), np.float32), np.zeros(n, np.int32)
        pipe.run_host(r.o_tmin, r.d_tmax, r.payload, h, q)
        ref.append(q.copy())
    inputs = [(torch.from_numpy(r.o_tmin).pin_memory(), torch.from_numpy(r.d_tmax).pin_memory(),
               torch.from_numpy(r.payload.view(np.int32)).pin_memory()) for r in waves]
    for trial in range(3):
        outs, hits, tickets = [], [], []
        for j, (o, d, p) in enumerate(inputs):
            pay = j % 2 == 0
            h = torch.zeros(n, 4).pin_memory()
            q = torch.full((n,), -1, dtype=torch.int32).pin_memory() if pay else None
            outs.append(q)
            hits.append(h)  # the buffers stay alive until the wait below
            tickets.append(pipe.submit_host(o, d, p if pay else None, h, q))
        pipe.wait(tickets[-1])  # a submission without payloads
        for j, q in enumerate(outs):
            if q is not None:
                assert np.array_equal(q.numpy(), ref[j]), (trial, j)
    assert rr.rr_device_error() == 0
    pipe.close()
