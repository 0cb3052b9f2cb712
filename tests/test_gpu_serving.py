"""GPU tests of the serving loop (continuous batching of ray-batch requests).

The same requests are answered one at a time (one slot, one request in the
server) and all together under a small memory budget (several slots, requests
queued, grouped and overlapped): every hit must be the same bit for bit, and
correct against the oracle under the trace rule.  With the adaptive estimate
the length tables end identical too (integer sums of the same hits).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu

SIZES = [1, 700, 5000, 30000, 2, 12000, 64, 50000, 4097, 900, 25000, 333]


@pytest.fixture(scope="module")
def scenes():
    tris = [W.scene_box_soup(seed=1),
            W.scene_terrain(seed=6, cells_x=64, cells_z=128, n_boxes=200),
            W.scene_terrain(seed=7, cells_x=48, cells_z=96, n_boxes=100)]
    reqs = []
    for k, n in enumerate(SIZES):
        s = k % 3
        kind = "glossy" if k % 5 in (1, 3) else "diffuse"
        r = W.request_rays(tris[s], n, kind, seed=300 + k)
        reqs.append((s, r))
    return tris, [rr.BVH(t) for t in tris], [W.scene_aabb(t) for t in tris], reqs


def _server(scenes, budget, slots, tsrc=rr.RR_T_FIXED, tables=None, upload=rr.RR_UPLOAD_ADAPTIVE):
    tris, bvhs, boxes, _ = scenes
    srv = rr.Server(budget_bytes=budget, slots=slots, max_batch_rays=1 << 20, t_source=tsrc, key_bits=32,
                    upload=upload)
    for s in range(3):
        sid = srv.add_scene(bvhs[s], boxes[s][0], boxes[s][1], tables[s] if tables else None)
        assert sid == s
    return srv


def _run(srv, reqs):
    hits = [np.zeros((r.o_tmin.shape[0], 4), np.float32) for _, r in reqs]
    tickets = [srv.submit(s, r.o_tmin, r.d_tmax, h) for (s, r), h in zip(reqs, hits)]
    times = [srv.wait(t) for t in tickets]
    return hits, times


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("adaptive", [False, True])
def test_results_same_alone_and_in_the_mix(scenes, adaptive):
    tris, bvhs, boxes, reqs = scenes
    tsrc = rr.RR_T_ADAPTIVE if adaptive else rr.RR_T_FIXED
    tabs_a = [rr.LengthTable(*boxes[s]) for s in range(3)] if adaptive else None
    tabs_m = [rr.LengthTable(*boxes[s]) for s in range(3)] if adaptive else None
    # alone: one slot, each request waited for before the next is submitted
    srv = _server(scenes, budget=1 << 30, slots=1, tsrc=tsrc, tables=tabs_a)
    alone = []
    for sr in reqs:
        h, t = _run(srv, [sr])
        assert t[0]["batch_requests"] == 1
        alone.append(h[0])
    srv.close()
    # in the mix: every request submitted at once; a budget for about two
    # requests' worth of memory forces queuing and grouping
    budget = 6 << 20
    srv = _server(scenes, budget=budget, slots=3, tsrc=tsrc, tables=tabs_m)
    mixed, times = _run(srv, reqs)
    st = srv.stats()
    srv.close()
    assert st["peak_reserved_bytes"] <= budget and st["reserved_bytes"] == 0 and st["waiting"] == 0
    assert st["batches"] < len(reqs) and st["max_batch_requests"] > 1
    for a, m in zip(alone, mixed):
        assert np.array_equal(_bits(a), _bits(m))
    for t in times:
        assert t["submit_ns"] <= t["start_ns"] <= t["done_ns"]
    # correct, not only consistent
    for (s, r), h in zip(reqs, mixed):
        oh, oi = oracle.BVH(tris[s]).trace(r.o_tmin, r.d_tmax)
        compare(tris[s], r.o_tmin, r.d_tmax, h, oh, oi)
    if adaptive:
        for ta, tm in zip(tabs_a, tabs_m):
            sa, ca = ta.read()
            sm, cm = tm.read()
            assert np.array_equal(sa, sm) and np.array_equal(ca, cm)
            assert ca.sum() > (1 << 20)  # hits were added
    assert rr.rr_device_error() == 0


def test_requests_arriving_while_others_run(scenes):
    """Submissions interleaved with waits: later requests join while earlier
    groups are on the device; pinned host tensors as buffers.  The rays go up
    through the copy engines, through the library's copy kernel, and by the
    adaptive choice: the hits are the same bit for bit and correct."""
    tris, bvhs, boxes, reqs = scenes
    pinned = []
    for s, r in reqs:
        o = torch.from_numpy(r.o_tmin).pin_memory()
        d = torch.from_numpy(r.d_tmax).pin_memory()
        pinned.append((s, o, d))
    results = {}
    for upload in (rr.RR_UPLOAD_ENGINES, rr.RR_UPLOAD_KERNEL, rr.RR_UPLOAD_ADAPTIVE):
        srv = _server(scenes, budget=64 << 20, slots=2, upload=upload)
        hits = [torch.zeros(o.shape[0], 4).pin_memory() for _, o, _ in pinned]
        tickets, modes = [], []
        for k, ((s, o, d), h) in enumerate(zip(pinned, hits)):
            tickets.append(srv.submit(s, o, d, h))
            if k % 4 == 3:
                modes.append(srv.wait(tickets[k - 2])["kernel_copies"])
                tickets[k - 2] = None
        for t in tickets:
            if t is not None:
                modes.append(srv.wait(t)["kernel_copies"])
        st = srv.stats()
        srv.close()
        if upload == rr.RR_UPLOAD_ENGINES:
            assert set(modes) == {0} and st["kernel_copy_groups"] == 0
        elif upload == rr.RR_UPLOAD_KERNEL:
            assert set(modes) == {1} and st["kernel_copy_groups"] == st["batches"]
        results[upload] = [h.numpy().copy() for h in hits]
    for upload in (rr.RR_UPLOAD_KERNEL, rr.RR_UPLOAD_ADAPTIVE):
        for a, b in zip(results[rr.RR_UPLOAD_ENGINES], results[upload]):
            assert np.array_equal(_bits(a), _bits(b))
    for (s, r), h in zip(reqs, results[rr.RR_UPLOAD_KERNEL]):
        oh, oi = oracle.BVH(tris[s]).trace(r.o_tmin, r.d_tmax)
        compare(tris[s], r.o_tmin, r.d_tmax, h, oh, oi)
    with pytest.raises(rr.RRError):  # unknown policy
        rr.Server(budget_bytes=1 << 20, upload=3)
    assert rr.rr_device_error() == 0


def test_server_rejects_bad_requests(scenes):
    srv = _server(scenes, budget=1 << 20, slots=1)
    big = W.random_rays_in_box(200000, [0] * 3, [1] * 3, seed=1)
    h = np.zeros((200000, 4), np.float32)
    with pytest.raises(rr.RRError):  # more memory than the whole budget
        srv.submit(0, big.o_tmin, big.d_tmax, h)
    with pytest.raises(rr.RRError):  # unknown scene
        srv.submit(7, big.o_tmin[:10], big.d_tmax[:10], h[:10])
    with pytest.raises(rr.RRError):  # unknown ticket
        srv.wait(12345)
    t = srv.submit(1, big.o_tmin[:0], big.d_tmax[:0], h[:0])  # empty request
    srv.wait(t)
    srv.close()


def test_server_closes_with_requests_in_flight(scenes):
    """Closing the server finishes what was submitted and frees it, waited for or not."""
    tris, bvhs, boxes, reqs = scenes
    srv = _server(scenes, budget=64 << 20, slots=2)
    hits = [np.zeros((r.o_tmin.shape[0], 4), np.float32) for _, r in reqs]
    for (s, r), h in zip(reqs, hits):
        srv.submit(s, r.o_tmin, r.d_tmax, h)
    srv.close()  # no waits
    for (s, r), h in zip(reqs[:3], hits[:3]):
        oh, oi = oracle.BVH(tris[s]).trace(r.o_tmin, r.d_tmax)
        compare(tris[s], r.o_tmin, r.d_tmax, h, oh, oi)
    assert rr.rr_device_error() == 0
