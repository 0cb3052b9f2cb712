"""GPU parity of the cheaper reorderings (Section 3.2 local sort, Section 4.4.1
indirect ray access) and of the any-hit kernel for shadow rays (Section 4).

Local sort: the permutation must equal the oracle's segment-wise stable sort bit
for bit.  Indirect access: the hits must equal, bit for bit, those of the same
kernel run on the gathered rays (the arithmetic per ray is identical), and the
oracle's closest hits under the usual rule.  Any-hit: occlusion must match the
oracle's closest-hit existence, and each reported triangle must really be met.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare, compare_any_hit

pytestmark = pytest.mark.gpu

SEGMENTS = [256, 512, 1024, 2048, 4096]


def _keys(n, bits, seed, dup=True):
    rng = np.random.default_rng(seed)
    if dup:  # few distinct values: long runs of equal keys exercise stability
        k = rng.integers(0, 64, size=n, dtype=np.uint64) * np.uint64(0x0123456789ABCDEF)
    else:
        k = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n,
                                                                                          dtype=np.uint64)
    if bits < 64:
        k &= np.uint64((1 << bits) - 1)
    return k


@pytest.mark.parametrize("segment", SEGMENTS)
@pytest.mark.parametrize("bits", [1, 16, 32, 33, 64])
@pytest.mark.parametrize("n", [1, 255, 4096 * 3 + 17, 100000])
def test_segment_sort_matches_oracle(segment, bits, n):
    keys = _keys(n, bits, seed=n + bits + segment, dup=(bits % 2 == 0))
    kt = torch.from_numpy(keys.astype(np.uint32 if bits <= 32 else np.uint64).view(
        np.int32 if bits <= 32 else np.int64)).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    kout = torch.empty_like(kt)
    rr.rr_sort_segments(kt, kout, perm, n, bits, segment)
    ref = oracle.segment_sort(keys, segment)
    assert np.array_equal(rr.u32_to_numpy(perm), ref)
    assert np.array_equal(rr.keys_to_numpy(kout), keys[ref])
    assert rr.rr_device_error() == 0


def test_segment_sort_rejects_bad_arguments():
    k = torch.zeros(16, dtype=torch.int32, device="cuda")
    p = torch.zeros(16, dtype=torch.int32, device="cuda")
    for seg in (0, 100, 8192):
        with pytest.raises(rr.RRError):
            rr.rr_sort_segments(k, None, p, 16, 32, seg)
    with pytest.raises(rr.RRError):
        rr.rr_sort_segments(k, None, p, 16, 65, 1024)
    rr.rr_sort_segments(k, None, p, 0, 32, 1024)  # n = 0 is a no-op


@pytest.fixture(scope="module")
def soup():
    tris = W.scene_box_soup(seed=1)
    return tris, rr.BVH(tris), oracle.BVH(tris)


def _bitwise(a):
    return np.ascontiguousarray(a).view(np.uint32)


@pytest.mark.parametrize("kind", ["global", "local", "reverse"])
def test_indirect_trace_equals_gathered_trace(soup, kind):
    tris, bvh, obvh = soup
    rays = W.rays_box_soup(tris, n=65536 + 77, seed=4)
    lo, hi = W.scene_aabb(tris)
    keys = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi)
    n = len(rays)
    if kind == "global":
        perm = oracle.stable_sort(keys)[0]
    elif kind == "local":
        perm = oracle.segment_sort(keys, 2048)
    else:
        perm = np.arange(n - 1, -1, -1, dtype=np.uint32)
    o, d, _ = rr.to_device_rays(rays)
    pt = torch.from_numpy(perm.view(np.int32)).cuda()
    hits_ind = torch.empty(n, 4, device="cuda")
    rr.rr_trace_ex(bvh, o, d, hits_ind, order=pt)
    sub = rays.subset(perm)
    so, sd, _ = rr.to_device_rays(sub)
    hits_sorted = torch.empty(n, 4, device="cuda")
    rr.rr_trace(bvh, so, sd, hits_sorted)
    g_ind = hits_ind.cpu().numpy()
    assert np.array_equal(_bitwise(g_ind[perm]), _bitwise(hits_sorted.cpu().numpy()))
    h, info = obvh.trace(rays.o_tmin, rays.d_tmax)
    compare(tris, rays.o_tmin, rays.d_tmax, g_ind, h, info)
    assert rr.rr_device_error() == 0


def test_indirect_trace_accumulate_equals_gathered(soup):
    tris, bvh, _ = soup
    rays = W.rays_box_soup(tris, n=50000, seed=6)
    lo, hi = W.scene_aabb(tris)
    keys = oracle.compute_keys(oracle.AILA, 64, rays.o_tmin, rays.d_tmax, lo, hi)
    perm = oracle.stable_sort(keys)[0]
    o, d, _ = rr.to_device_rays(rays)
    t1, t2 = rr.LengthTable(lo, hi), rr.LengthTable(lo, hi)
    h1 = torch.empty(len(rays), 4, device="cuda")
    rr.rr_trace_ex(bvh, o, d, h1, order=torch.from_numpy(perm.view(np.int32)).cuda(), table=t1)
    so, sd, _ = rr.to_device_rays(rays.subset(perm))
    h2 = torch.empty(len(rays), 4, device="cuda")
    rr.rr_trace_accumulate(bvh, so, sd, h2, t2)
    assert np.array_equal(_bitwise(h1.cpu().numpy()[perm]), _bitwise(h2.cpu().numpy()))
    assert np.array_equal(t1.read(), t2.read())
    assert rr.rr_device_error() == 0


def test_indirect_bad_index_is_flagged_not_traced(soup):
    _, bvh, _ = soup
    rays = W.random_rays_in_box(1000, [0.1] * 3, [0.9] * 3, seed=2)
    o, d, _ = rr.to_device_rays(rays)
    order = np.arange(1000, dtype=np.uint32)
    order[10] = 1000      # out of range
    order[11] = 0xFFFFFFFF
    hits = torch.full((1000, 4), 7.0, device="cuda")
    rr.rr_trace_ex(bvh, o, d, hits, order=torch.from_numpy(order.view(np.int32)).cuda())
    assert rr.rr_device_error() == rr.RR_DEVERR_BAD_INDEX
    g = hits.cpu().numpy()
    assert np.all(g[10] == 7.0) and np.all(g[11] == 7.0)  # rays 10 and 11 were never traced
    assert np.all(g[12:, 3] != 7.0)


@pytest.mark.parametrize("indirect", [False, True])
def test_any_hit_shadow_rays(soup, indirect):
    tris, bvh, obvh = soup
    rays = W.shadow_rays(tris, 60000, seed=3, light_center=(0.5, 0.95, 0.5))
    o, d, _ = rr.to_device_rays(rays)
    n = len(rays)
    hits = torch.empty(n, 4, device="cuda")
    order = None
    if indirect:
        lo, hi = W.scene_aabb(tris)
        keys = oracle.compute_keys(oracle.OCTAHEDRON, 32, rays.o_tmin, rays.d_tmax, lo, hi)
        order = torch.from_numpy(oracle.stable_sort(keys)[0].view(np.int32)).cuda()
    rr.rr_trace_ex(bvh, o, d, hits, order=order, flags=rr.RR_TRACE_ANY_HIT)
    h, info = obvh.trace(rays.o_tmin, rays.d_tmax)
    res = compare_any_hit(tris, rays.o_tmin, rays.d_tmax, hits.cpu().numpy(), h, info)
    assert 0.2 < res["occluded"] / n < 0.95, res
    assert rr.rr_device_error() == 0


def test_any_hit_on_terrain_and_unoccluded_light():
    tris = W.scene_terrain(seed=2, cells_x=64, cells_z=128, n_boxes=200)
    rays = W.shadow_rays(tris, 40000, seed=9)
    bvh = rr.BVH(tris)
    o, d, _ = rr.to_device_rays(rays)
    hits = torch.empty(len(rays), 4, device="cuda")
    rr.rr_trace_ex(bvh, o, d, hits, flags=rr.RR_TRACE_ANY_HIT)
    h, info = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    compare_any_hit(tris, rays.o_tmin, rays.d_tmax, hits.cpu().numpy(), h, info)
    # rays that end before reaching anything: tmax tiny
    short = W.Rays(rays.o_tmin.copy(), rays.d_tmax.copy(), rays.payload)
    short.d_tmax[:, 3] = 2e-4
    o2, d2, _ = rr.to_device_rays(short)
    rr.rr_trace_ex(bvh, o2, d2, hits, flags=rr.RR_TRACE_ANY_HIT)
    h2, info2 = oracle.BVH(tris).trace(short.o_tmin, short.d_tmax)
    compare_any_hit(tris, short.o_tmin, short.d_tmax, hits.cpu().numpy(), h2, info2)
    assert rr.rr_device_error() == 0


def test_any_hit_rejects_table(soup):
    tris, bvh, _ = soup
    lo, hi = W.scene_aabb(tris)
    t = rr.LengthTable(lo, hi)
    x = torch.zeros(4, 4, device="cuda")
    h = torch.zeros(4, 4, device="cuda")
    with pytest.raises(rr.RRError):
        rr.rr_trace_ex(bvh, x, x.clone(), h, flags=rr.RR_TRACE_ANY_HIT, table=t)
    with pytest.raises(rr.RRError):
        rr.rr_trace_ex(bvh, x, x.clone(), h, flags=0x10)
