"""GPU parity: BVH build + closest-hit trace, and the one-bounce pipeline.

Hits are compared with the oracle's binary64 closest hits under the rule in
hitcheck.py (same triangle, t within 1e-5 relative; ties and edge-grazing
rays classified).  The oracle BVH used for the larger scenes is itself pinned
to the brute-force definition in the CPU tests.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu


def gpu_trace(bvh, rays):
    o, d, _ = rr.to_device_rays(rays)
    hits = torch.empty(len(rays), 4, dtype=torch.float32, device="cuda")
    rr.rr_trace(bvh, o, d, hits)
    torch.cuda.synchronize()
    return hits.cpu().numpy()


def check(tris, rays, brute=False, or_bvh=None, max_ambiguous=None):
    bvh = rr.BVH(tris)
    g = gpu_trace(bvh, rays)
    if brute:
        h, info = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    else:
        h, info = (or_bvh or oracle.BVH(tris)).trace(rays.o_tmin, rays.d_tmax)
    res = compare(tris, rays.o_tmin, rays.d_tmax, g, h, info, max_ambiguous=max_ambiguous)
    assert rr.rr_device_error() == 0
    return res, g, h


def test_closed_form_box_interior():
    tris = W._box_tris(np.zeros(3), np.ones(3), inward=True).astype(np.float32)
    rays = W.random_rays_in_box(5000, [0.01] * 3, [0.99] * 3, seed=3)
    res, g, _ = check(tris, rays, brute=True)
    assert res["hit_rate"] == 1.0
    o = rays.o_tmin[:, :3].astype(np.float64)
    d = rays.d_tmax[:, :3].astype(np.float64)
    with np.errstate(divide="ignore"):
        tc = np.where(d != 0, (np.where(d > 0, 1.0, 0.0) - o) / d, np.inf)
    assert np.allclose(g[:, 0], tc.min(axis=1), rtol=1e-5, atol=0)


@pytest.mark.parametrize("n_tris", [0, 1, 2, 3, 4, 5, 8, 9, 33, 100])
def test_tiny_scenes_brute_force(n_tris):
    rng = np.random.default_rng(n_tris)
    tris = (rng.random((n_tris, 9)) * 2 - 0.5).astype(np.float32)
    rays = W.random_rays_in_box(4096, [-1] * 3, [2] * 3, seed=n_tris + 100)
    check(tris, rays, brute=True)


def test_box_soup_small_brute_force():
    tris = W.scene_box_soup(seed=4, n_random=512)
    rays = W.rays_box_soup(tris, n=8192, seed=4)
    res, _, _ = check(tris, rays, brute=True)
    assert res["hit_rate"] > 0.99


def test_interval_ends_and_degenerate_rays():
    tris = W.scene_box_soup(seed=5, n_random=256)
    rays = W.rays_box_soup(tris, n=4096, seed=5)
    o = rays.o_tmin.copy()
    d = rays.d_tmax.copy()
    o[:512, 3] = 0.3          # larger tmin
    d[512:1024, 3] = 0.05     # short tmax
    d[1024:1100, :3] = 0.0    # zero direction: no hit
    d[1100:1200, 0] = 0.0     # axis-parallel directions
    d[1200:1300, 1] = 0.0
    o[1300:1400, 3] = 5.0     # tmin > tmax: empty interval
    d[1300:1400, 3] = 1.0
    r = W.Rays(o, d, rays.payload)
    # axis-parallel rays that start on a wall of the unit box run inside the
    # wall's plane: coplanar, hence grazing/edge cases by construction
    res, _, _ = check(tris, r, brute=True, max_ambiguous=16)
    assert res["definite"] == 0


def test_degenerate_triangles_never_hit():
    tris = np.array([[0, 0, 0, 1, 1, 1, 2, 2, 2],        # collinear
                     [0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5, 0.5],  # a point
                     [0, 0, 0, 1, 0, 0, 0, 1, 0]], np.float32)
    rays = W.random_rays_in_box(4096, [-1] * 3, [2] * 3, seed=7)
    _, g, _ = check(tris, rays, brute=True)
    tri = g[:, 3].view(np.uint32)
    assert np.all((tri == 2) | (tri == rr.MISS))


def test_config1_full_65536_rays():
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=1)
    res, _, _ = check(tris, rays)
    assert res["hit_rate"] > 0.99


def test_trace_is_order_agnostic_and_deterministic():
    """The hit of each ray does not depend on where the ray sits in the buffer."""
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=2)
    bvh = rr.BVH(tris)
    g1 = gpu_trace(bvh, rays)
    g2 = gpu_trace(bvh, rays)
    assert np.array_equal(g1.view(np.uint32), g2.view(np.uint32))
    p = np.random.default_rng(1).permutation(len(rays))
    g3 = gpu_trace(bvh, rays.subset(p))
    assert np.array_equal(g3.view(np.uint32), g1[p].view(np.uint32))


def test_bvh_info_and_box():
    tris = W.scene_box_soup(seed=1)
    bvh = rr.BVH(tris)
    i = bvh.info()
    lo, hi = W.scene_aabb(tris)
    assert i.n_tris == tris.shape[0]
    assert list(i.aabb_lo) == list(lo) and list(i.aabb_hi) == list(hi)
    assert i.n_nodes > 0 and i.depth >= 2 and i.node_bytes == 80 * i.n_nodes
    with pytest.raises(rr.RRError):
        rr.BVH(np.array([[0, 0, 0, 1, np.nan, 0, 0, 1, 0]], np.float32))


def test_bvh_serialize_round_trip():
    """A reloaded BVH traces bit-identically to the built one, reports the same
    info, serializes to the same bytes, and damaged bytes are refused before
    anything is uploaded."""
    tris = W.scene_box_soup(seed=6)
    rays = W.rays_box_soup(tris, n=65536, seed=6)
    built = rr.BVH(tris)
    blob = built.serialize()
    i0 = built.info()
    assert len(blob) == 64 + 80 * i0.n_nodes + 48 * i0.n_tris + 32 * i0.n_tris
    loaded = rr.BVH(serialized=blob)
    i1 = loaded.info()
    for f in ("n_tris", "n_nodes", "n_leaves", "depth", "node_bytes", "tri_bytes"):
        assert getattr(i0, f) == getattr(i1, f), f
    assert list(i0.aabb_lo) == list(i1.aabb_lo) and list(i0.aabb_hi) == list(i1.aabb_hi)
    assert loaded.serialize() == blob
    g0 = gpu_trace(built, rays)
    g1 = gpu_trace(loaded, rays)
    assert np.array_equal(g0.view(np.uint32), g1.view(np.uint32))
    bad = bytearray(blob)
    bad[64 + 16: 64 + 20] = (i0.n_nodes + 5).to_bytes(4, "little")  # the root's first child past the end
    with pytest.raises(rr.RRError):
        rr.BVH(serialized=bytes(bad))
    with pytest.raises(rr.RRError):
        rr.BVH(serialized=blob[:-1])
    empty = rr.BVH(np.zeros((0, 9), np.float32))
    again = rr.BVH(serialized=empty.serialize())
    assert again.info().n_tris == 0 and len(empty.serialize()) == 64
    h = gpu_trace(again, rays.subset(np.arange(100)))
    assert np.all(np.isinf(h[:, 0]))
    assert rr.rr_device_error() == 0


@pytest.fixture(scope="module")
def terrain():
    tris = W.scene_terrain()
    return tris, rr.BVH(tris), oracle.BVH(tris)


def test_config2_full_size_sampled(terrain):
    """Full 1,168,576-triangle scene and full 2,073,600-ray wavefronts traced
    in one launch; 20,000 sampled rays compared with the oracle."""
    tris, bvh, obvh = terrain
    info = bvh.info()
    assert info.n_tris == tris.shape[0]
    rng = np.random.default_rng(11)
    for rays in (W.camera_rays(W.Camera()), W.surface_rays(tris, 2073600, seed=12)):
        g = gpu_trace(bvh, rays)
        idx = np.sort(rng.choice(len(rays), 20000, replace=False))
        sub = rays.subset(idx)
        h, inf = obvh.trace(sub.o_tmin, sub.d_tmax)
        compare(tris, sub.o_tmin, sub.d_tmax, g[idx], h, inf)
    assert rr.rr_device_error() == 0


def test_config2_secondary_rays_from_oracle_hits(terrain):
    """A path-tracer bounce built from oracle hits (no CUDA input): 50,000 rays."""
    tris, bvh, obvh = terrain
    cam = W.camera_rays(W.Camera()).subset(np.arange(0, 2073600, 41)[:50000])
    h1, _ = obvh.trace(cam.o_tmin, cam.d_tmax)
    sec = W.next_bounce(tris, cam, h1, 1, seed=2)
    g = gpu_trace(bvh, sec)
    h, inf = obvh.trace(sec.o_tmin, sec.d_tmax)
    res = compare(tris, sec.o_tmin, sec.d_tmax, g, h, inf)
    assert res["hit_rate"] > 0.5


# ------------------------------------------------------------------ one bounce

def oracle_bounce(tris, rays, lo, hi, layout, bits, tsrc, table=None, obvh=None):
    keys = oracle.compute_keys(layout, bits, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=tsrc, table=table)
    perm, _ = oracle.stable_sort(keys)
    o, d, p = oracle.permute(rays.o_tmin, rays.d_tmax, rays.payload, perm)
    h, info = (obvh or oracle.BVH(tris)).trace(o, d)
    if table is not None:
        table.accumulate(lo, hi, o, d, h)
    return keys, perm, o, d, p, h, info


def check_table_close(table, otable, ambiguous, exclude_cells=()):
    """The GPU table accumulates the GPU's fp32 hit distances and the oracle's
    table its binary64 ones, so cells agree to the trace tolerance: counts
    exactly (up to edge-ambiguous rays), sums within 1e-5 relative plus one
    fixed-point unit per ray.  exclude_cells: cells of edge-ambiguous rays,
    whose two hits may lie at different distances."""
    s, c = table.read()
    dc = c.astype(np.int64) - otable.cnt.astype(np.int64)
    assert np.abs(dc).sum() <= ambiguous
    same = dc == 0
    same[np.asarray(list(exclude_cells), np.int64)] = False
    added = otable.sum[same].astype(np.float64) - 4194304.0
    bound = 1e-5 * added + (otable.cnt[same].astype(np.float64) - 1.0) + 1.0
    diff = np.abs(s[same].astype(np.float64) - otable.sum[same].astype(np.float64))
    assert np.all(diff <= bound)


@pytest.mark.parametrize("name,layout,olayout,bits,tsrc,otsrc", [
    ("aila32", rr.RR_KEY_AILA, oracle.AILA, 32, rr.RR_T_FIXED, oracle.T_FIXED),
    ("tp64_fixed", rr.RR_KEY_TWO_POINT, oracle.TWO_POINT, 64, rr.RR_T_FIXED, oracle.T_FIXED),
    ("tp64_adaptive", rr.RR_KEY_TWO_POINT, oracle.TWO_POINT, 64, rr.RR_T_ADAPTIVE, oracle.T_ADAPTIVE),
])
def test_pipeline_matches_oracle_config1(name, layout, olayout, bits, tsrc, otsrc):
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=3)
    lo, hi = W.scene_aabb(tris)
    E = oracle.largest_extent(lo, hi)
    obvh = oracle.BVH(tris)
    bvh = rr.BVH(tris)
    adaptive = tsrc == rr.RR_T_ADAPTIVE
    table = rr.LengthTable(lo, hi) if adaptive else None
    params = rr.key_params(layout, bits, lo, hi, t_source=tsrc, table=table)
    pipe = rr.Pipeline(bvh, len(rays), params, radix_bits=8)
    o, d, p = rr.to_device_rays(rays)
    hits = torch.empty(len(rays), 4, device="cuda")
    pout = torch.empty_like(p)
    n = len(rays)
    # host entries: pageable buffers, page-locked buffers, page-locked hits at
    # an offset inside their allocation with pageable payloads (mixed)
    for entry in ("device", "host", "host_pinned", "host_mixed"):
        if adaptive:
            table.reset()
        otable = oracle.LengthTable(E) if adaptive else None
        if entry == "device":
            pipe.run(o, d, p, hits, pout)
            torch.cuda.synchronize()
            gh, gp = hits.cpu().numpy(), rr.u32_to_numpy(pout)
        elif entry == "host":
            gh = np.zeros((n, 4), np.float32)
            gp = np.zeros(n, np.uint32)
            pipe.run_host(rays.o_tmin, rays.d_tmax, rays.payload, gh, gp)
        elif entry == "host_pinned":
            ht = torch.zeros(n, 4).pin_memory()
            pt = torch.zeros(n, dtype=torch.int32).pin_memory()
            pipe.run_host(torch.from_numpy(rays.o_tmin).pin_memory(), torch.from_numpy(rays.d_tmax).pin_memory(),
                          torch.from_numpy(rays.payload.view(np.int32)).pin_memory(), ht, pt)
            gh, gp = ht.numpy().copy(), pt.numpy().view(np.uint32).copy()
        else:
            ht = torch.full((n + 3, 4), -7.0).pin_memory()
            gp = np.zeros(n, np.uint32)
            pipe.run_host(rays.o_tmin, rays.d_tmax, rays.payload, ht[1:n + 1], gp)
            whole = ht.numpy()
            assert (whole[0] == -7.0).all() and (whole[n + 1:] == -7.0).all(), "stores outside the hit range"
            gh = whole[1:n + 1].copy()
        keys, perm, so, sd, sp, h, info = oracle_bounce(tris, rays, lo, hi, olayout, bits, otsrc, otable, obvh)
        assert np.array_equal(gp, sp)  # payload order == oracle permutation
        if entry == "device":
            dev_hits = gh.copy()
        else:  # the host entry returns the device entry's hits, bit for bit
            assert np.array_equal(gh.view(np.uint32), dev_hits.view(np.uint32))
        res = compare(tris, so, sd, gh, h, info)
        if adaptive:
            check_table_close(table, otable, res["ambiguous"])
    assert rr.rr_device_error() == 0
    pipe.close()


def test_pipeline_submissions_in_flight_match_one_after_another():
    """Host submissions with two in flight (the upload of one overlapping the
    kernels of the one before) give the bytes of the same bounces run one after
    the other, with the adaptive table carried from bounce to bounce.  Page-locked
    and pageable output buffers, uneven sizes, and a ticket waited on twice."""
    tris = W.scene_box_soup(seed=2)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    sizes = [65536, 40001, 65536, 777]
    waves = [W.rays_box_soup(tris, n=m, seed=20 + j) for j, m in enumerate(sizes)]
    table = rr.LengthTable(lo, hi)
    params = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
    pipe = rr.Pipeline(bvh, max(sizes), params, radix_bits=8)

    def outputs(m, pinned):
        if pinned:
            return torch.zeros(m, 4).pin_memory(), torch.zeros(m, dtype=torch.int32).pin_memory()
        return np.zeros((m, 4), np.float32), np.zeros(m, np.int32)

    def as_np(x):
        return (x.numpy() if isinstance(x, torch.Tensor) else x).copy()

    table.reset()
    ref = []
    for r in waves:
        h, q = outputs(len(r), False)
        pipe.run_host(r.o_tmin, r.d_tmax, r.payload, h, q)
        ref.append((h.copy(), q.copy()))
    ref_table = table.read()

    table.reset()
    inputs = [(torch.from_numpy(r.o_tmin).pin_memory(), torch.from_numpy(r.d_tmax).pin_memory(),
               torch.from_numpy(r.payload.view(np.int32)).pin_memory()) for r in waves]
    outs = [outputs(len(r), pinned=(j != 1)) for j, r in enumerate(waves)]
    tickets = []
    for j, (o, d, p) in enumerate(inputs):
        tickets.append(pipe.submit_host(o, d, p, *outs[j]))
        if j >= 1:
            pipe.wait(tickets[j - 1])
    pipe.wait(tickets[-1])
    pipe.wait(tickets[0])  # long done: returns at once
    for j in range(len(waves)):
        h, q = as_np(outs[j][0]), as_np(outs[j][1])
        assert np.array_equal(h.view(np.uint32), ref[j][0].view(np.uint32)), j
        assert np.array_equal(q, ref[j][1]), j
    got_table = table.read()
    assert all(np.array_equal(a, b) for a, b in zip(got_table, ref_table))
    assert pipe.submit_host(waves[0].o_tmin, waves[0].d_tmax, None, np.zeros((0, 4), np.float32), None, n=0) == 0
    with pytest.raises(rr.RRError):
        pipe.wait(10 ** 6)
    assert rr.rr_device_error() == 0
    pipe.close()


def test_pipeline_rejects_bad_arguments():
    tris = W.scene_box_soup(seed=1, n_random=64)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    params = rr.key_params(rr.RR_KEY_AILA, 32, lo, hi)
    pipe = rr.Pipeline(bvh, 100, params)
    rays = W.rays_box_soup(tris, n=200, seed=1)
    o, d, p = rr.to_device_rays(rays)
    hits = torch.empty(200, 4, device="cuda")
    with pytest.raises(rr.RRError):
        pipe.run(o, d, p, hits, torch.empty_like(p))  # n > max_n
    with pytest.raises(rr.RRError):
        rr.Pipeline(bvh, 100, params, radix_bits=6)


def test_trace_accumulate_equals_trace_then_accumulate():
    """The fused kernel gives the same hits and the same table as the two calls."""
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=4)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    o, d, _ = rr.to_device_rays(rays)
    t1, t2 = rr.LengthTable(lo, hi), rr.LengthTable(lo, hi)
    h1 = torch.empty(len(rays), 4, device="cuda")
    h2 = torch.empty(len(rays), 4, device="cuda")
    rr.rr_trace(bvh, o, d, h1)
    rr.rr_length_table_accumulate(t1, o, d, h1)
    rr.rr_trace_accumulate(bvh, o, d, h2, t2)
    torch.cuda.synchronize()
    assert np.array_equal(h1.cpu().numpy().view(np.uint32), h2.cpu().numpy().view(np.uint32))
    s1, c1 = t1.read()
    s2, c2 = t2.read()
    assert np.array_equal(s1, s2) and np.array_equal(c1, c2)
    assert int(c2.sum()) > (1 << 20)


def test_capsule_coherence_matches_oracle_and_ranks_orders():
    """Per-run capsule areas match the oracle (fp32 vs binary64), and sorting by
    the Two Point key lowers the mean area (Section 4.3's measure)."""
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=5)
    lo, hi = W.scene_aabb(tris)
    E = float(oracle.largest_extent(lo, hi))
    hits, _ = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    o, d, _ = rr.to_device_rays(rays)
    h = torch.from_numpy(hits).cuda()
    g = rr.rr_coherence_capsule(o, d, h, E).cpu().numpy()
    ref = oracle.capsule_areas(rays.o_tmin, rays.d_tmax, hits, E)
    assert g.shape == ref.shape == (1024,)
    assert np.allclose(g, ref, rtol=2e-4, atol=1e-6)
    for subset, n in ((64, 100), (17, 1000), (64, 5)):
        gs = rr.rr_coherence_capsule(o[:n].contiguous(), d[:n].contiguous(), h[:n].contiguous(), E,
                                     subset=subset).cpu().numpy()
        rs = oracle.capsule_areas(rays.o_tmin[:n], rays.d_tmax[:n], hits[:n], E, subset=subset)
        assert np.allclose(gs, rs, rtol=2e-4, atol=1e-6)
    keys = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi)
    perm, _ = oracle.stable_sort(keys)
    sorted_area = oracle.capsule_areas(rays.o_tmin[perm], rays.d_tmax[perm], hits[perm], E).mean()
    assert sorted_area < 0.5 * ref.mean()
