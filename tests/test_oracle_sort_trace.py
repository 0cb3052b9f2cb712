"""Pins of the oracle's sort, reorder, trace and length table (CPU only).

Sort: invariants, brute force over all orders of tiny inputs, and Python's
stable ``sorted`` (a library routine).  Trace: closed-form distances inside an
axis-aligned box, rays aimed at known barycentric points, interval ends, and
the oracle BVH against the brute-force definition.  Length table: the
hand-computed cells of Section 3.1.6's dummy-ray initialisation.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2506_11273_gb300 import workloads as W

# ------------------------------------------------------------------ sort


def _check_stable_sorted(keys, perm):
    n = keys.shape[0]
    assert np.array_equal(np.sort(perm), np.arange(n, dtype=np.uint32))
    sk = keys[perm]
    assert np.all(sk[1:] >= sk[:-1])
    same = sk[1:] == sk[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, 1000, 4097])
def test_sort_invariants_and_python_sorted(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 17, size=n).astype(np.uint64) << np.uint64(40)
    keys |= rng.integers(0, 3, size=n).astype(np.uint64)
    perm, sk = oracle.stable_sort(keys)
    _check_stable_sorted(keys, perm)
    assert np.array_equal(sk, keys[perm])
    ref = sorted(range(n), key=lambda i: int(keys[i]))  # Python's sort is stable
    assert perm.tolist() == ref


def test_sort_brute_force_all_orders():
    """For n <= 6, exactly one permutation is sorted and stable; it is the oracle's."""
    rng = np.random.default_rng(1)
    for n in range(0, 7):
        for _ in range(5):
            keys = rng.integers(0, 3, size=n).astype(np.uint64)
            good = []
            for p in itertools.permutations(range(n)):
                sk = [int(keys[i]) for i in p]
                ok = all(sk[i] < sk[i + 1] or (sk[i] == sk[i + 1] and p[i] < p[i + 1])
                         for i in range(n - 1))
                if ok:
                    good.append(list(p))
            assert len(good) == 1
            perm, _ = oracle.stable_sort(keys)
            assert perm.tolist() == good[0]


def test_sort_full_64bit_range():
    keys = np.array([2**64 - 1, 0, 2**63, 2**63 - 1, 2**64 - 1, 1], np.uint64)
    perm, sk = oracle.stable_sort(keys)
    assert perm.tolist() == [1, 5, 3, 2, 0, 4]


@pytest.mark.parametrize("n,segment", [(0, 4), (1, 1), (10, 1), (10, 3), (1000, 64), (1000, 1000),
                                       (1000, 4096), (4097, 1024)])
def test_segment_sort_invariants(n, segment):
    """Each segment holds a stable sort of its own keys; segment >= n is the
    global sort and segment 1 the identity."""
    rng = np.random.default_rng(n + segment)
    keys = rng.integers(0, 9, size=n).astype(np.uint64) << np.uint64(30)
    perm = oracle.segment_sort(keys, segment)
    for s in range(0, n, segment):
        seg = perm[s:s + segment]
        assert np.array_equal(np.sort(seg), np.arange(s, min(n, s + segment), dtype=np.uint32))
        ref = sorted(range(s, min(n, s + segment)), key=lambda i: int(keys[i]))
        assert seg.tolist() == ref
    if segment >= n:
        assert np.array_equal(perm, oracle.stable_sort(keys)[0])
    if segment == 1:
        assert np.array_equal(perm, np.arange(n, dtype=np.uint32))


def test_permute_is_bitwise_gather():
    rng = np.random.default_rng(2)
    n = 777
    o = rng.normal(size=(n, 4)).astype(np.float32)
    o[5, 0] = np.nan
    d = rng.normal(size=(n, 4)).astype(np.float32)
    p = rng.integers(0, 2**32, size=n, dtype=np.uint64).astype(np.uint32)
    perm = rng.permutation(n).astype(np.uint32)
    oo, dd, pp = oracle.permute(o, d, p, perm)
    assert np.array_equal(oo.view(np.uint32), o[perm].view(np.uint32))
    assert np.array_equal(dd.view(np.uint32), d[perm].view(np.uint32))
    assert np.array_equal(pp, p[perm])


# ------------------------------------------------------------------ trace

BOX = W._box_tris(np.zeros(3), np.ones(3), inward=True).astype(np.float32)


def test_trace_closed_form_inside_unit_box():
    """From inside [0,1]^3 the hit is the nearest wall: t = min_c (wall_c - o_c)/d_c."""
    r = W.random_rays_in_box(2000, [0.05] * 3, [0.95] * 3, seed=4)
    hits, info = oracle.trace_brute(BOX, r.o_tmin, r.d_tmax)
    o = r.o_tmin[:, :3].astype(np.float64)
    d = r.d_tmax[:, :3].astype(np.float64)
    wall = np.where(d > 0, 1.0, 0.0)
    with np.errstate(divide="ignore"):
        tc = np.where(d != 0, (wall - o) / d, np.inf)
    t_exp = tc.min(axis=1)
    axis = tc.argmin(axis=1)
    tri = oracle.hit_tri(hits)
    assert np.all(tri != oracle.MISS)
    assert np.allclose(info[:, 0], t_exp, rtol=1e-12, atol=0)
    # the triangle lies on the wall of that axis and side
    v = BOX[tri].reshape(-1, 3, 3).astype(np.float64)
    side = wall[np.arange(len(axis)), axis]
    assert np.all(v[np.arange(len(axis)), :, axis] == side[:, None])


def test_trace_known_barycentric_points_and_two_sided():
    rng = np.random.default_rng(6)
    tris = (rng.random((50, 9)) * 4 - 2).astype(np.float32)
    for k in range(50):
        tri = tris[k]
        v0, v1, v2 = tri[0:3].astype(np.float64), tri[3:6].astype(np.float64), tri[6:9].astype(np.float64)
        u, v = rng.random() * 0.6 + 0.05, rng.random() * 0.3 + 0.02
        P = v0 + u * (v1 - v0) + v * (v2 - v0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        s = 0.5 + rng.random()
        for sign in (1.0, -1.0):  # either side of the plane
            dd = sign * d
            o = P - s * dd
            ok, t, uu, vv = oracle.ray_triangle(o, dd, tri)
            assert ok
            assert abs(t - s) < 1e-9 and abs(uu - u) < 1e-9 and abs(vv - v) < 1e-9


@pytest.mark.parametrize("edge", ["u", "v", "w"])
def test_ray_triangle_uv_signed_margin_at_each_edge(edge):
    """or_ray_triangle_uv, the helper that decides which hit disagreements are
    edge cases: rays aimed at points just inside and just outside each edge
    of a triangle (tiny steps across the edge) return the barycentrics of the
    target point and its distance, in closed form, from both sides, and the
    signed margin min(u, v, 1-u-v) changes sign exactly across the edge."""
    tri = np.array([0.25, 0.5, 0.125, 1.25, 0.75, 0.375, 0.5, 1.5, -0.25], np.float32)
    v0, v1, v2 = (tri[0:3].astype(np.float64), tri[3:6].astype(np.float64), tri[6:9].astype(np.float64))
    e1, e2 = v1 - v0, v2 - v0
    rng = np.random.default_rng({"u": 1, "v": 2, "w": 3}[edge])
    for step in (1e-3, 1e-6, -1e-6, -1e-3):  # > 0: inside by `step`, < 0: outside
        s = rng.uniform(0.2, 0.8)
        if edge == "u":      # edge v0-v2: u = step
            u, v = step, s * (1 - step)
        elif edge == "v":    # edge v0-v1: v = step
            u, v = s * (1 - step), step
        else:                # edge v1-v2: 1 - u - v = step
            u = s * (1 - step)
            v = 1 - step - u
        p = v0 + u * e1 + v * e2
        for sign in (1.0, -1.0):
            d = sign * np.array([0.3, -0.2, 1.0]) + 0.1 * rng.standard_normal(3)
            t_true = rng.uniform(0.5, 3.0)
            o = p - t_true * d
            ok, t, uu, vv = oracle.ray_plane_barycentrics(o, d, tri)
            assert ok
            assert abs(t - t_true) <= 1e-12 * t_true
            assert abs(uu - u) <= 1e-12 and abs(vv - v) <= 1e-12
            margin = min(uu, vv, 1.0 - uu - vv)
            assert abs(margin - step) <= 1e-12
            assert (margin > 0) == (step > 0)
    # a ray in the triangle's plane has no solution
    n = np.cross(e1, e2)
    d_par = np.cross(n, e1)
    ok, _, _, _ = oracle.ray_plane_barycentrics(v0 - d_par, d_par, tri)
    assert not ok


def test_trace_open_interval_and_parallel_miss():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)  # z = 0 plane
    o_tmin = np.array([[0.25, 0.25, 1.0, 0.0]], np.float32)
    d = np.array([[0, 0, -1, np.inf]], np.float32)
    h, _ = oracle.trace_brute(tri, o_tmin, d)
    assert oracle.hit_tri(h)[0] == 0 and h[0, 0] == 1.0
    # tmax equal to the hit distance: open interval, no hit
    d2 = d.copy()
    d2[0, 3] = 1.0
    h, _ = oracle.trace_brute(tri, o_tmin, d2)
    assert oracle.hit_tri(h)[0] == oracle.MISS and np.isinf(h[0, 0])
    # tmin equal to the hit distance: no hit
    o2 = o_tmin.copy()
    o2[0, 3] = 1.0
    h, _ = oracle.trace_brute(tri, o2, d)
    assert oracle.hit_tri(h)[0] == oracle.MISS
    # ray parallel to the plane
    h, _ = oracle.trace_brute(tri, np.array([[0.25, 0.25, 0.0, 0.0]], np.float32),
                              np.array([[1, 0, 0, np.inf]], np.float32))
    assert oracle.hit_tri(h)[0] == oracle.MISS
    # zero-area triangle never hits
    deg = np.array([0, 0, 0, 1, 1, 0, 2, 2, 0], np.float32)
    h, _ = oracle.trace_brute(deg, np.array([[0.5, 0.5, 1, 0]], np.float32), d)
    assert oracle.hit_tri(h)[0] == oracle.MISS


def test_trace_equal_t_takes_lowest_id():
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0], np.float32)
    tris = np.stack([tri, tri, tri])
    h, _ = oracle.trace_brute(tris, np.array([[0.25, 0.25, 1.0, 0.0]], np.float32),
                              np.array([[0, 0, -1, np.inf]], np.float32))
    assert oracle.hit_tri(h)[0] == 0
    bvh = oracle.BVH(tris)
    h2, _ = bvh.trace(np.array([[0.25, 0.25, 1.0, 0.0]], np.float32),
                      np.array([[0, 0, -1, np.inf]], np.float32))
    assert oracle.hit_tri(h2)[0] == 0


def test_trace_empty_scene():
    r = W.random_rays_in_box(10, [0] * 3, [1] * 3, seed=1)
    h, _ = oracle.trace_brute(np.zeros((0, 9), np.float32), r.o_tmin, r.d_tmax)
    assert np.all(oracle.hit_tri(h) == oracle.MISS) and np.all(np.isinf(h[:, 0]))
    b = oracle.BVH(np.zeros((0, 9), np.float32))
    h, _ = b.trace(r.o_tmin, r.d_tmax)
    assert np.all(oracle.hit_tri(h) == oracle.MISS)


def test_bvh_equals_brute_force_on_box_soup():
    tris = W.scene_box_soup(seed=1, n_random=1024)
    rays = W.rays_box_soup(tris, n=3000, seed=1)
    extra = W.random_rays_in_box(1000, [-0.5] * 3, [1.5] * 3, seed=8, tmin=0.0)
    bvh = oracle.BVH(tris)
    for r, min_hit in ((rays, 0.99), (extra, 0.2)):
        hb, ib = oracle.trace_brute(tris, r.o_tmin, r.d_tmax)
        hv, iv = bvh.trace(r.o_tmin, r.d_tmax)
        assert np.array_equal(hb.view(np.uint32), hv.view(np.uint32))
        assert np.array_equal(ib, iv)
        assert (oracle.hit_tri(hb) != oracle.MISS).mean() > min_hit


def test_bvh_equals_brute_force_on_terrain_patch():
    tris = W.scene_terrain(seed=3, cells_x=32, cells_z=64, n_boxes=200)
    rays = W.surface_rays(tris, 2000, seed=3)
    hb, ib = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    hv, iv = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    assert np.array_equal(hb.view(np.uint32), hv.view(np.uint32))


# ------------------------------------------------------------------ length table

def test_table_initial_estimate_is_quarter_extent():
    for E in (1.0, 2.0, 3.0, 0.7):
        tab = oracle.LengthTable(E)
        assert tab.cnt.min() == 1 and tab.cnt.max() == 1
        assert int(tab.sum[0]) == 4194304  # 0.25 * 2^24
        assert tab.estimate(12345) == np.float32(0.25) * np.float32(E)


def test_table_hand_computed_cell():
    """Three hits of lengths 0.5E, E, 0.125E join the dummy 0.25E ray:
    mean = (0.25 + 0.5 + 1 + 0.125)/4 E = 0.46875 E."""
    E = np.float32(2.0)
    lo = np.zeros(3, np.float32)
    hi = np.array([2, 1, 1], np.float32)
    tab = oracle.LengthTable(E)
    o = np.array([[0.3, 0.4, 0.5, 0.0]] * 4, np.float32)
    d = np.array([[0, 1, 0, np.inf]] * 4, np.float32)
    hits = np.zeros((4, 4), np.float32)
    hits[:, 0] = [1.0, 2.0, 0.25, 5.0]
    tri = np.array([7, 8, 9, oracle.MISS], np.uint32)
    hits[:, 3] = tri.view(np.float32)
    tab.accumulate(lo, hi, o, d, hits)
    cell = oracle.table_cell(o[0, :3], d[0, :3], lo, hi)
    assert int(tab.cnt[cell]) == 4
    assert int(tab.sum[cell]) == 4194304 + 8388608 + 16777216 + 2097152
    assert tab.estimate(cell) == np.float32(0.46875 * 2.0)
    assert int(tab.cnt.sum()) == (1 << 20) + 3


def test_table_fixed_length_clamps():
    d = np.array([0, 0, 1], np.float32)
    assert oracle.fixed_length(1e9, d, 1.0) == 64 * 2**24
    assert oracle.fixed_length(-1.0, d, 1.0) == 0
    assert oracle.fixed_length(0.5, d, 1.0) == 2**23
    # world-space length: a direction of length 2 doubles it
    assert oracle.fixed_length(0.25, np.array([0, 2, 0], np.float32), 1.0) == 2**23


def test_table_order_independent():
    tris = W.scene_box_soup(seed=1, n_random=256)
    rays = W.rays_box_soup(tris, n=4000, seed=2)
    hits, _ = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    lo, hi = W.scene_aabb(tris)
    E = oracle.largest_extent(lo, hi)
    a = oracle.LengthTable(E)
    a.accumulate(lo, hi, rays.o_tmin, rays.d_tmax, hits)
    p = np.random.default_rng(0).permutation(len(rays))
    b = oracle.LengthTable(E)
    b.accumulate(lo, hi, rays.o_tmin[p], rays.d_tmax[p], hits[p])
    assert np.array_equal(a.sum, b.sum) and np.array_equal(a.cnt, b.cnt)
    nhit = int((oracle.hit_tri(hits) != oracle.MISS).sum())
    assert int(a.cnt.sum()) == (1 << 20) + nhit


def test_adaptive_key_uses_table_estimate():
    """An ADAPTIVE Two Point key equals the GIVEN key with the cell's estimate."""
    tris = W.scene_box_soup(seed=1, n_random=256)
    rays = W.rays_box_soup(tris, n=2000, seed=3)
    hits, _ = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    lo, hi = W.scene_aabb(tris)
    E = oracle.largest_extent(lo, hi)
    tab = oracle.LengthTable(E)
    tab.accumulate(lo, hi, rays.o_tmin, rays.d_tmax, hits)
    ka = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi,
                             tsrc=oracle.T_ADAPTIVE, table=tab)
    t_est = np.array([tab.estimate(oracle.table_cell(rays.o_tmin[i, :3], rays.d_tmax[i, :3], lo, hi))
                      for i in range(len(rays))], np.float32)
    kg = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi,
                             tsrc=oracle.T_GIVEN, t_given=t_est)
    assert np.array_equal(ka, kg)
    # and the estimates moved away from the dummy value where rays hit
    assert np.mean(t_est != np.float32(0.25) * E) > 0.5


# ------------------------------------------------------------------ capsule coherence measure

def _rays_from(o, d, t):
    n = len(o)
    o_tmin = np.zeros((n, 4), np.float32)
    d_tmax = np.zeros((n, 4), np.float32)
    hits = np.zeros((n, 4), np.float32)
    o_tmin[:, :3] = o
    d_tmax[:, :3] = d
    d_tmax[:, 3] = np.inf
    hits[:, 0] = t
    hits[:, 3] = np.zeros(n, np.uint32).view(np.float32)
    return o_tmin, d_tmax, hits


def test_capsule_of_parallel_rays_is_a_cylinder():
    """64 rays on a circle of radius r, all along +z with length h: hemispheres
    of radius r at both ends and a cylinder between, area 4*pi*r^2 + 2*pi*r*h."""
    r, h = 0.5, 3.0
    ang = np.arange(64) * 2 * np.pi / 64
    o = np.stack([r * np.cos(ang), r * np.sin(ang), np.zeros(64)], 1)
    d = np.tile([0, 0, 1.0], (64, 1))
    ot, dt, hits = _rays_from(o, d, np.full(64, h))
    a = oracle.capsule_areas(ot, dt, hits, E=10.0)
    assert a.shape == (1,)
    r_meas = np.mean(np.hypot(o[:, 0].astype(np.float32), o[:, 1].astype(np.float32)))
    assert abs(a[0] - (4 * np.pi * r_meas ** 2 + 2 * np.pi * r_meas * h)) < 1e-6 * a[0]


def test_capsule_of_a_cone_and_a_point():
    """Rays from one point fanning out to a circle: r_o = 0, r_t = R: the area is
    a hemisphere of radius R plus the cone's lateral area pi*R*sqrt(h^2 + R^2)."""
    R, h = 2.0, 5.0
    ang = np.arange(64) * 2 * np.pi / 64
    tgt = np.stack([R * np.cos(ang), R * np.sin(ang), np.full(64, h)], 1)
    o = np.zeros((64, 3))
    d = tgt / np.linalg.norm(tgt, axis=1, keepdims=True)
    ot, dt, hits = _rays_from(o, d, np.linalg.norm(tgt, axis=1))
    a = oracle.capsule_areas(ot, dt, hits, E=10.0)[0]
    assert abs(a - (2 * np.pi * R * R + np.pi * R * np.sqrt(h * h + R * R))) < 1e-4 * a


def test_capsule_subsets_and_misses():
    rng = np.random.default_rng(4)
    o = rng.random((200, 3))
    d = rng.normal(size=(200, 3))
    ot, dt, hits = _rays_from(o, d, rng.random(200))
    a = oracle.capsule_areas(ot, dt, hits, E=1.0)
    assert a.shape == (3,)  # 200 // 64; the tail of 8 is ignored
    for g in range(3):
        sl = slice(64 * g, 64 * g + 64)
        assert a[g] == oracle.capsule_areas(ot[sl], dt[sl], hits[sl], E=1.0)[0]
    # a miss terminates at 4*E
    h2 = hits.copy()
    h2[:64, 3] = np.full(64, oracle.MISS, np.uint32).view(np.float32)
    h3 = hits.copy()
    h3[:64, 0] = 4.0
    assert oracle.capsule_areas(ot, dt, h2, E=1.0)[0] == oracle.capsule_areas(ot, dt, h3, E=1.0)[0]
    # coherent rays give a smaller capsule than the same rays shuffled
    o_c = np.repeat(rng.random((4, 3)), 64, axis=0) + rng.random((256, 3)) * 0.01
    d_c = np.repeat(rng.normal(size=(4, 3)), 64, axis=0) + rng.normal(size=(256, 3)) * 0.01
    ot, dt, hits = _rays_from(o_c, d_c, np.full(256, 0.5))
    p = rng.permutation(256)
    assert oracle.capsule_areas(ot, dt, hits, 1.0).mean() < oracle.capsule_areas(ot[p], dt[p], hits[p], 1.0).mean()
