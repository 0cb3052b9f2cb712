"""GPU parity: keys, stable radix sort, reorder and length table against the oracle.

Keys, permutations, reordered rays and table cells are integers or bit copies,
so every comparison is exact.  All inputs come from the seeded generators or
from the oracle; nothing the CUDA path produced is fed to the oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LAYOUTS = {"aila": (rr.RR_KEY_AILA, oracle.AILA), "compact": (rr.RR_KEY_AILA_COMPACT, oracle.AILA_COMPACT),
           "two_point": (rr.RR_KEY_TWO_POINT, oracle.TWO_POINT), "origin": (rr.RR_KEY_ORIGIN, oracle.ORIGIN),
           "reis": (rr.RR_KEY_REIS, oracle.REIS), "costa": (rr.RR_KEY_COSTA, oracle.COSTA),
           "octahedron": (rr.RR_KEY_OCTAHEDRON, oracle.OCTAHEDRON)}
ALL_LAYOUTS = list(LAYOUTS)
TSRC = {"fixed": (rr.RR_T_FIXED, oracle.T_FIXED), "adaptive": (rr.RR_T_ADAPTIVE, oracle.T_ADAPTIVE),
        "given": (rr.RR_T_GIVEN, oracle.T_GIVEN)}


@pytest.fixture(scope="module")
def soup():
    tris = W.scene_box_soup(seed=1)
    rays = W.rays_box_soup(tris, n=65536, seed=1)
    lo, hi = W.scene_aabb(tris)
    return tris, rays, lo, hi


@pytest.fixture(scope="module")
def soup_hits(soup):
    tris, rays, lo, hi = soup
    hits, _ = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    return hits


def gpu_keys(rays, layout, bits, lo, hi, tsrc=rr.RR_T_FIXED, ratio=0.25, t_given=None, table=None):
    o, d, _ = rr.to_device_rays(rays)
    tg = torch.from_numpy(np.ascontiguousarray(t_given, np.float32)).cuda() if t_given is not None else None
    p = rr.key_params(layout, bits, lo, hi, t_source=tsrc, ratio=ratio, t_given=tg, table=table)
    keys = torch.empty(len(rays), dtype=rr.key_dtype(bits), device="cuda")
    rr.rr_compute_keys(o, d, p, keys)
    torch.cuda.synchronize()
    return rr.keys_to_numpy(keys)


def assert_no_device_error():
    assert rr.rr_device_error() == 0


# ------------------------------------------------------------------ keys

@pytest.mark.parametrize("name", ALL_LAYOUTS)
@pytest.mark.parametrize("bits", [1, 3, 4, 16, 20, 31, 32, 33, 48, 63, 64])
def test_keys_match_oracle(soup, name, bits):
    tris, rays, lo, hi = soup
    g, o = LAYOUTS[name]
    k_gpu = gpu_keys(rays, g, bits, lo, hi)
    k_or = oracle.compute_keys(o, bits, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=oracle.T_FIXED, ratio=0.25)
    assert np.array_equal(k_gpu, k_or)
    assert_no_device_error()


def test_two_point_given_matches_oracle(soup, soup_hits):
    tris, rays, lo, hi = soup
    t = soup_hits[:, 0].copy()  # oracle hit distances; misses are +inf (-> 4E)
    k_gpu = gpu_keys(rays, rr.RR_KEY_TWO_POINT, 64, lo, hi, tsrc=rr.RR_T_GIVEN, t_given=t)
    k_or = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=oracle.T_GIVEN,
                               t_given=t)
    assert np.array_equal(k_gpu, k_or)


def test_length_table_and_adaptive_keys_match_oracle(soup, soup_hits):
    tris, rays, lo, hi = soup
    E = oracle.largest_extent(lo, hi)
    tab = rr.LengthTable(lo, hi)
    s0, c0 = tab.read()
    assert np.all(s0 == 4194304) and np.all(c0 == 1)
    o, d, _ = rr.to_device_rays(rays)
    h = torch.from_numpy(soup_hits).cuda()
    tab.accumulate(o, d, h)
    ot = oracle.LengthTable(E)
    ot.accumulate(lo, hi, rays.o_tmin, rays.d_tmax, soup_hits)
    s, c = tab.read()
    assert np.array_equal(s, ot.sum) and np.array_equal(c, ot.cnt)
    for bits in (32, 64):
        k_gpu = gpu_keys(rays, rr.RR_KEY_TWO_POINT, bits, lo, hi, tsrc=rr.RR_T_ADAPTIVE, table=tab)
        k_or = oracle.compute_keys(oracle.TWO_POINT, bits, rays.o_tmin, rays.d_tmax, lo, hi,
                                   tsrc=oracle.T_ADAPTIVE, table=ot)
        assert np.array_equal(k_gpu, k_or)
    # accumulation is order independent: a second pass over shuffled rays
    p = np.random.default_rng(0).permutation(len(rays))
    r2 = rays.subset(p)
    o2, d2, _ = rr.to_device_rays(r2)
    tab.accumulate(o2, d2, torch.from_numpy(np.ascontiguousarray(soup_hits[p])).cuda())
    ot.accumulate(lo, hi, r2.o_tmin, r2.d_tmax, soup_hits[p])
    s, c = tab.read()
    assert np.array_equal(s, ot.sum) and np.array_equal(c, ot.cnt)
    tab.reset()
    s, c = tab.read()
    assert np.all(s == 4194304) and np.all(c == 1)
    tab.close()


def _edge_rays(n, seed):
    rng = np.random.default_rng(seed)
    o = rng.uniform(-0.5, 1.5, size=(n, 4)).astype(np.float32)
    d = rng.normal(size=(n, 4)).astype(np.float32)
    special = [np.nan, np.inf, -np.inf, 0.0, -0.0, 1e-38, 1e30, -1e30]
    for c in range(3):
        idx = rng.choice(n, size=n // 8, replace=False)
        o[idx, c] = rng.choice(special, size=idx.size)
        idx = rng.choice(n, size=n // 8, replace=False)
        d[idx, c] = rng.choice(special, size=idx.size)
    d[: n // 16, :3] = 0.0  # zero directions
    o[:, 3] = 0.0
    d[:, 3] = np.inf
    return W.Rays(o, d, np.arange(n, dtype=np.uint32))


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 257, 4097])
def test_keys_edge_values_and_sizes(n):
    rays = _edge_rays(n, n)
    boxes = [(np.zeros(3, np.float32), np.ones(3, np.float32)),
             (np.array([0, 0.5, 0], np.float32), np.array([1, 0.5, 2], np.float32))]  # flat axis
    for lo, hi in boxes:
        for name in ALL_LAYOUTS:
            g, o = LAYOUTS[name]
            for bits in (32, 64):
                k_gpu = gpu_keys(rays, g, bits, lo, hi)
                k_or = oracle.compute_keys(o, bits, rays.o_tmin, rays.d_tmax, lo, hi)
                assert np.array_equal(k_gpu, k_or), (name, bits)
        t = np.random.default_rng(n).choice([np.inf, np.nan, -1.0, 0.0, 0.3, 1e20], size=n).astype(np.float32)
        k_gpu = gpu_keys(rays, rr.RR_KEY_TWO_POINT, 64, lo, hi, tsrc=rr.RR_T_GIVEN, t_given=t)
        k_or = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi,
                                   tsrc=oracle.T_GIVEN, t_given=t)
        assert np.array_equal(k_gpu, k_or)
    assert_no_device_error()


def test_keys_reject_bad_arguments(soup):
    tris, rays, lo, hi = soup
    o, d, _ = rr.to_device_rays(rays.subset(slice(0, 16)))
    keys = torch.empty(16, dtype=torch.int64, device="cuda")
    for bad in (dict(bits=0), dict(bits=65), dict(layout=7)):
        kw = dict(layout=rr.RR_KEY_AILA, bits=32)
        kw.update(bad)
        p = rr.key_params(kw["layout"], kw["bits"], lo, hi)
        with pytest.raises(rr.RRError) as e:
            rr.rr_compute_keys(o, d, p, keys)
        assert e.value.status == 1
    p = rr.key_params(rr.RR_KEY_AILA, 32, hi, lo)  # inverted box
    with pytest.raises(rr.RRError):
        rr.rr_compute_keys(o, d, p, keys)
    p = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE)  # no table
    with pytest.raises(rr.RRError):
        rr.rr_compute_keys(o, d, p, keys)
    other = rr.LengthTable(lo, hi + 1)
    p = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=other)
    with pytest.raises(rr.RRError):
        rr.rr_compute_keys(o, d, p, keys)
    # n == 0 is a no-op
    rr.rr_compute_keys(o, d, rr.key_params(rr.RR_KEY_AILA, 32, lo, hi), keys, n=0)


# ------------------------------------------------------------------ sort

def gpu_sort(keys_np, bits, radix_bits, want_keys=True):
    n = keys_np.shape[0]
    wide = bits > 32
    kt = torch.from_numpy(keys_np.astype(np.uint64).view(np.int64) if wide
                          else keys_np.astype(np.uint32).view(np.int32)).cuda()
    ko = torch.empty_like(kt) if want_keys else None
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = rr.sort_workspace(n, bits, radix_bits)
    rr.rr_sort(kt, ko, perm, n, bits, radix_bits, ws)
    torch.cuda.synchronize()
    before = rr.keys_to_numpy(kt)
    assert np.array_equal(before, keys_np.astype(np.uint64)), "keys_in was modified"
    return rr.u32_to_numpy(perm), (rr.keys_to_numpy(ko) if want_keys else None)


def _random_keys(n, bits, rng, dup=False):
    hi = np.uint64(2 ** bits - 1) if bits < 64 else np.uint64(2 ** 64 - 1)
    k = rng.integers(0, 2 ** 63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    if bits < 64:
        k &= hi
    if dup:
        k = (k % np.uint64(7)) << np.uint64(max(0, bits - 3)) if bits >= 3 else k % np.uint64(2)
        k &= hi
    return k


@pytest.mark.parametrize("radix_bits", [8, 4])
@pytest.mark.parametrize("bits", [1, 7, 8, 13, 16, 31, 32, 33, 48, 64])
@pytest.mark.parametrize("n", [1, 2, 33, 3071, 3072, 3073, 4096, 4097, 70001])
def test_sort_matches_oracle(radix_bits, bits, n):
    rng = np.random.default_rng(bits * 1000 + n)
    for dup in (False, True):
        keys = _random_keys(n, bits, rng, dup)
        perm_or, sk_or = oracle.stable_sort(keys)
        perm, sk = gpu_sort(keys, bits, radix_bits)
        assert np.array_equal(perm, perm_or)
        assert np.array_equal(sk, sk_or)
    assert_no_device_error()


@pytest.mark.parametrize("radix_bits", [8, 4])
@pytest.mark.parametrize("bits", [32, 64])
def test_sort_long_passes_match_oracle(radix_bits, bits):
    """Passes of at least eight tiles per SM take the four-blocks-per-SM form
    (values loaded after the ranking); just below that they take the
    three-block form.  Both sides of the switch, with a one-key ragged tail
    and repeated keys, against the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tile = 256 * (12 if bits > 32 else 16)
    rng = np.random.default_rng(77 + bits + radix_bits)
    for tiles in (8 * sms - 1, 8 * sms + 1):
        n = (tiles - 1) * tile + 1
        keys = _random_keys(n, bits, rng, dup=tiles > 8 * sms)
        perm_or, _ = oracle.stable_sort(keys)
        perm, _ = gpu_sort(keys, bits, radix_bits, want_keys=False)
        assert np.array_equal(perm, perm_or), (tiles, n)
    assert_no_device_error()


@pytest.mark.parametrize("radix_bits", [8, 4])
@pytest.mark.parametrize("bits", [32, 64])
def test_sort_one_and_two_wave_passes_match_oracle(radix_bits, bits):
    """Digit passes of just under and just over one and two full waves of
    three blocks per SM (a tile's look-back then waits on tiles that start
    later), with a ragged last tile and repeated keys, against the oracle."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tile = 256 * (12 if bits > 32 else 16)
    rng = np.random.default_rng(99 + bits + radix_bits)
    for tiles in (3 * sms - 1, 3 * sms + 1, 6 * sms - 1, 6 * sms + 1):
        n = (tiles - 1) * tile + 7
        keys = _random_keys(n, bits, rng, dup=tiles % 2 == 1)
        perm_or, sk_or = oracle.stable_sort(keys)
        perm, sk = gpu_sort(keys, bits, radix_bits)
        assert np.array_equal(perm, perm_or), (tiles, n)
        assert np.array_equal(sk, sk_or), (tiles, n)
    assert_no_device_error()


@pytest.mark.parametrize("bits", [32, 64])
def test_sort_without_key_output_and_determinism(bits):
    rng = np.random.default_rng(5)
    keys = _random_keys(300001, bits, rng, dup=True)
    perm_or, _ = oracle.stable_sort(keys)
    p1, _ = gpu_sort(keys, bits, 8, want_keys=False)
    p2, _ = gpu_sort(keys, bits, 8, want_keys=False)
    assert np.array_equal(p1, perm_or) and np.array_equal(p2, p1)


def test_sort_all_equal_and_presorted_and_reversed():
    n = 100000
    for keys in (np.full(n, 5, np.uint64), np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64)[::-1].copy()):
        perm_or, _ = oracle.stable_sort(keys)
        for bits in (17, 40):
            perm, _ = gpu_sort(keys, bits, 8)
            assert np.array_equal(perm, perm_or)


def test_sort_rejects_bad_arguments():
    n = 100
    k = torch.zeros(n, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = rr.sort_workspace(n, 32, 8)
    with pytest.raises(rr.RRError):
        rr.rr_sort(k, None, perm, n, 32, 5, ws)  # radix width
    with pytest.raises(rr.RRError):
        rr.rr_sort(k, None, perm, n, 0, 8, ws)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(rr.RRError):
        rr.rr_sort(k, None, perm, n, 32, 8, small)  # workspace too small
    with pytest.raises(rr.RRError):
        rr.rr_sort(k, k, perm, n, 32, 8, ws)  # keys_out aliases keys_in
    rr.rr_sort(k, None, perm, 0, 32, 8, ws)  # n == 0 is a no-op


def test_sort_real_keys_config1(soup):
    tris, rays, lo, hi = soup
    for name, bits in (("aila", 32), ("two_point", 64)):
        g, o = LAYOUTS[name]
        keys = oracle.compute_keys(o, bits, rays.o_tmin, rays.d_tmax, lo, hi)
        perm_or, _ = oracle.stable_sort(keys)
        perm, _ = gpu_sort(keys, bits, 8)
        assert np.array_equal(perm, perm_or)


# ------------------------------------------------------------------ reorder

@pytest.mark.parametrize("n", [1, 511, 512, 513, 65536, 100003])
def test_permute_bitwise(n):
    rng = np.random.default_rng(n)
    o = rng.normal(size=(n, 4)).astype(np.float32)
    d = rng.normal(size=(n, 4)).astype(np.float32)
    o[: n // 10, 0] = np.nan
    pay = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    perm = rng.permutation(n).astype(np.uint32)
    oo, dd, pp = oracle.permute(o, d, pay, perm)
    go, gd = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gp = torch.from_numpy(pay.view(np.int32)).cuda()
    gperm = torch.from_numpy(perm.view(np.int32)).cuda()
    oo_g, dd_g, pp_g = torch.empty_like(go), torch.empty_like(gd), torch.empty_like(gp)
    rr.rr_permute(go, gd, gp, gperm, oo_g, dd_g, pp_g)
    assert np.array_equal(oo_g.cpu().numpy().view(np.uint32), oo.view(np.uint32))
    assert np.array_equal(dd_g.cpu().numpy().view(np.uint32), dd.view(np.uint32))
    assert np.array_equal(rr.u32_to_numpy(pp_g), pp)
    # without payload
    oo_g.zero_()
    rr.rr_permute(go, gd, None, gperm, oo_g, dd_g, None)
    assert np.array_equal(oo_g.cpu().numpy().view(np.uint32), oo.view(np.uint32))


def test_permute_rejects_overlap():
    n = 64
    a = torch.zeros(n, 4, device="cuda")
    perm = torch.arange(n, dtype=torch.int32, device="cuda")
    with pytest.raises(rr.RRError):
        rr.rr_permute(a, a, None, perm, a, torch.zeros_like(a), None)


# ------------------------------------------------------------------ full-size wavefront

def test_full_size_keys_and_sort_config2():
    """2,073,600 camera rays and 2,073,600 stand-in secondary rays of the
    1.17M-triangle terrain: every key and the whole permutation match."""
    tris = W.scene_terrain()
    lo, hi = W.scene_aabb(tris)
    cam = W.camera_rays(W.Camera())
    sec = W.surface_rays(tris, 2073600, seed=9)
    for rays in (cam, sec):
        for name, bits in (("aila", 64), ("two_point", 64)):
            g, o = LAYOUTS[name]
            k_gpu = gpu_keys(rays, g, bits, lo, hi)
            k_or = oracle.compute_keys(o, bits, rays.o_tmin, rays.d_tmax, lo, hi)
            assert np.array_equal(k_gpu, k_or)
            perm_or, _ = oracle.stable_sort(k_or)
            perm, _ = gpu_sort(k_or, bits, 8, want_keys=False)
            assert np.array_equal(perm, perm_or)
    assert_no_device_error()


def test_adaptive_keys_with_extreme_table_contents(soup):
    """Cells with large sums and counts (the estimate divides a 64-bit sum by
    a count): keys still match the oracle reading the same table."""
    tris, rays, lo, hi = soup
    E = oracle.largest_extent(lo, hi)
    rng = np.random.default_rng(17)
    cnt = rng.integers(1, 2 ** 32 - 1, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    cnt[::3] = rng.integers(1, 50, size=cnt[::3].size).astype(np.uint32)
    mean = rng.integers(0, 2 ** 30, size=1 << 20, dtype=np.uint64)
    extra = (rng.random(1 << 20) * cnt).astype(np.uint64)
    s = mean * cnt.astype(np.uint64) + extra
    tab = rr.LengthTable(lo, hi)
    tab.write(s, cnt)
    ot = oracle.LengthTable(E)
    ot.sum[:] = s
    ot.cnt[:] = cnt
    k_gpu = gpu_keys(rays, rr.RR_KEY_TWO_POINT, 64, lo, hi, tsrc=rr.RR_T_ADAPTIVE, table=tab)
    k_or = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=oracle.T_ADAPTIVE,
                               table=ot)
    assert np.array_equal(k_gpu, k_or)


@pytest.mark.parametrize("n", [1, 3, 255, 256, 257, 1000, 4097, 65535])
@pytest.mark.parametrize("name,bits,tsrc", [("two_point", 64, "adaptive"), ("aila", 32, "fixed"),
                                            ("octahedron", 40, "fixed"), ("two_point", 20, "given")])
def test_keys_ragged_sizes(soup, soup_hits, n, name, bits, tsrc):
    """Ray counts that end inside a 256-ray tile: the staged copies of the last
    tile are shorter, and every key still matches the oracle."""
    tris, rays, lo, hi = soup
    sub = rays.subset(np.arange(n))
    layout, olayout = LAYOUTS[name]
    ts, ots = TSRC[tsrc]
    E = oracle.largest_extent(lo, hi)
    tab, ot, tg = None, None, None
    if tsrc == "adaptive":
        ot = oracle.LengthTable(E)
        ot.accumulate(lo, hi, rays.o_tmin, rays.d_tmax, soup_hits)
        tab = rr.LengthTable(lo, hi)
        tab.write(ot.sum, ot.cnt)
    if tsrc == "given":
        tg = np.random.default_rng(n).random(n).astype(np.float32)
    k_gpu = gpu_keys(sub, layout, bits, lo, hi, tsrc=ts, t_given=tg, table=tab)
    k_or = oracle.compute_keys(olayout, bits, sub.o_tmin, sub.d_tmax, lo, hi, tsrc=ots, t_given=tg, table=ot)
    assert np.array_equal(k_gpu, k_or)
    assert_no_device_error()
