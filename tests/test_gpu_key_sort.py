"""GPU parity of rr_key_sort: the keys of Section 3.1 and their stable radix
sort of Section 3.2 in one call, the sort's digit counting done by the key
kernel.  Keys and permutations are integers: every comparison is exact, against
the oracle's keys and the oracle's stable sort of them."""
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


@pytest.fixture(scope="module")
def soup():
    tris = W.scene_box_soup(seed=3)
    rays = W.rays_box_soup(tris, n=65536, seed=3)
    lo, hi = W.scene_aabb(tris)
    return tris, rays, lo, hi


def key_sort(rays, params, radix_bits, ws=None):
    n = len(rays)
    o, d, _ = rr.to_device_rays(rays)
    keys = torch.empty(n, dtype=rr.key_dtype(params.bits), device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    if ws is None:
        ws = rr.sort_workspace(n, params.bits, radix_bits)
    rr.rr_key_sort(o, d, params, keys, perm, radix_bits, ws)
    torch.cuda.synchronize()
    return rr.keys_to_numpy(keys), perm.cpu().numpy().view(np.uint32)


def oracle_key_sort(rays, layout, bits, lo, hi, **kw):
    keys = oracle.compute_keys(layout, bits, rays.o_tmin, rays.d_tmax, lo, hi, **kw)
    perm, _ = oracle.stable_sort(keys)
    return keys, perm


@pytest.mark.parametrize("name", list(LAYOUTS))
@pytest.mark.parametrize("bits", [1, 8, 20, 32, 33, 64])
@pytest.mark.parametrize("radix_bits", [8, 4])
def test_key_sort_matches_oracle(soup, name, bits, radix_bits):
    tris, rays, lo, hi = soup
    g, o = LAYOUTS[name]
    p = rr.key_params(g, bits, lo, hi)
    k_gpu, perm_gpu = key_sort(rays, p, radix_bits)
    k_or, perm_or = oracle_key_sort(rays, o, bits, lo, hi, tsrc=oracle.T_FIXED, ratio=0.25)
    assert np.array_equal(k_gpu, k_or)
    assert np.array_equal(perm_gpu, perm_or)
    assert rr.rr_device_error() == 0


@pytest.mark.parametrize("n", [1, 2, 255, 257, 3071, 3073, 12289])
def test_key_sort_ragged_sizes(soup, n):
    tris, rays, lo, hi = soup
    sub = rays.subset(np.arange(n))
    for bits, radix_bits in ((64, 8), (32, 4), (13, 8)):
        p = rr.key_params(rr.RR_KEY_TWO_POINT, bits, lo, hi)
        k_gpu, perm_gpu = key_sort(sub, p, radix_bits)
        k_or, perm_or = oracle_key_sort(sub, oracle.TWO_POINT, bits, lo, hi, tsrc=oracle.T_FIXED, ratio=0.25)
        assert np.array_equal(k_gpu, k_or) and np.array_equal(perm_gpu, perm_or), (n, bits, radix_bits)


def test_key_sort_adaptive_table(soup):
    """ADAPTIVE keys: the table is built by the oracle from oracle hits and
    written to the device, then keys and sort come from one call."""
    tris, rays, lo, hi = soup
    hits, _ = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    E = oracle.largest_extent(lo, hi)
    ot = oracle.LengthTable(E)
    ot.accumulate(lo, hi, rays.o_tmin, rays.d_tmax, hits)
    tab = rr.LengthTable(lo, hi)
    tab.write(ot.sum, ot.cnt)
    p = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=tab)
    k_gpu, perm_gpu = key_sort(rays, p, 8)
    k_or, perm_or = oracle_key_sort(rays, oracle.TWO_POINT, 64, lo, hi, tsrc=oracle.T_ADAPTIVE, table=ot)
    assert np.array_equal(k_gpu, k_or) and np.array_equal(perm_gpu, perm_or)
    tab.close()


def test_key_sort_given_estimate(soup):
    """GIVEN estimates (the oracle's hit distances; misses are +inf, which the
    key replaces by 4E) through the fused call."""
    tris, rays, lo, hi = soup
    hits, _ = oracle.BVH(tris).trace(rays.o_tmin, rays.d_tmax)
    t = np.ascontiguousarray(hits[:, 0], np.float32)
    tg = torch.from_numpy(t).cuda()
    for bits, radix_bits in ((64, 8), (48, 4), (20, 8)):
        p = rr.key_params(rr.RR_KEY_TWO_POINT, bits, lo, hi, t_source=rr.RR_T_GIVEN, t_given=tg)
        k_gpu, perm_gpu = key_sort(rays, p, radix_bits)
        k_or, perm_or = oracle_key_sort(rays, oracle.TWO_POINT, bits, lo, hi, tsrc=oracle.T_GIVEN, t_given=t)
        assert np.array_equal(k_gpu, k_or) and np.array_equal(perm_gpu, perm_or), (bits, radix_bits)


def test_key_sort_long_passes_and_workspace_reuse():
    """Enough rays for every key block to loop over several tiles and for the
    digit passes to take the four-blocks-per-SM form (at least eight 3072-key
    tiles per SM), one workspace reused across calls of both entry points:
    each call starts its counts from zero."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = (8 * sms + 1) * 3072 + 5
    tris = W.scene_box_soup(seed=4)
    lo, hi = W.scene_aabb(tris)
    ws = rr.sort_workspace(n, 64, 8)
    for seed in (4, 5):
        rays = W.rays_box_soup(tris, n=n, seed=seed)
        p = rr.key_params(rr.RR_KEY_AILA, 64, lo, hi)
        k_gpu, perm_gpu = key_sort(rays, p, 8, ws=ws)
        k_or, perm_or = oracle_key_sort(rays, oracle.AILA, 64, lo, hi)
        assert np.array_equal(k_gpu, k_or) and np.array_equal(perm_gpu, perm_or), seed
        # the same workspace through the two-call form in between
        keys = torch.from_numpy(k_or.view(np.int64)).cuda()
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        rr.rr_sort(keys, None, perm, n, 64, 8, ws)
        torch.cuda.synchronize()
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), perm_or)
    assert rr.rr_device_error() == 0


def test_key_sort_launches_one_kernel_fewer(soup):
    tris, rays, lo, hi = soup
    n = len(rays)
    o, d, _ = rr.to_device_rays(rays)
    p = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = rr.sort_workspace(n, 64, 8)
    c0 = rr.rr_kernel_launch_count()
    rr.rr_compute_keys(o, d, p, keys)
    rr.rr_sort(keys, None, perm, n, 64, 8, ws)
    c1 = rr.rr_kernel_launch_count()
    rr.rr_key_sort(o, d, p, keys, perm, 8, ws)
    c2 = rr.rr_kernel_launch_count()
    torch.cuda.synchronize()
    assert c1 - c0 == 1 + 1 + 8 and c2 - c1 == 1 + 8


def test_key_sort_rejects_bad_arguments(soup):
    tris, rays, lo, hi = soup
    n = 1000
    o, d, _ = rr.to_device_rays(rays.subset(np.arange(n)))
    p = rr.key_params(rr.RR_KEY_AILA, 64, lo, hi)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    ws = rr.sort_workspace(n, 64, 8)
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, p, keys, perm, 5, ws)  # radix width
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, p, keys, perm, 8, torch.empty(64, dtype=torch.uint8, device="cuda"))
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, p, keys, keys.view(torch.int32)[:n], 8, ws)  # perm aliases keys
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, p, o.view(torch.int64)[:n], perm, 8, ws)  # keys overwrite the rays
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, p, keys, perm, 8, rr.sort_workspace(n, 32, 8))  # workspace for 32-bit keys
    bad = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE)  # no table
    with pytest.raises(rr.RRError):
        rr.rr_key_sort(o, d, bad, keys, perm, 8, ws)
    rr.rr_key_sort(o, d, p, keys, perm, 8, ws, n=0)  # n == 0 is a no-op
    torch.cuda.synchronize()
    assert rr.rr_device_error() == 0
