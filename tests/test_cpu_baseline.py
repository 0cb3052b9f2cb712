"""The bench's CPU baseline runs the oracle on every host core by splitting the
rays into ranges; its keys, permutation, hits and length table must be those
of the single-threaded oracle, bit for bit."""
import numpy as np
import pytest

import bench
import oracle
from paper_2506_11273_gb300 import workloads as W


@pytest.mark.parametrize("threads", [2, 3, 8])
def test_threaded_oracle_bounce_equals_single_thread(threads):
    tris = W.scene_terrain(seed=2, cells_x=64, cells_z=128, n_boxes=300)
    lo, hi = W.scene_aabb(tris)
    obvh = oracle.BVH(tris)
    rays = W.surface_rays(tris, 30001, seed=77)
    rays.o_tmin[::5] = rays.o_tmin[0]  # equal keys across the ranges: stability matters
    rays.d_tmax[::5] = rays.d_tmax[0]
    E = oracle.largest_extent(lo, hi)
    prime = W.surface_rays(tris, 5000, seed=5)
    ph, _ = obvh.trace(prime.o_tmin, prime.d_tmax)
    out = []
    for th in (1, threads):
        table = oracle.LengthTable(E)
        table.accumulate(lo, hi, prime.o_tmin, prime.d_tmax, ph)
        k, p, h = bench.oracle_bounce(lo, hi, rays, obvh, table, threads=th)
        out.append((k, p, h.view(np.uint32), table.sum.copy(), table.cnt.copy()))
    for a, b in zip(*out):
        assert np.array_equal(a, b)
    assert np.array_equal(out[0][1], oracle.stable_sort(out[0][0])[0])


def test_stable_merge_keeps_lower_indices_first():
    ka = np.array([1, 3, 3, 7], np.uint64)
    kb = np.array([0, 3, 3, 9], np.uint64)
    k, p = bench.stable_merge((ka, np.array([0, 1, 2, 3], np.uint32)), (kb, np.array([4, 5, 6, 7], np.uint32)))
    assert k.tolist() == [0, 1, 3, 3, 3, 3, 7, 9]
    assert p.tolist() == [4, 0, 1, 2, 5, 6, 3, 7]
