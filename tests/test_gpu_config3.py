"""GPU parity at the scale-sweep size: 4,674,304 triangles (1024x2048-cell terrain
+ 40,000 boxes) and 8,294,400 camera rays (3840x2160), plus a trace-free
secondary wavefront of the same size.

Every key and the whole permutation are compared at 64 bits; hits of 20,000
sampled rays per wavefront are compared with the oracle BVH (itself pinned to
the brute-force definition).  The sweep's key widths 16/32/48 are checked on
the same rays, and the sort with 4- and 8-bit digits.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    tris = W.scene_terrain(seed=3, cells_x=1024, cells_z=2048, n_boxes=40000)
    assert tris.shape[0] == 4674304
    return tris, W.scene_aabb(tris)


@pytest.fixture(scope="module")
def wavefronts(scene):
    tris, _ = scene
    cam = W.camera_rays(W.Camera(width=3840, height=2160), seed=3)
    sec = W.surface_rays(tris, 8294400, seed=31)
    return {"camera": cam, "secondary": sec}


def test_trace_full_size_sampled(scene, wavefronts):
    tris, _ = scene
    bvh = rr.BVH(tris)
    info = bvh.info()
    assert info.n_tris == tris.shape[0]
    obvh = oracle.BVH(tris)
    rng = np.random.default_rng(3)
    for name, rays in wavefronts.items():
        o, d, _ = rr.to_device_rays(rays)
        hits = torch.empty(len(rays), 4, device="cuda")
        rr.rr_trace(bvh, o, d, hits)
        g = hits.cpu().numpy()
        idx = np.sort(rng.choice(len(rays), 20000, replace=False))
        sub = rays.subset(idx)
        h, inf = obvh.trace(sub.o_tmin, sub.d_tmax)
        res = compare(tris, sub.o_tmin, sub.d_tmax, g[idx], h, inf)
        assert res["hit_rate"] > 0.5, (name, res)
        del o, d, hits
    assert rr.rr_device_error() == 0


@pytest.mark.parametrize("bits", [16, 32, 48, 64])
def test_keys_and_sort_full_size(scene, wavefronts, bits):
    tris, (lo, hi) = scene
    rays = wavefronts["secondary"]
    o, d, _ = rr.to_device_rays(rays)
    keys = torch.empty(len(rays), dtype=rr.key_dtype(bits), device="cuda")
    rr.rr_compute_keys(o, d, rr.key_params(rr.RR_KEY_TWO_POINT, bits, lo, hi), keys)
    k_gpu = rr.keys_to_numpy(keys)
    k_or = oracle.compute_keys(oracle.TWO_POINT, bits, rays.o_tmin, rays.d_tmax, lo, hi)
    assert np.array_equal(k_gpu, k_or)
    perm_or, _ = oracle.stable_sort(k_or)
    for radix_bits in (8, 4):
        perm = torch.empty(len(rays), dtype=torch.int32, device="cuda")
        ws = rr.sort_workspace(len(rays), bits, radix_bits)
        rr.rr_sort(keys, None, perm, len(rays), bits, radix_bits, ws)
        assert np.array_equal(rr.u32_to_numpy(perm), perm_or), radix_bits
        del ws, perm
    assert rr.rr_device_error() == 0
