"""CPU checks of the hit comparison rule (tests/hitcheck.py) that every trace
parity test applies: a hit list equal to the oracle's passes, and a planted
mistake in the GPU side (a dropped hit, another triangle, a wrong distance) is
reported as a definite mismatch; the binary32 error bounds grow as the ray
grazes the triangle's plane and vanish for a well-conditioned hit."""
import numpy as np
import pytest

import hitcheck
import oracle
from paper_2506_11273_gb300 import workloads as W

MISS_F = np.array([oracle.MISS], np.uint32).view(np.float32)[0]


@pytest.fixture(scope="module")
def soup():
    tris = W.scene_box_soup(seed=4, n_random=512)
    rays = W.rays_box_soup(tris, n=8192, seed=4)
    h, info = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
    return tris, rays, h, info


def test_identical_hits_pass(soup):
    tris, rays, h, info = soup
    res = hitcheck.compare(tris, rays.o_tmin, rays.d_tmax, h.copy(), h, info, label="identical")
    assert res["definite"] == 0 and res["ambiguous"] == 0 and res["ties"] == 0


@pytest.mark.parametrize("plant", ["miss", "other_triangle", "far_t", "spurious_hit"])
def test_planted_mistakes_are_definite(soup, plant):
    tris, rays, h, info = soup
    hit = h[:, 3].view(np.uint32) != oracle.MISS
    # the hit with the clearest margin: no binary32 rounding can excuse it
    i = int(np.argmax(np.where(hit, info[:, 1], -1.0)))
    g = h.copy()
    if plant == "miss":
        g[i, 0], g[i, 3] = np.inf, MISS_F
    elif plant == "other_triangle":
        g[i, 3] = np.array([(int(h[i, 3].view(np.uint32)) + 1) % len(tris)], np.uint32).view(np.float32)[0]
    elif plant == "far_t":
        g[i, 0] *= 1.001
    else:  # a hit reported for a ray the oracle finds no hit for
        j = int(np.flatnonzero(~hit)[0]) if (~hit).any() else None
        if j is None:
            pytest.skip("no missing ray in this scene")
        g[j] = h[i]
    with pytest.raises(AssertionError, match="mismatch"):
        hitcheck.compare(tris, rays.o_tmin, rays.d_tmax, g, h, info, label="planted")


def test_error_bounds_grow_when_grazing():
    """The bounds scale like 1/|cos| of the angle between ray and plane: a
    ray at 1e-4 from the plane gets bounds 10^3 times those of a ray through
    the plane's normal, both aimed at the same point."""
    tri = np.array([0.1, 0.2, 0.3, 1.3, 0.4, 0.1, 0.3, 1.1, 0.7], np.float32)
    v0, v1, v2 = tri[:3].astype(np.float64), tri[3:6].astype(np.float64), tri[6:].astype(np.float64)
    p = v0 + 0.3 * (v1 - v0) + 0.3 * (v2 - v0)
    n = np.cross(v1 - v0, v2 - v0)
    n /= np.linalg.norm(n)
    along = (v1 - v0) / np.linalg.norm(v1 - v0)
    res = {}
    for eps in (1.0, 1e-4):
        d = along + eps * n
        ok, t, u, v, eb, et = hitcheck.fp32_bounds(p - d, d, tri)
        assert ok and abs(t - 1.0) < 1e-9 and abs(u - 0.3) < 1e-9 and abs(v - 0.3) < 1e-9
        res[eps] = (eb, et)
    assert res[1.0][0] < 1e-5 and res[1.0][1] < 1e-5
    assert res[1e-4][0] > 1e3 * res[1.0][0] and res[1e-4][1] > 1e3 * res[1.0][1]
