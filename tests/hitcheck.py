"""Comparison of GPU hits with the oracle's closest hits.

The rule for the trace: the same triangle id and t within 1e-5 relative.  A
different id is accepted only where two candidate t values tie within 1e-5:
the oracle re-evaluates the GPU's triangle in binary64 and must meet its
plane, inside or on the triangle, at that distance.  A remaining disagreement
is "edge-ambiguous" when the ray passes within EDGE_MARGIN (in barycentric
coordinates) of an edge of the oracle's triangle or of the GPU's triangle:
fp32 Moller-Trumbore cannot decide those rays as the binary64 oracle does.
The same holds for rays that graze a triangle's plane (|cos| < GRAZING_COS)
and for hits within 1e-5 of the ray's tmin or tmax, where the open interval
decides in fp32 what binary64 decides otherwise.  Their count must stay below
AMBIGUOUS_FRACTION of the rays; any other disagreement fails.
"""
import numpy as np

import oracle

T_REL = 1e-5
EDGE_MARGIN = 2e-4
GRAZING_COS = 1e-4
AMBIGUOUS_FRACTION = 1e-4


def _plane_hit(o, d, tris, tri_id):
    ok, t, u, v = oracle.ray_plane_barycentrics(o, d, tris[tri_id])
    return ok, t, min(u, v, 1.0 - u - v)


def _cos(d, tris, tri_id):
    t = tris[tri_id].astype(np.float64)
    n = np.cross(t[3:6] - t[0:3], t[6:9] - t[0:3])
    den = np.linalg.norm(n) * np.linalg.norm(d)
    return abs(float(np.dot(n, d))) / den if den > 0 else 0.0


def _near_interval_end(t, tmin, tmax):
    return abs(t - tmin) <= T_REL * max(1.0, abs(t)) or abs(t - tmax) <= T_REL * abs(t)


def compare(tris, o_tmin, d_tmax, gpu_hits, or_hits, or_info, max_ambiguous=None):
    """Returns a dict of counts; raises AssertionError on a definite mismatch."""
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    n = o_tmin.shape[0]
    g_tri = np.ascontiguousarray(gpu_hits[:, 3]).view(np.uint32)
    o_tri = np.ascontiguousarray(or_hits[:, 3]).view(np.uint32)
    g_t = gpu_hits[:, 0].astype(np.float64)
    o_t = or_info[:, 0]
    both_miss = (g_tri == oracle.MISS) & (o_tri == oracle.MISS)
    same = (g_tri == o_tri) & ~both_miss
    with np.errstate(invalid="ignore"):
        same_ok = same & (np.abs(g_t - o_t) <= T_REL * np.abs(o_t))
    bad = np.flatnonzero(~both_miss & ~same_ok)
    ties, ambiguous, definite = 0, [], []
    for i in bad:
        o = o_tmin[i, :3].astype(np.float64)
        d = d_tmax[i, :3].astype(np.float64)
        gt, ot = int(g_tri[i]), int(o_tri[i])
        tol = T_REL * abs(o_t[i])
        g_plane = _plane_hit(o, d, tris, gt) if gt != oracle.MISS else None
        if gt != oracle.MISS and ot != oracle.MISS and gt != ot:
            ok, tg, mg = g_plane
            if ok and mg >= -EDGE_MARGIN and abs(g_t[i] - o_t[i]) <= tol and abs(tg - o_t[i]) <= tol:
                ties += 1
                continue
        tmin, tmax = float(o_tmin[i, 3]), float(d_tmax[i, 3])
        amb = (ot != oracle.MISS and (or_info[i, 1] < EDGE_MARGIN or _cos(d, tris, ot) < GRAZING_COS
                                      or _near_interval_end(o_t[i], tmin, tmax))) or \
              (g_plane is not None and g_plane[0] and (abs(g_plane[2]) < EDGE_MARGIN or
                                                      _cos(d, tris, gt) < GRAZING_COS or
                                                      _near_interval_end(g_plane[1], tmin, tmax)))
        (ambiguous if amb else definite).append(int(i))
    res = dict(n=n, ties=ties, ambiguous=len(ambiguous), definite=len(definite), ambiguous_idx=ambiguous,
               hit_rate=float(np.mean(o_tri != oracle.MISS)) if n else 0.0,
               examples=[(i, float(gpu_hits[i, 0]), int(g_tri[i]), float(o_t[i]), int(o_tri[i]),
                          float(or_info[i, 1]), o_tmin[i].tolist(), d_tmax[i].tolist())
                         for i in ambiguous[:4]])
    if definite:
        i = definite[0]
        raise AssertionError("hit mismatch on %d of %d rays, e.g. ray %d: gpu (t=%r, tri=%d) oracle (t=%r, "
                             "tri=%d, margin=%r)" % (len(definite), n, i, gpu_hits[i, 0], g_tri[i], o_t[i],
                                                     o_tri[i], or_info[i, 1]))
    limit = max(1, AMBIGUOUS_FRACTION * n) if max_ambiguous is None else max_ambiguous
    assert len(ambiguous) <= limit, res
    return res


def compare_any_hit(tris, o_tmin, d_tmax, gpu_hits, or_hits, or_info, max_ambiguous=None):
    """Any-hit rule: a ray is occluded exactly when the oracle finds a closest
    hit; the triangle the GPU reports must itself be met inside (tmin, tmax) at
    the reported t (1e-5 relative).  Edge, grazing and interval-end rays are
    classified as in ``compare``."""
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    n = o_tmin.shape[0]
    g_tri = np.ascontiguousarray(gpu_hits[:, 3]).view(np.uint32)
    o_tri = np.ascontiguousarray(or_hits[:, 3]).view(np.uint32)
    g_occ = g_tri != oracle.MISS
    o_occ = o_tri != oracle.MISS
    ambiguous, definite = [], []
    for i in range(n):
        if not g_occ[i] and not o_occ[i]:
            continue
        o = o_tmin[i, :3].astype(np.float64)
        d = d_tmax[i, :3].astype(np.float64)
        tmin, tmax = float(o_tmin[i, 3]), float(d_tmax[i, 3])
        amb = False
        if g_occ[i]:
            gt = int(g_tri[i])
            ok, tp, mg = _plane_hit(o, d, tris, gt)
            inside = ok and mg >= 0.0 and tmin < tp < tmax and abs(gpu_hits[i, 0] - tp) <= T_REL * abs(tp)
            amb_g = ok and (abs(mg) < EDGE_MARGIN or _cos(d, tris, gt) < GRAZING_COS or
                            _near_interval_end(tp, tmin, tmax))
            if not inside:
                (ambiguous if amb_g else definite).append(i)
                continue
            if o_occ[i]:
                continue
            amb = amb_g
        else:
            ot = int(o_tri[i])
            amb = or_info[i, 1] < EDGE_MARGIN or _cos(d, tris, ot) < GRAZING_COS or \
                _near_interval_end(or_info[i, 0], tmin, tmax)
        (ambiguous if amb else definite).append(i)
    res = dict(n=n, occluded=int(o_occ.sum()), ambiguous=len(ambiguous), definite=len(definite))
    if definite:
        i = definite[0]
        raise AssertionError("any-hit mismatch on %d of %d rays, e.g. ray %d: gpu (t=%r, tri=%d) oracle "
                             "(t=%r, tri=%d)" % (len(definite), n, i, gpu_hits[i, 0], g_tri[i], or_info[i, 0],
                                                 o_tri[i]))
    limit = max(1, AMBIGUOUS_FRACTION * n) if max_ambiguous is None else max_ambiguous
    assert len(ambiguous) <= limit, res
    return res
