"""Comparison of GPU hits with the oracle's closest hits.

The rule for the trace: the same triangle id and t within 1e-5 relative.  A
different id is accepted only where two candidate t values tie within 1e-5:
the oracle re-evaluates the GPU's triangle in binary64 and must meet its
plane, inside the triangle up to the kernel's rounding error, at that
distance.

Any remaining disagreement must be one that the kernel's binary32
Moller-Trumbore test cannot decide the way the binary64 oracle does.  For each
triangle involved, ``fp32_bounds`` gives first-order forward error bounds of
the kernel's barycentrics and distance (the gamma_n bounds of Higham, Accuracy
and Stability of Numerical Algorithms, 2002, section 3.1, applied to the
kernel's sequence of products, cross products and dot products).  A
triangle's decision is *uncertain* when its binary64 margin min(u, v, 1-u-v)
lies within twice its barycentric bound (never less than EDGE_FLOOR, the
1e-6 of the stated reading), or its distance lies within twice its distance
bound of tmin or tmax.  A disagreement is excused only when

  - the GPU's triangle (if any) is met by the ray up to its bounds,
  - at least one of the two decisions is uncertain,
  - a certain oracle hit is matched by a GPU hit that is no farther, and a
    certain GPU hit by an oracle hit that is no farther;

every other disagreement fails.  Excused rays are counted per class (edge:
a barycentric margin inside its bound; interval end: a distance inside its
bound of tmin or tmax) and their number must stay within AMBIGUOUS_FRACTION
of the rays (at least one).  Every comparison is recorded in ``LOG`` so that
the test session prints the counts per test.
"""
import numpy as np

import oracle

T_REL = 1e-5
EDGE_FLOOR = 1e-6
BOUND_FACTOR = 2.0
AMBIGUOUS_FRACTION = 1e-5
U32 = 2.0 ** -24  # unit roundoff of binary32

LOG = []  # (label, result dict) of every comparison in this process
CURRENT_TEST = None  # set per test by conftest.py


def _gamma(k):
    return k * U32 / (1.0 - k * U32)


def _abs_cross(a, b):
    return np.array([abs(a[1] * b[2]) + abs(a[2] * b[1]),
                     abs(a[2] * b[0]) + abs(a[0] * b[2]),
                     abs(a[0] * b[1]) + abs(a[1] * b[0])])


def fp32_bounds(o, d, tri):
    """(ok, t, u, v, err_bary, err_t): the binary64 Moller-Trumbore solution for
    the ray (o, d) and the triangle (9 floats, as given to the BVH builder),
    and first-order bounds of the error of the kernel's binary32 evaluation of
    u, v, 1-u-v (err_bary, the largest of the three) and t.

    The kernel forms e1 = fl(v1 - v0), e2 = fl(v2 - v0), tv = fl(o - v0),
    pv = d x e2, det = e1 . pv, u = (tv . pv) / det, qv = tv x e1,
    v = (d . qv) / det, t = (e2 . qv) / det.  With P = |d| x |e2| and
    Q = |tv| x |e1| (cross products of absolute values), each numerator N with
    absolute-value sum A is off by at most gamma_k * A for the k roundings on
    its longest path, and a quotient N / det picks up the relative error of
    det (gamma_8 * |e1| . P / |det|) and one rounding."""
    ok, t, u, v = oracle.ray_plane_barycentrics(o, d, tri)
    if not ok:
        return False, np.nan, np.nan, np.nan, np.inf, np.inf
    tr = np.asarray(tri, np.float64)
    v0 = tr[0:3]
    e1 = tr[3:6] - v0
    e2 = tr[6:9] - v0
    tv = np.asarray(o, np.float64) - v0
    dd = np.asarray(d, np.float64)
    P = _abs_cross(dd, e2)
    Q = _abs_cross(tv, e1)
    det_abs = abs(float(np.dot(e1, np.cross(dd, e2))))
    if det_abs == 0.0:
        return False, np.nan, np.nan, np.nan, np.inf, np.inf
    rel_det = _gamma(8) * float(np.dot(np.abs(e1), P)) / det_abs
    eu = _gamma(7) * float(np.dot(np.abs(tv), P)) / det_abs + (rel_det + U32) * abs(u)
    ev = _gamma(7) * float(np.dot(np.abs(dd), Q)) / det_abs + (rel_det + U32) * abs(v)
    ew = eu + ev + U32 * (abs(u) + abs(v) + 1.0)
    et = _gamma(7) * float(np.dot(np.abs(e2), Q)) / det_abs + (rel_det + U32) * abs(t)
    return True, t, u, v, max(eu, ev, ew), et


class _Tri:
    """One triangle's binary64 verdict for a ray, with the kernel's bounds."""

    def __init__(self, o, d, tris, tri_id, tmin, tmax):
        self.id = tri_id
        self.ok, self.t, u, v, eb, et = fp32_bounds(o, d, tris[tri_id])
        self.margin = min(u, v, 1.0 - u - v) if self.ok else -np.inf
        self.eb = max(EDGE_FLOOR, BOUND_FACTOR * eb)
        self.et = BOUND_FACTOR * et
        self.edge = self.ok and abs(self.margin) < self.eb
        self.end = self.ok and (abs(self.t - tmin) < self.et or abs(self.t - tmax) < self.et)
        # met by the ray up to the kernel's rounding
        self.plausible = self.ok and self.margin >= -self.eb and tmin - self.et < self.t < tmax + self.et

    @property
    def uncertain(self):
        return self.edge or self.end


def _classify(o, d, tris, gt, ot, g_t, o_t, tmin, tmax):
    """None (a definite mismatch), 'tie', 'edge' or 'interval_end'."""
    tol = T_REL * abs(o_t) if np.isfinite(o_t) else 0.0
    G = _Tri(o, d, tris, gt, tmin, tmax) if gt != oracle.MISS else None
    O = _Tri(o, d, tris, ot, tmin, tmax) if ot != oracle.MISS else None
    if G is not None and O is not None and gt != ot:
        if G.ok and G.margin >= -G.eb and abs(g_t - o_t) <= tol and abs(G.t - o_t) <= tol:
            return "tie"
    if G is not None and not G.plausible:
        return None
    if not ((G is not None and G.uncertain) or (O is not None and O.uncertain)):
        return None
    if O is not None and not O.uncertain:  # a certain oracle hit: the GPU must hit no farther
        if G is None or not G.t < o_t + tol:
            return None
    if G is not None and not G.uncertain:  # a certain GPU hit: the oracle must hit no farther
        if O is None or not o_t < G.t + T_REL * abs(G.t):
            return None
    edge = (G is not None and G.edge) or (O is not None and O.edge)
    return "edge" if edge else "interval_end"


def _limit(n, max_ambiguous):
    return max(1, int(AMBIGUOUS_FRACTION * n)) if max_ambiguous is None else max_ambiguous


def compare(tris, o_tmin, d_tmax, gpu_hits, or_hits, or_info, max_ambiguous=None, label=None):
    """Returns a dict of counts; raises AssertionError on a definite mismatch
    or on more excused rays than the limit."""
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
    counts = {"tie": 0, "edge": 0, "interval_end": 0}
    excused, definite = [], []
    for i in bad:
        o = o_tmin[i, :3].astype(np.float64)
        d = d_tmax[i, :3].astype(np.float64)
        c = _classify(o, d, tris, int(g_tri[i]), int(o_tri[i]), float(g_t[i]), float(o_t[i]),
                      float(o_tmin[i, 3]), float(d_tmax[i, 3]))
        if c is None:
            definite.append(int(i))
            continue
        counts[c] += 1
        if c != "tie":
            excused.append(int(i))
    res = dict(n=n, ties=counts["tie"], ambiguous=len(excused), edge=counts["edge"],
               interval_end=counts["interval_end"], definite=len(definite), ambiguous_idx=excused,
               hit_rate=float(np.mean(o_tri != oracle.MISS)) if n else 0.0,
               limit=_limit(n, max_ambiguous),
               examples=[(i, float(gpu_hits[i, 0]), int(g_tri[i]), float(o_t[i]), int(o_tri[i]),
                          float(or_info[i, 1]), o_tmin[i].tolist(), d_tmax[i].tolist())
                         for i in excused[:4]])
    LOG.append((label or CURRENT_TEST, {k: res[k] for k in ("n", "ties", "edge", "interval_end", "definite", "limit")}))
    if definite:
        i = definite[0]
        raise AssertionError("hit mismatch on %d of %d rays, e.g. ray %d: gpu (t=%r, tri=%d) oracle (t=%r, "
                             "tri=%d, margin=%r)" % (len(definite), n, i, gpu_hits[i, 0], g_tri[i], o_t[i],
                                                     o_tri[i], or_info[i, 1]))
    assert len(excused) <= res["limit"], res
    return res


def compare_any_hit(tris, o_tmin, d_tmax, gpu_hits, or_hits, or_info, max_ambiguous=None, label=None):
    """Any-hit rule: a ray is occluded exactly when the oracle finds a closest
    hit; the triangle the GPU reports must itself be met inside (tmin, tmax) at
    the reported t (1e-5 relative).  A disagreement is excused only where the
    deciding triangle's test is uncertain in binary32, as in ``compare``."""
    tris = np.ascontiguousarray(tris, np.float32).reshape(-1, 9)
    n = o_tmin.shape[0]
    g_tri = np.ascontiguousarray(gpu_hits[:, 3]).view(np.uint32)
    o_tri = np.ascontiguousarray(or_hits[:, 3]).view(np.uint32)
    g_occ = g_tri != oracle.MISS
    o_occ = o_tri != oracle.MISS
    counts = {"edge": 0, "interval_end": 0}
    excused, definite = [], []
    for i in range(n):
        if not g_occ[i] and not o_occ[i]:
            continue
        o = o_tmin[i, :3].astype(np.float64)
        d = d_tmax[i, :3].astype(np.float64)
        tmin, tmax = float(o_tmin[i, 3]), float(d_tmax[i, 3])
        if g_occ[i]:
            G = _Tri(o, d, tris, int(g_tri[i]), tmin, tmax)
            inside = G.ok and G.margin >= 0.0 and tmin < G.t < tmax and \
                abs(gpu_hits[i, 0] - G.t) <= T_REL * abs(G.t)
            if inside and o_occ[i]:
                continue
            # a GPU hit the oracle does not confirm: excused only on the edge
            # of the GPU's own triangle, at the reported distance
            if G.plausible and G.uncertain and abs(gpu_hits[i, 0] - G.t) <= T_REL * abs(G.t) + G.et:
                counts["edge" if G.edge else "interval_end"] += 1
                excused.append(i)
            else:
                definite.append(i)
        else:
            O = _Tri(o, d, tris, int(o_tri[i]), tmin, tmax)
            if O.uncertain:
                counts["edge" if O.edge else "interval_end"] += 1
                excused.append(i)
            else:
                definite.append(i)
    res = dict(n=n, occluded=int(o_occ.sum()), ambiguous=len(excused), edge=counts["edge"],
               interval_end=counts["interval_end"], definite=len(definite), limit=_limit(n, max_ambiguous))
    LOG.append((label or CURRENT_TEST, {k: res[k] for k in ("n", "edge", "interval_end", "definite", "limit")}))
    if definite:
        i = definite[0]
        raise AssertionError("any-hit mismatch on %d of %d rays, e.g. ray %d: gpu (t=%r, tri=%d) oracle "
                             "(t=%r, tri=%d)" % (len(definite), n, i, gpu_hits[i, 0], g_tri[i], or_info[i, 0],
                                                 o_tri[i]))
    assert len(excused) <= res["limit"], res
    return res
