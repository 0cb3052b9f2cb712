"""Seeded synthetic scenes and ray wavefronts.

This module holds the input generators shared by the CUDA path, the tests and
the bench.  It contains none of the reordering method's arithmetic: no sorting
keys, no termination estimate, no sort, no gather, no ray/triangle or ray/box
intersection and no length table.  Everything here is numpy on the host, drawn
from ``numpy.random.Generator(PCG64(seed))`` so that the same seed gives the same
scene and rays on any machine with the same numpy.

The paper measures on public scenes (Bitterli 2016, McGuire 2017; Section 4)
with a wavefront path tracer (Section 4: next-event estimation, 8 spp, 1920x1080).
Those scenes are not available, so the synthetic scenes below stand in for
them.  Their triangle counts bracket the paper's 262k-2833k (Table 1), and the
path-tracer wavefronts have the paper's structure: camera rays, then secondary
rays that scatter off diffuse and glossy surfaces.

Layouts (shared with the C ABI):
  tris     float32 [T, 9]   v0.xyz, v1.xyz, v2.xyz per triangle
  o_tmin   float32 [N, 4]   origin.xyz, tmin
  d_tmax   float32 [N, 4]   direction.xyz (unit length), tmax
  payload  uint32  [N]      caller data carried through the reorder (pixel id)
  hits     float32 [N, 4]   t, u, v, tri (tri stored as uint32 bits; miss: t=inf, tri=0xFFFFFFFF)
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

MISS = 0xFFFFFFFF


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclass
class Rays:
    o_tmin: np.ndarray   # float32 [N,4]
    d_tmax: np.ndarray   # float32 [N,4]
    payload: np.ndarray  # uint32 [N]

    def __len__(self) -> int:
        return int(self.o_tmin.shape[0])

    def subset(self, idx) -> "Rays":
        return Rays(np.ascontiguousarray(self.o_tmin[idx]),
                    np.ascontiguousarray(self.d_tmax[idx]),
                    np.ascontiguousarray(self.payload[idx]))


def make_rays(o, d, tmin, tmax, payload) -> Rays:
    n = o.shape[0]
    o_tmin = np.empty((n, 4), np.float32)
    d_tmax = np.empty((n, 4), np.float32)
    o_tmin[:, :3] = o
    o_tmin[:, 3] = tmin
    d_tmax[:, :3] = d
    d_tmax[:, 3] = tmax
    return Rays(o_tmin, d_tmax, np.ascontiguousarray(payload, dtype=np.uint32))


# --------------------------------------------------------------------------
# small geometric helpers (float64)
# --------------------------------------------------------------------------

def _normalize(v):
    n = np.sqrt(np.sum(v * v, axis=-1, keepdims=True))
    n = np.where(n > 0, n, 1.0)
    return v / n


def _onb(n):
    """Orthonormal basis around unit vectors n [M,3] (Duff et al. 2017, branchless)."""
    sign = np.where(n[:, 2] >= 0, 1.0, -1.0)
    a = -1.0 / (sign + n[:, 2])
    b = n[:, 0] * n[:, 1] * a
    t = np.stack([1.0 + sign * n[:, 0] * n[:, 0] * a, sign * b, -sign * n[:, 0]], axis=1)
    bb = np.stack([b, sign + n[:, 1] * n[:, 1] * a, -n[:, 1]], axis=1)
    return t, bb


def _cosine_dirs(n, rng):
    """Cosine-weighted hemisphere directions about unit normals n [M,3]."""
    m = n.shape[0]
    r1 = rng.random(m)
    r2 = rng.random(m)
    phi = 2.0 * math.pi * r1
    sin_t = np.sqrt(r2)
    cos_t = np.sqrt(1.0 - r2)
    t, b = _onb(n)
    d = (t * (np.cos(phi) * sin_t)[:, None] + b * (np.sin(phi) * sin_t)[:, None]
         + n * cos_t[:, None])
    return _normalize(d)


def _phong_dirs(r, exponent, rng):
    """Directions about unit lobe axes r [M,3] with density proportional to cos^exponent."""
    m = r.shape[0]
    r1 = rng.random(m)
    r2 = rng.random(m)
    cos_a = r2 ** (1.0 / (exponent + 1.0))
    sin_a = np.sqrt(np.maximum(0.0, 1.0 - cos_a * cos_a))
    phi = 2.0 * math.pi * r1
    t, b = _onb(r)
    d = (t * (np.cos(phi) * sin_a)[:, None] + b * (np.sin(phi) * sin_a)[:, None]
         + r * cos_a[:, None])
    return _normalize(d)


def tri_geometry(tris: np.ndarray):
    """(v0, e1, e2, unit winding normal, area) in float64 for a [T,9] soup."""
    t = tris.astype(np.float64)
    v0 = t[:, 0:3]
    e1 = t[:, 3:6] - v0
    e2 = t[:, 6:9] - v0
    c = np.cross(e1, e2)
    area2 = np.sqrt(np.sum(c * c, axis=1))
    return v0, e1, e2, _normalize(c), 0.5 * area2


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def _box_tris(lo, hi, inward: bool):
    """12 triangles of axis-aligned boxes lo/hi [B,3]; winding normal inward or outward."""
    lo = np.asarray(lo, np.float64).reshape(-1, 3)
    hi = np.asarray(hi, np.float64).reshape(-1, 3)
    B = lo.shape[0]
    out = []
    for axis in range(3):
        u, v = (axis + 1) % 3, (axis + 2) % 3
        for side in (0, 1):
            plane = np.where(side == 0, lo[:, axis], hi[:, axis])
            quad = np.zeros((B, 4, 3))
            quad[:, :, axis] = plane[:, None]
            # corners (u,v): (lo,lo) (hi,lo) (hi,hi) (lo,hi)
            quad[:, 0, u], quad[:, 0, v] = lo[:, u], lo[:, v]
            quad[:, 1, u], quad[:, 1, v] = hi[:, u], lo[:, v]
            quad[:, 2, u], quad[:, 2, v] = hi[:, u], hi[:, v]
            quad[:, 3, u], quad[:, 3, v] = lo[:, u], hi[:, v]
            # winding (0,1,2) has normal +axis (u x v = axis for a cyclic triple)
            want_plus = (side == 0) == inward
            order = [(0, 1, 2), (0, 2, 3)] if want_plus else [(0, 2, 1), (0, 3, 2)]
            for a, b, c in order:
                out.append(np.concatenate([quad[:, a], quad[:, b], quad[:, c]], axis=1))
    # interleave per box: box i's 12 triangles are contiguous
    arr = np.stack(out, axis=1)  # [B,12,9]
    return arr.reshape(B * 12, 9)


def scene_box_soup(seed: int = 1, n_random: int = 4096, jitter: float = 0.02) -> np.ndarray:
    """Tiny scene: the unit box [0,1]^3 (12 triangles, inward winding) enclosing
    ``n_random`` small triangles (centroids uniform in [0,1]^3, vertices at
    centroid + U[-jitter, jitter]^3).  4,108 triangles at the defaults."""
    rng = rng_for(seed)
    box = _box_tris(np.zeros(3), np.ones(3), inward=True)
    c = rng.random((n_random, 3))
    v = c[:, None, :] + rng.uniform(-jitter, jitter, size=(n_random, 3, 3))
    soup = np.concatenate([box, v.reshape(n_random, 9)], axis=0)
    return np.ascontiguousarray(soup.astype(np.float32))


def _value_noise_fbm(x, z, rng, base=(8, 16), octaves=5, gain=0.5, extent=(1.0, 2.0)):
    """fBm of value noise on lattices of base*2^o cells over [0,ex]x[0,ez], in [0,1]."""
    total = np.zeros_like(x)
    amp = 1.0
    norm = 0.0
    for o in range(octaves):
        nx, nz = base[0] << o, base[1] << o
        lat = rng.random((nx + 1, nz + 1))
        fx = np.clip(x / extent[0], 0.0, 1.0) * nx
        fz = np.clip(z / extent[1], 0.0, 1.0) * nz
        ix = np.minimum(fx.astype(np.int64), nx - 1)
        iz = np.minimum(fz.astype(np.int64), nz - 1)
        tx = fx - ix
        tz = fz - iz
        sx = tx * tx * (3.0 - 2.0 * tx)
        sz = tz * tz * (3.0 - 2.0 * tz)
        a = lat[ix, iz] * (1 - sx) + lat[ix + 1, iz] * sx
        b = lat[ix, iz + 1] * (1 - sx) + lat[ix + 1, iz + 1] * sx
        total += amp * (a * (1 - sz) + b * sz)
        norm += amp
        amp *= gain
    return total / norm


def _valley(x, z):
    """Smooth valley the terrain sits in: walls rise toward x=0, x=1 and z=2."""
    return (2.0 * x - 1.0) ** 2 + (z / 2.0) ** 4


def scene_terrain(seed: int = 2, cells_x: int = 512, cells_z: int = 1024,
                  n_boxes: int = 10000, noise: float = 0.15) -> np.ndarray:
    """Displaced-grid heightfield over x in [0,1], z in [0,2] (2 triangles per
    cell; height = a smooth valley (2x-1)^2 + (z/2)^4 plus ``noise`` * fBm value
    noise of 5 octaves, base lattice 8x16, gain 0.5) and ``n_boxes`` axis-aligned
    boxes of 12 triangles each (centre x~U[0,1], z~U[0,2], y = valley + U[0,0.3],
    half-extents U[0.002,0.01]).

    The valley keeps most camera and secondary rays inside the scene, as in
    the paper's interior scenes.  Defaults give 1,048,576 + 120,000 =
    1,168,576 triangles; 1024x2048 cells with 40,000 boxes give
    4,194,304 + 480,000 = 4,674,304."""
    rng = rng_for(seed)
    xs = np.linspace(0.0, 1.0, cells_x + 1)
    zs = np.linspace(0.0, 2.0, cells_z + 1)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    Y = noise * _value_noise_fbm(X, Z, rng) + _valley(X, Z)
    V = np.stack([X, Y, Z], axis=-1)  # [cx+1, cz+1, 3]
    v00 = V[:-1, :-1].reshape(-1, 3)
    v10 = V[1:, :-1].reshape(-1, 3)
    v01 = V[:-1, 1:].reshape(-1, 3)
    v11 = V[1:, 1:].reshape(-1, 3)
    # winding with +y normals: (v00, v01, v11) and (v00, v11, v10)
    t1 = np.concatenate([v00, v01, v11], axis=1)
    t2 = np.concatenate([v00, v11, v10], axis=1)
    hf = np.stack([t1, t2], axis=1).reshape(-1, 9)
    bx = rng.random(n_boxes)
    bz = rng.random(n_boxes) * 2.0
    by = _valley(bx, bz) + rng.random(n_boxes) * 0.3
    cen = np.stack([bx, by, bz], axis=1)
    half = rng.uniform(0.002, 0.01, size=(n_boxes, 3))
    boxes = _box_tris(cen - half, cen + half, inward=False)
    soup = np.concatenate([hf, boxes], axis=0)
    return np.ascontiguousarray(soup.astype(np.float32))


def scene_aabb(tris: np.ndarray):
    v = tris.reshape(-1, 3)
    return v.min(axis=0).astype(np.float32), v.max(axis=0).astype(np.float32)


# --------------------------------------------------------------------------
# rays
# --------------------------------------------------------------------------

def surface_points(tris: np.ndarray, n: int, rng: np.random.Generator):
    """Points uniform by area on the soup: (points [n,3] f64, tri ids [n], unit winding normals [n,3])."""
    v0, e1, e2, nrm, area = tri_geometry(tris)
    p = area / area.sum()
    ids = rng.choice(tris.shape[0], size=n, p=p)
    r1 = rng.random(n)
    r2 = rng.random(n)
    s = np.sqrt(r1)
    b1 = s * (1.0 - r2)
    b2 = s * r2
    pts = v0[ids] + e1[ids] * b1[:, None] + e2[ids] * b2[:, None]
    return pts, ids, nrm[ids]


def rays_box_soup(tris: np.ndarray, n: int = 65536, seed: int = 1,
                  tmin: float = 1e-4) -> Rays:
    """Secondary rays for the tiny scene: origins uniform by area on the
    triangles, cosine-weighted directions about the winding normal, shuffled
    (Fisher-Yates via ``Generator.permutation``); tmin=1e-4, tmax=+inf."""
    rng = rng_for(seed * 7919 + 17)
    pts, _, nrm = surface_points(tris, n, rng)
    d = _cosine_dirs(nrm, rng)
    perm = rng.permutation(n)
    return make_rays(pts[perm].astype(np.float32), d[perm].astype(np.float32),
                     np.float32(tmin), np.float32(np.inf), perm.astype(np.uint32))


@dataclass
class Camera:
    pos: tuple = (0.5, 0.6, 0.1)
    look_at: tuple = (0.5, 0.2, 1.2)
    vfov_deg: float = 60.0
    width: int = 1920
    height: int = 1080


def camera_rays(cam: Camera, seed: int = 2) -> Rays:
    """One jittered primary ray per pixel, in pixel (row-major) order; payload = pixel id."""
    rng = rng_for(seed * 104729 + 3)
    W, H = cam.width, cam.height
    pos = np.asarray(cam.pos, np.float64)
    fwd = _normalize(np.asarray(cam.look_at, np.float64) - pos)
    right = _normalize(np.cross(fwd, np.array([0.0, 1.0, 0.0])))
    up = np.cross(right, fwd)
    th = math.tan(math.radians(cam.vfov_deg) * 0.5)
    aspect = W / H
    py, px = np.divmod(np.arange(W * H, dtype=np.int64), W)
    jx = rng.random(W * H)
    jy = rng.random(W * H)
    sx = (2.0 * (px + jx) / W - 1.0) * th * aspect
    sy = (1.0 - 2.0 * (py + jy) / H) * th
    d = _normalize(fwd[None, :] + sx[:, None] * right[None, :] + sy[:, None] * up[None, :])
    o = np.broadcast_to(pos, d.shape)
    return make_rays(o.astype(np.float32), d.astype(np.float32), np.float32(0.0),
                     np.float32(np.inf), np.arange(W * H, dtype=np.uint32))


def material_is_glossy(tri_ids: np.ndarray) -> np.ndarray:
    """Material by hash of triangle id: 30% Phong (exponent 100), 70% Lambertian."""
    h = (tri_ids.astype(np.uint64) * np.uint64(2654435761)) & np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(15)
    return (h % np.uint64(1000)) < np.uint64(300)


PHONG_EXPONENT = 100.0


def scatter(tris: np.ndarray, points, tri_ids, incoming, rng, tmin: float = 1e-4):
    """BSDF sampling at surface points.  Returns (dirs [M,3] f64, alive [M] bool).

    Lambertian: cosine-weighted about the normal facing the incoming ray.
    Phong: cos^100 lobe about the mirror direction; samples below the surface die."""
    n = tri_geometry(tris[tri_ids])[3]
    flip = np.sum(n * incoming, axis=1) > 0
    n[flip] = -n[flip]
    glossy = material_is_glossy(tri_ids)
    d = np.empty_like(n)
    alive = np.ones(n.shape[0], bool)
    if (~glossy).any():
        d[~glossy] = _cosine_dirs(n[~glossy], rng)
    if glossy.any():
        i = incoming[glossy]
        ng = n[glossy]
        r = _normalize(i - 2.0 * np.sum(i * ng, axis=1, keepdims=True) * ng)
        dg = _phong_dirs(r, PHONG_EXPONENT, rng)
        d[glossy] = dg
        alive[np.flatnonzero(glossy)[np.sum(dg * ng, axis=1) <= 0]] = False
    return d, alive


def next_bounce(tris: np.ndarray, rays: Rays, hits: np.ndarray, bounce: int, seed: int,
                rr_after: int = 2, survival: float = 0.7, tmin: float = 1e-4) -> Rays:
    """Path-tracer shading step: from the rays of ``bounce`` (1-based) and their
    closest hits, build the compacted wavefront of bounce+1.  Misses terminate;
    Russian roulette with ``survival`` applies once ``bounce >= rr_after``.
    The order of surviving rays is kept (stream compaction)."""
    rng = rng_for(seed * 1_000_003 + bounce)
    tri = hits[:, 3].view(np.uint32)
    hit = tri != MISS
    idx = np.flatnonzero(hit)
    o = rays.o_tmin[idx, :3].astype(np.float64)
    d_in = rays.d_tmax[idx, :3].astype(np.float64)
    t = hits[idx, 0].astype(np.float64)
    p = o + d_in * t[:, None]
    dirs, alive = scatter(tris, p, tri[idx], d_in, rng, tmin)
    if bounce >= rr_after:
        alive &= rng.random(idx.shape[0]) < survival
    keep = np.flatnonzero(alive)
    return make_rays(p[keep].astype(np.float32), dirs[keep].astype(np.float32), np.float32(tmin),
                     np.float32(np.inf), rays.payload[idx[keep]])


def surface_rays(tris: np.ndarray, n: int, seed: int, eye=(0.5, 0.6, 0.1),
                 tmin: float = 1e-4) -> Rays:
    """Trace-free stand-in for a secondary wavefront: origins uniform by area,
    directions sampled from the surface's BSDF as if lit from ``eye`` (occlusion
    ignored), in random order.  Used where an input must not depend on a trace."""
    rng = rng_for(seed * 7 + 11)
    pts, ids, _ = surface_points(tris, n, rng)
    incoming = _normalize(pts - np.asarray(eye, np.float64)[None, :])
    d, alive = scatter(tris, pts, ids, incoming, rng, tmin)
    # dead glossy samples are re-drawn as mirror directions so every ray is valid
    if (~alive).any():
        dead = np.flatnonzero(~alive)
        nn = tri_geometry(tris[ids[dead]])[3]
        flip = np.sum(nn * incoming[dead], axis=1) > 0
        nn[flip] = -nn[flip]
        i = incoming[dead]
        d[dead] = _normalize(i - 2.0 * np.sum(i * nn, axis=1, keepdims=True) * nn)
    return make_rays(pts.astype(np.float32), d.astype(np.float32), np.float32(tmin),
                     np.float32(np.inf), np.arange(n, dtype=np.uint32))


def random_rays_in_box(n: int, lo, hi, seed: int, tmin: float = 0.0, tmax: float = np.inf) -> Rays:
    """Uniform origins in [lo,hi] and uniform unit directions (for edge-case tests)."""
    rng = rng_for(seed)
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    o = lo + rng.random((n, 3)) * (hi - lo)
    d = _normalize(rng.normal(size=(n, 3)))
    return make_rays(o.astype(np.float32), d.astype(np.float32), np.float32(tmin),
                     np.float32(tmax), np.arange(n, dtype=np.uint32))


def shadow_rays(tris: np.ndarray, n: int, seed: int, light_center=None, light_frac: float = 0.05,
                tmin: float = 1e-4) -> Rays:
    """Next-event-estimation shadow rays: origins uniform by area on the soup,
    each aimed at a uniform point of a square area light whose side is
    ``light_frac`` of the largest scene extent (the evaluation setup of
    Section 4), placed above the scene's centre unless ``light_center`` is given.
    d = light point - origin (not normalised), so the segment is t in
    (tmin, 1 - 1e-4); in random order."""
    rng = rng_for(seed * 13 + 5)
    lo, hi = scene_aabb(tris)
    lo = lo.astype(np.float64)
    hi = hi.astype(np.float64)
    E = float(np.max(hi - lo))
    c = np.array([(lo[0] + hi[0]) / 2, hi[1] + 0.05 * E, (lo[2] + hi[2]) / 2]) if light_center is None \
        else np.asarray(light_center, np.float64)
    pts, _, _ = surface_points(tris, n, rng)
    side = light_frac * E
    lp = c[None, :] + np.stack([(rng.random(n) - 0.5) * side, np.zeros(n), (rng.random(n) - 0.5) * side], axis=1)
    d = lp - pts
    perm = rng.permutation(n)
    return make_rays(pts[perm].astype(np.float32), d[perm].astype(np.float32), np.float32(tmin),
                     np.float32(1.0 - 1e-4), perm.astype(np.uint32))


def request_rays(tris: np.ndarray, n: int, kind: str, seed: int, eye=(0.5, 0.6, 0.1),
                 tmin: float = 1e-4) -> Rays:
    """Secondary rays of one serving request: origins uniform by area, in random
    order.  ``kind`` "diffuse": cosine-weighted about the normal facing ``eye``;
    "glossy": the Phong-100 lobe about the mirror direction of the ray from
    ``eye`` (samples below the surface are folded back to the mirror direction)."""
    rng = rng_for(seed * 31 + (7 if kind == "glossy" else 3))
    pts, ids, _ = surface_points(tris, n, rng)
    incoming = _normalize(pts - np.asarray(eye, np.float64)[None, :])
    nn = tri_geometry(tris[ids])[3]
    flip = np.sum(nn * incoming, axis=1) > 0
    nn[flip] = -nn[flip]
    if kind == "glossy":
        r = _normalize(incoming - 2.0 * np.sum(incoming * nn, axis=1, keepdims=True) * nn)
        d = _phong_dirs(r, PHONG_EXPONENT, rng)
        below = np.sum(d * nn, axis=1) <= 0
        d[below] = r[below]
    else:
        d = _cosine_dirs(nn, rng)
    return make_rays(pts.astype(np.float32), d.astype(np.float32), np.float32(tmin),
                     np.float32(np.inf), np.arange(n, dtype=np.uint32))


def shadow_rays_to_light(points: np.ndarray, center, side: float, seed: int, tmin: float = 1e-4) -> Rays:
    """Shadow rays from given surface points (e.g. a wavefront's hit points, in
    their order) to uniform points of a square area light of side ``side``
    centred at ``center`` (horizontal, as in ``shadow_rays``); d = light point -
    origin, t in (tmin, 1 - 1e-4)."""
    rng = rng_for(seed * 17 + 9)
    n = points.shape[0]
    c = np.asarray(center, np.float64)
    lp = c[None, :] + np.stack([(rng.random(n) - 0.5) * side, np.zeros(n), (rng.random(n) - 0.5) * side], axis=1)
    d = lp - points.astype(np.float64)
    return make_rays(points.astype(np.float32), d.astype(np.float32), np.float32(tmin), np.float32(1.0 - 1e-4),
                     np.arange(n, dtype=np.uint32))
