"""GPU parity at the benchmark sizes, in the launch configurations bench.py times.

* Path tracer (1,168,576 triangles), a 1,196,335-ray wavefront (the bounce-3
  size) through the timed step: Two Point key with the adaptive estimate at 64
  bits and its 8-bit radix sort in one rr_key_sort call, gather, trace, then
  the length-table update.
  Every key, the whole permutation and every reordered ray are compared; hits
  on a 20,000-ray sample; the table after the update against the oracle's.
* Batched: 32 wavefronts (17,808,070 rays) over 4 resident scenes as one graph
  with the configuration the autotuner picks on this workload (24-bit keys,
  8-bit digits): the whole batch permutation, hits on a sample.
* Served: full-size requests (up to 4M rays) against the largest resident
  scenes, alone and in a mix: identical hits, and correct on a sample.

The rays are trace-free stand-ins (origins on the surfaces, BSDF directions)
so that no oracle input depends on the CUDA path; the table is built by the
oracle from its own hits and written to the device.
"""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def test_path_tracer_step_full_size():
    from test_gpu_trace import check_table_close
    tris = W.scene_terrain(seed=2)
    assert tris.shape[0] == 1168576
    lo, hi = W.scene_aabb(tris)
    bvh, obvh = rr.BVH(tris), oracle.BVH(tris)
    E = oracle.largest_extent(lo, hi)
    prime = W.surface_rays(tris, 200000, seed=11)
    ph, _ = obvh.trace(prime.o_tmin, prime.d_tmax)
    ot = oracle.LengthTable(E)
    ot.accumulate(lo, hi, prime.o_tmin, prime.d_tmax, ph)
    table = rr.LengthTable(lo, hi)
    table.write(ot.sum, ot.cnt)
    rays = W.surface_rays(tris, 1196335, seed=12)
    n = len(rays)
    o, d, p = rr.to_device_rays(rays)
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    so, sd, sp = torch.empty_like(o), torch.empty_like(d), torch.empty_like(p)
    hits = torch.empty(n, 4, device="cuda")
    params = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
    ws = rr.sort_workspace(n, 64, 8)
    rr.rr_key_sort(o, d, params, keys, perm, 8, ws)
    # the two-call form (keys, then the sort with its own counting pass), on
    # the same table before the trace updates it
    keys2 = torch.empty_like(keys)
    perm2 = torch.empty_like(perm)
    rr.rr_compute_keys(o, d, params, keys2)
    rr.rr_sort(keys2, None, perm2, n, 64, 8, rr.sort_workspace(n, 64, 8))
    rr.rr_permute(o, d, p, perm, so, sd, sp)
    rr.rr_trace_accumulate(bvh, so, sd, hits, table)
    k_or = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=oracle.T_ADAPTIVE,
                               table=ot)
    assert np.array_equal(rr.keys_to_numpy(keys), k_or)
    p_or, _ = oracle.stable_sort(k_or)
    assert np.array_equal(rr.u32_to_numpy(perm), p_or)
    assert torch.equal(keys2, keys) and torch.equal(perm2, perm)
    oo, od, op = oracle.permute(rays.o_tmin, rays.d_tmax, rays.payload, p_or)
    assert np.array_equal(_bits(so.cpu().numpy()), _bits(oo))
    assert np.array_equal(_bits(sd.cpu().numpy()), _bits(od))
    assert np.array_equal(sp.cpu().numpy().view(np.uint32), op)
    g = hits.cpu().numpy()
    idx = np.sort(np.random.default_rng(5).choice(n, 20000, replace=False))
    h, info = obvh.trace(oo[idx], od[idx])
    res = compare(tris, oo[idx], od[idx], g[idx], h, info)
    assert res["hit_rate"] > 0.5
    # the table after the update: the oracle adds its own hits of every ray
    h_all, info_all = obvh.trace(oo, od)
    res_all = compare(tris, oo, od, g, h_all, info_all)
    cells = {oracle.table_cell(oo[i, :3], od[i, :3], lo, hi) for i in res_all["ambiguous_idx"]}
    ot.accumulate(lo, hi, oo, od, h_all)
    check_table_close(table, ot, ambiguous=max(res_all["ambiguous"], 1), exclude_cells=cells)
    assert rr.rr_device_error() == 0


def test_batched_full_size():
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(np.log(1e4), np.log(2e6), bench.BATCH_WAVEFRONTS)).astype(np.int64)
    which = rng.integers(0, len(bench.BATCH_SCENES), bench.BATCH_WAVEFRONTS)
    scenes = [W.scene_terrain(seed=40 + k, cells_x=cx, cells_z=cz, n_boxes=nb)
              for k, (cx, cz, nb) in enumerate(bench.BATCH_SCENES)]
    bvhs = [rr.BVH(t) for t in scenes]
    boxes = [W.scene_aabb(t) for t in scenes]
    fronts, rays = [], []
    for k in range(bench.BATCH_WAVEFRONTS):
        s = int(which[k])
        rays.append(W.surface_rays(scenes[s], int(sizes[k]), seed=500 + k))
        fronts.append((bvhs[s], None, boxes[s][0], boxes[s][1], int(sizes[k])))
    batch = rr.Batch(fronts, rr.RR_KEY_TWO_POINT, rr.RR_T_FIXED)
    n = batch.n
    assert n == 17808070
    o = torch.from_numpy(np.concatenate([r.o_tmin for r in rays])).cuda()
    d = torch.from_numpy(np.concatenate([r.d_tmax for r in rays])).cuda()
    hits = torch.empty(n, 4, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    batch.run(o, d, hits, rr.Batch.config(24, 8, 128), perm)
    g_perm = rr.u32_to_numpy(perm)
    g = hits.cpu().numpy()
    del o, d
    off = 0
    sample = np.random.default_rng(6)
    for k in range(bench.BATCH_WAVEFRONTS):
        s = int(which[k])
        lo, hi = boxes[s]
        r = rays[k]
        cnt = len(r)
        keys = oracle.compute_keys(oracle.TWO_POINT, 24, r.o_tmin, r.d_tmax, lo, hi)
        assert np.array_equal(g_perm[off:off + cnt], oracle.stable_sort(keys)[0] + np.uint32(off)), k
        idx = np.sort(sample.choice(cnt, min(cnt, 700), replace=False))
        h, info = _obvh(scenes, s).trace(r.o_tmin[idx], r.d_tmax[idx])
        compare(scenes[s], r.o_tmin[idx], r.d_tmax[idx], g[off + idx], h, info)
        off += cnt
    batch.close()
    assert rr.rr_device_error() == 0


def _obvh(scenes, s, cache={}):
    key = (id(scenes), s)
    if key not in cache:
        cache[key] = oracle.BVH(scenes[s])
    return cache[key]


def test_served_full_size_requests():
    picks = [0, 4, 7]  # 49,804, 999,648 and 4,000,502 triangles
    scenes = [W.scene_terrain(seed=60 + k, cells_x=bench.SERVE_SCENES[k][0], cells_z=bench.SERVE_SCENES[k][1],
                              n_boxes=bench.SERVE_SCENES[k][2]) for k in picks]
    assert scenes[2].shape[0] == 4000502
    bvhs = [rr.BVH(t) for t in scenes]
    reqs = [(2, W.request_rays(scenes[2], 4 << 20, "diffuse", seed=1)),
            (1, W.request_rays(scenes[1], 1 << 20, "glossy", seed=2)),
            (0, W.request_rays(scenes[0], 4097, "diffuse", seed=3)),
            (2, W.request_rays(scenes[2], 300000, "glossy", seed=4))]

    def serve(slots, together):
        srv = rr.Server(budget_bytes=120 << 30, slots=slots, max_batch_rays=1 << 25, key_bits=24, trace_block=128)
        for s in range(3):
            srv.add_scene(bvhs[s], *W.scene_aabb(scenes[s]))
        out = [np.zeros((len(r), 4), np.float32) for _, r in reqs]
        if together:
            ts = [srv.submit(s, r.o_tmin, r.d_tmax, h) for (s, r), h in zip(reqs, out)]
            for t in ts:
                srv.wait(t)
        else:
            for (s, r), h in zip(reqs, out):
                srv.wait(srv.submit(s, r.o_tmin, r.d_tmax, h))
        srv.close()
        return out

    alone = serve(1, False)
    mixed = serve(4, True)
    rng = np.random.default_rng(7)
    for (s, r), a, m in zip(reqs, alone, mixed):
        assert np.array_equal(_bits(a), _bits(m))
        idx = np.sort(rng.choice(len(r), min(len(r), 4000), replace=False))
        h, info = _obvh(scenes, s).trace(r.o_tmin[idx], r.d_tmax[idx])
        compare(scenes[s], r.o_tmin[idx], r.d_tmax[idx], m[idx], h, info)
    assert rr.rr_device_error() == 0
