"""Child process of test_gpu_failure.py: the config-1 bounce (keys, sort,
reorder, trace, table update), a two-wavefront batch and a served request on
the bounds-checked library, compared with the oracle; then a permutation
with one entry out of range, which the checked reorder flags and skips."""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import oracle  # noqa: E402
from hitcheck import compare  # noqa: E402
from paper_2506_11273_gb300 import rr  # noqa: E402
from paper_2506_11273_gb300 import workloads as W  # noqa: E402

assert os.path.basename(rr.LIB_PATH) == "librr_checked.so"
rr.lib()
maps = open("/proc/self/maps").read()
assert "librr_checked.so" in maps and "/librr.so" not in maps
print("checked library loaded")

tris = W.scene_box_soup(seed=1)
rays = W.rays_box_soup(tris, n=65536, seed=1)
lo, hi = W.scene_aabb(tris)
bvh = rr.BVH(tris)
table = rr.LengthTable(lo, hi)
params = rr.key_params(rr.RR_KEY_TWO_POINT, 64, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
pipe = rr.Pipeline(bvh, len(rays), params, radix_bits=8)
o, d, p = rr.to_device_rays(rays)
hits = torch.empty(len(rays), 4, device="cuda")
pout = torch.empty_like(p)
pipe.run(o, d, p, hits, pout)
torch.cuda.synchronize()
otab = oracle.LengthTable(oracle.largest_extent(lo, hi))
keys = oracle.compute_keys(oracle.TWO_POINT, 64, rays.o_tmin, rays.d_tmax, lo, hi, tsrc=oracle.T_ADAPTIVE, table=otab)
perm, _ = oracle.stable_sort(keys)
so, sd, sp = oracle.permute(rays.o_tmin, rays.d_tmax, rays.payload, perm)
assert np.array_equal(rr.u32_to_numpy(pout), sp)
oh, oi = oracle.trace_brute(tris, so, sd)
compare(tris, so, sd, hits.cpu().numpy(), oh, oi)
half = len(rays) // 2
batch = rr.Batch([(bvh, None, lo, hi, half), (bvh, None, lo, hi, len(rays) - half)], rr.RR_KEY_AILA)
bh = torch.empty(len(rays), 4, device="cuda")
batch.run(o, d, bh, rr.Batch.config(24, 8, 256))
torch.cuda.synchronize()
uh, ui = oracle.trace_brute(tris, rays.o_tmin, rays.d_tmax)
compare(tris, rays.o_tmin, rays.d_tmax, bh.cpu().numpy(), uh, ui)
batch.close()
srv = rr.Server(budget_bytes=1 << 28, slots=2)
sid = srv.add_scene(bvh, lo, hi)
sh = np.zeros((len(rays), 4), np.float32)
srv.wait(srv.submit(sid, rays.o_tmin, rays.d_tmax, sh))
srv.close()
compare(tris, rays.o_tmin, rays.d_tmax, sh, uh, ui)
flags = rr.rr_device_error()
assert flags == 0, flags
print("clean")
# one permutation entry out of range: the checked reorder flags it and skips it
n = 1000
bad = torch.arange(n, dtype=torch.int32, device="cuda")
bad[17] = n + 5
go = torch.full((n, 4), -7.0, device="cuda")
gd = torch.full((n, 4), -7.0, device="cuda")
rr.rr_permute(o[:n].contiguous(), d[:n].contiguous(), None, bad, go, gd, None)
torch.cuda.synchronize()
assert rr.rr_device_error() == rr.RR_DEVERR_BAD_INDEX
g = go.cpu().numpy()
assert np.all(g[17] == -7.0) and np.array_equal(g[:17], rays.o_tmin[:17]) and np.array_equal(g[18:], rays.o_tmin[18:n])
print("bad index flagged")
