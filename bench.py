"""Benchmark of the per-bounce reordered path on the path-tracer workload.

Workload (1920x1080, 1 spp, 4 bounces): the 1,168,576-triangle terrain scene,
camera rays, then secondary rays scattered off 70% Lambertian / 30% Phong-100
surfaces with Russian roulette after bounce 2.  The wavefronts are built once
(untimed) by tracing them in their natural pixel order.  One timed step is one
pass of the whole hot path over the bounce-3 wavefront:

    Two Point key (adaptive termination estimate, 64 bits)
    -> stable radix sort (8-bit digits, 8 passes) -> gather of the ray SoA
    -> closest-hit trace with the length-table update in the same kernel

`value` is rays / step time (MRays/s, inputs resident in HBM, L2 flushed
between steps).  `unsorted_mrays` traces the same rays in their original
order; `e2e` runs a stream of the same bounce through rr_pipeline_submit_host /
rr_pipeline_wait with page-locked host buffers (two in flight), every step's
transfers and the L2 flushes between steps inside the timed region.  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "end-to-end MRays/s sorted vs unsorted per bounce; sort GB/s vs HBM peak; p99 latency"
UNIT = "MRays/s"
KEY_BITS = 64
RADIX_BITS = 8
# algorithmic bytes per ray (reads + writes of the data a phase must touch)
BYTES_KEY = 32 + 8
BYTES_SORT = 8 + (KEY_BITS // RADIX_BITS) * 2 * (8 + 4) - 4   # 196 for 64-bit keys, 8-bit digits
BYTES_GATHER = 4 + 36 + 36
BYTES_TRACE = 32 + 16
BYTES_ACCUM = 32 + 16
TRACE_SOURCES = ["paper_2506_11273_gb300/csrc/rr_trace.cu", "paper_2506_11273_gb300/csrc/rr_trace.h",
                 "paper_2506_11273_gb300/csrc/rr_common.cuh", "paper_2506_11273_gb300/csrc/rr_bvh.cpp",
                 "paper_2506_11273_gb300/csrc/rr_keymath.cuh", "paper_2506_11273_gb300/csrc/rr_batch.cuh"]
# One ncu capture of the trace kernel on this workload (bounce-3 wavefront, sorted
# rays, `trace_kernel<0, 0, 0, 128>`): DRAM bytes read + written and warp
# instructions per launch, valid only while the trace sources hash to `sources`
# (sha256 of TRACE_SOURCES, first 16 hex digits); otherwise traffic is reported as null.
TRACE_NCU = {"sources": "16c2fbc1e738e3cd", "dram_bytes": 171183616 + 16250624, "warp_instructions": 540485561}
# issue-slot peak: 4 warp instructions per cycle per SM (one per scheduler) x 152 SMs
SMS, ISSUE_PER_SM_CYCLE, MAX_SM_MHZ = 152, 4, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--bounce", type=int, default=3)
    ap.add_argument("--small", action="store_true", help="tiny scene and wavefront (for profiling runs)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other keys, reorder variants, shadow rays and per-bounce sweep (the e2e run stays)")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-execution measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--sweep", action="store_true",
                    help="scale sweep instead of the bench line: 4.67M-triangle scene, 3840x2160 bounce-2 "
                         "wavefront, key bits 16/32/48/64 x radix 4/8, phase split")
    return ap.parse_args()


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mrays(world: int, rays_per_rank_step: int, steps: int, max_total_ms: float) -> float:
    """Weak scaling: every rank traces its own wavefront; the job's throughput is
    all ranks' rays over the slowest rank's time."""
    return world * rays_per_rank_step * steps / (max_total_ms * 1e-3) / 1e6


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def trace_ncu_counts():
    """(DRAM bytes, warp instructions) per trace launch from the recorded ncu
    capture, or (None, None) when the trace kernel's sources have changed since."""
    h = hashlib.sha256()
    try:
        for src in TRACE_SOURCES:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
    except OSError:
        return None, None
    if TRACE_NCU["sources"] != h.hexdigest()[:16]:
        return None, None
    return TRACE_NCU["dram_bytes"], TRACE_NCU["warp_instructions"]


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, window: str = "the timed region"):
        self.dev = device_index
        self.window = window
        self.p = None
        self.out = None
        self.skip = 0
        self.path = "/tmp/rr_clocks_%d_%d.csv" % (os.getpid(), device_index)

    def _lines(self) -> int:
        try:
            return open(self.path).read().count("\n")
        except OSError:
            return 0

    def __enter__(self):
        try:
            self.out = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.p = None
        if self.p is not None:
            # the sampler is live before the window opens; its samples from
            # before the window are left out of the summary
            t_end = time.time() + 3.0
            while self._lines() == 0 and time.time() < t_end and self.p.poll() is None:
                time.sleep(0.02)
            self.skip = self._lines()
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        if self.out is not None:
            self.out.close()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.remove(self.path)
        except OSError:
            rows = []
        inside = rows[self.skip:]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "window": self.window}
        rows = inside or rows[-1:]
        sm = [float(r[1]) for r in rows if len(r) > 8]
        mx = [float(r[2]) for r in rows if len(r) > 8]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) > 8:
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_window": len(inside),
                "window": self.window}


def build_workload(small: bool, seed: int):
    from paper_2506_11273_gb300 import workloads as W
    if small:
        tris = W.scene_terrain(seed=seed, cells_x=128, cells_z=256, n_boxes=1000)
        cam = W.Camera(width=480, height=270)
    else:
        tris = W.scene_terrain(seed=seed)
        cam = W.Camera()
    return tris, cam


# ----------------------------------------------------------------------------- ours

def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2506_11273_gb300 import rr
    from paper_2506_11273_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    t0 = time.time()
    tris, cam = build_workload(args.small, seed=2)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    info = bvh.info()
    table = rr.LengthTable(lo, hi)

    # wavefronts of the path tracer, traced in natural (pixel) order; the
    # adaptive table learns from every traced bounce, as the paper's does
    fronts = []
    rays = W.camera_rays(cam, seed=2 + 1000 * rank)
    for b in range(1, 5):
        fronts.append(rays)
        o, d, _ = rr.to_device_rays(rays, dev)
        h = torch.empty(len(rays), 4, device=dev)
        rr.rr_trace(bvh, o, d, h)
        if b < args.bounce:
            table.accumulate(o, d, h)
        hn = h.cpu().numpy()
        if b < 4:
            rays = W.next_bounce(tris, rays, hn, b, seed=2 + 1000 * rank)
    setup_s = time.time() - t0

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def bounce_buffers(rays):
        n = len(rays)
        o, d, p = rr.to_device_rays(rays, dev)
        bufs = dict(o=o, d=d, p=p, n=n,
                    keys=torch.empty(n, dtype=torch.int64, device=dev),
                    perm=torch.empty(n, dtype=torch.int32, device=dev),
                    ws=rr.sort_workspace(n, KEY_BITS, RADIX_BITS, dev),
                    keys32=torch.empty(n, dtype=torch.int32, device=dev),
                    ws32=rr.sort_workspace(n, 32, RADIX_BITS, dev),
                    so=torch.empty_like(o), sd=torch.empty_like(d), sp=torch.empty_like(p),
                    hits=torch.empty(n, 4, device=dev))
        return bufs

    params_tp = rr.key_params(rr.RR_KEY_TWO_POINT, KEY_BITS, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
    params_aila = rr.key_params(rr.RR_KEY_AILA, KEY_BITS, lo, hi)

    def make_step(B, params, accumulate, bits=KEY_BITS, sort="global", segment=2048, reorder="gather"):
        """One bounce: key -> sort (global onesweep, or local per segment) ->
        reorder (gather the SoA, or trace through the permutation) -> trace.
        sort="fused": keys and global sort in one rr_key_sort call (the sort's
        digit counting done by the key kernel); its time is the key phase and
        the sort phase reads zero."""
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        keys, ws = (B["keys"], B["ws"]) if bits > 32 else (B["keys32"], B["ws32"])
        tbl = table if accumulate else None

        def step():
            ev[0].record(stream)
            if sort == "fused":
                rr.rr_key_sort(B["o"], B["d"], params, keys, B["perm"], RADIX_BITS, ws)
                ev[1].record(stream)
            else:
                rr.rr_compute_keys(B["o"], B["d"], params, keys)
                ev[1].record(stream)
                if sort == "global":
                    rr.rr_sort(keys, None, B["perm"], B["n"], bits, RADIX_BITS, ws)
                else:
                    rr.rr_sort_segments(keys, None, B["perm"], B["n"], bits, segment)
            ev[2].record(stream)
            if reorder == "gather":
                rr.rr_permute(B["o"], B["d"], B["p"], B["perm"], B["so"], B["sd"], B["sp"])
                ev[3].record(stream)
                if accumulate:  # trace and length-table update in one kernel
                    rr.rr_trace_accumulate(bvh, B["so"], B["sd"], B["hits"], table)
                else:
                    rr.rr_trace(bvh, B["so"], B["sd"], B["hits"])
            else:  # indirect access: the trace reads the rays through perm
                ev[3].record(stream)
                rr.rr_trace_ex(bvh, B["o"], B["d"], B["hits"], order=B["perm"], table=tbl)
            ev[4].record(stream)
            ev[5].record(stream)

        def phases():
            return [ev[i].elapsed_time(ev[i + 1]) for i in range(5)]
        return step, phases

    def make_unsorted(B):
        def step():
            rr.rr_trace(bvh, B["o"], B["d"], B["hits"])
        return step

    def timed(step, K, W_, phases=None):
        for _ in range(W_):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ph = []
        total = 0.0
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        for k in range(K):
            flush.zero_()
            starts[k].record(stream)
            step()
            ends[k].record(stream)
            if phases is not None:
                torch.cuda.synchronize()
                ph.append(phases())
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        times = [starts[k].elapsed_time(ends[k]) for k in range(K)]
        total = float(sum(times))
        return total, times, ph

    head = fronts[args.bounce - 1]
    B = bounce_buffers(head)
    n = B["n"]
    step_tp, phases_tp = make_step(B, params_tp, True, sort="fused")
    l0 = rr.rr_kernel_launch_count()
    step_sep, phases_sep = make_step(B, params_tp, True)
    # clocks: nvidia-smi samples every 100 ms, longer than the timed steps, so
    # the window also covers the same step run untimed for 0.4 s right after
    # them, under the same load
    with ClockSampler(local, "the timed steps and 0.4 s of the same step right after them") as clk:
        total_ms, times, ph = timed(step_tp, args.steps, args.warmup, phases_tp)
        launches = (rr.rr_kernel_launch_count() - l0)
        launches_timed = launches * args.steps // (args.steps + args.warmup)
        t_soak = time.time()
        while time.time() - t_soak < 0.4:
            flush.zero_()
            step_tp()
            torch.cuda.synchronize()
    # the same step with keys and sort as two calls: the key and sort phases on
    # their own (for their HBM fractions)
    _, _, ph_sep = timed(step_sep, max(3, args.steps // 2), 3, phases_sep)
    E_scene = float(np.max(hi - lo))

    def capsule_mean(o_, d_, h_):
        """Mean capsule area of the runs of 64 consecutive rays (Section 4.3)."""
        return float(rr.rr_coherence_capsule(o_, d_, h_, E_scene).mean().item())

    coherence = {"two_point_adaptive64": capsule_mean(B["so"], B["sd"], B["hits"])}
    clocks = clk.summary()
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    value = whole_job_mrays(world, n, args.steps, total_ms)
    ph = np.array(ph)
    med_f = [float(x) for x in np.median(ph, axis=0)]
    med_s = [float(x) for x in np.median(np.array(ph_sep), axis=0)]
    phase_ms = {"key_and_sort": med_f[0], "gather": med_f[2], "trace_and_accum": med_f[3],
                "key": med_s[0], "sort": med_s[1]}
    if rr.rr_device_error() != 0:
        raise RuntimeError("device error flag set during the bench")

    extra = {}
    # unsorted trace of the same rays, same conditions
    tot_u, _, _ = timed(make_unsorted(B), args.steps, args.warmup)
    unsorted = n * args.steps / (tot_u * 1e-3) / 1e6
    coherence["unsorted"] = capsule_mean(B["o"], B["d"], B["hits"])
    if not args.no_extra:
        # the origin-direction (Aila) key on the same rays
        step_aila, phases_aila = make_step(B, params_aila, False)
        tot_a, _, ph_a = timed(step_aila, max(3, args.steps // 2), 3, phases_aila)
        aila = n * max(3, args.steps // 2) / (tot_a * 1e-3) / 1e6
        extra["aila_mrays"] = round(aila, 2)
        extra["aila_trace_ms"] = round(float(np.median(np.array(ph_a)[:, 3])), 4)
        coherence["aila64"] = capsule_mean(B["so"], B["sd"], B["hits"])
        # the paper's 32-bit Two Point key (Table 1 uses 32-bit keys) on the same rays
        params_tp32 = rr.key_params(rr.RR_KEY_TWO_POINT, 32, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
        step_32, phases_32 = make_step(B, params_tp32, False, bits=32)
        tot_32, _, ph_32 = timed(step_32, max(3, args.steps // 2), 3, phases_32)
        extra["two_point_32bit_mrays"] = round(n * max(3, args.steps // 2) / (tot_32 * 1e-3) / 1e6, 2)
        extra["two_point_32bit_phases_ms"] = {k: round(float(v), 4) for k, v in
                                              zip(["key", "sort", "gather", "trace"], np.median(np.array(ph_32), axis=0)[:4])}

        # Two Point Real (the paper's bound): the estimate is each ray's true hit
        # distance, taken from the unsorted trace above
        tg = (B["hits"][:, 0] * torch.linalg.norm(B["d"][:, :3], dim=1)).contiguous()
        params_real = rr.key_params(rr.RR_KEY_TWO_POINT, KEY_BITS, lo, hi, t_source=rr.RR_T_GIVEN, t_given=tg)
        step_real, phases_real = make_step(B, params_real, False)
        tot_r, _, ph_r = timed(step_real, max(3, args.steps // 2), 3, phases_real)
        extra["two_point_real_mrays"] = round(n * max(3, args.steps // 2) / (tot_r * 1e-3) / 1e6, 2)
        extra["two_point_real_trace_ms"] = round(float(np.median(np.array(ph_r)[:, 3])), 4)
        coherence["two_point_real64"] = capsule_mean(B["so"], B["sd"], B["hits"])
        extra["shadow_rays"] = bench_shadow(args, B, bvh, tris, lo, hi, flush, timed, stream)

        # every key family of Section 3.1 at 32 bits (the paper's Table 1 uses
        # 32-bit keys): trace speedup over the unsorted rays and the capsule
        # coherence of the sorted order
        t_uns_ms = tot_u / args.steps
        fam = {}
        kf = max(3, args.steps // 2)
        for name, layout, ts, kw in [
                ("origin", rr.RR_KEY_ORIGIN, rr.RR_T_FIXED, {}), ("reis", rr.RR_KEY_REIS, rr.RR_T_FIXED, {}),
                ("costa", rr.RR_KEY_COSTA, rr.RR_T_FIXED, {}), ("aila", rr.RR_KEY_AILA, rr.RR_T_FIXED, {}),
                ("aila_compact", rr.RR_KEY_AILA_COMPACT, rr.RR_T_FIXED, {}),
                ("octahedron", rr.RR_KEY_OCTAHEDRON, rr.RR_T_FIXED, {}),
                ("two_point_fixed", rr.RR_KEY_TWO_POINT, rr.RR_T_FIXED, {}),
                ("two_point_adaptive", rr.RR_KEY_TWO_POINT, rr.RR_T_ADAPTIVE, {"table": table}),
                ("two_point_real", rr.RR_KEY_TWO_POINT, rr.RR_T_GIVEN, {"t_given": tg})]:
            prm = rr.key_params(layout, 32, lo, hi, t_source=ts, **kw)
            st_f, pf_f = make_step(B, prm, False, bits=32)
            _, _, ph_f = timed(st_f, kf, 3, pf_f)
            tr = float(np.median(np.array(ph_f)[:, 3]))
            fam[name] = {"trace_ms": round(tr, 4), "trace_speedup": round(t_uns_ms / tr, 3),
                         "capsule_rel": round(capsule_mean(B["so"], B["sd"], B["hits"]) / coherence["unsorted"], 3)}
        extra["key_families_32bit"] = fam

        # cheaper reorderings of the same bounce (local sort, indirect access)
        variants = {}
        kv = max(3, args.steps // 2)
        params_costa32 = rr.key_params(rr.RR_KEY_COSTA, 32, lo, hi)
        params_costa24 = rr.key_params(rr.RR_KEY_COSTA, 24, lo, hi)
        params_costa16 = rr.key_params(rr.RR_KEY_COSTA, 16, lo, hi)
        for name, kw in [("global64_indirect", dict(params=params_tp, accumulate=True, reorder="indirect")),
                         ("costa24_indirect", dict(params=params_costa24, accumulate=False, bits=24,
                                                   reorder="indirect")),
                         ("costa16_indirect", dict(params=params_costa16, accumulate=False, bits=16,
                                                   reorder="indirect")),
                         ("costa32_gather", dict(params=params_costa32, accumulate=False, bits=32)),
                         ("costa32_indirect", dict(params=params_costa32, accumulate=False, bits=32,
                                                   reorder="indirect")),
                         ("global32_indirect", dict(params=params_tp32, accumulate=True, bits=32, reorder="indirect")),
                         ("local1024_indirect", dict(params=params_tp, accumulate=True, sort="segment", segment=1024,
                                                     reorder="indirect")),
                         ("local2048_indirect", dict(params=params_tp, accumulate=True, sort="segment", segment=2048,
                                                     reorder="indirect")),
                         ("local4096_indirect", dict(params=params_tp, accumulate=True, sort="segment", segment=4096,
                                                     reorder="indirect")),
                         ("local4096_gather", dict(params=params_tp, accumulate=True, sort="segment", segment=4096))]:
            st_v, pf_v = make_step(B, **kw)
            tot_v, _, ph_v = timed(st_v, kv, 3, pf_v)
            med = np.median(np.array(ph_v), axis=0)
            variants[name] = {"mrays": round(n * kv / (tot_v * 1e-3) / 1e6, 2),
                              "phases_ms": {k: round(float(v), 4) for k, v in
                                            zip(["key", "sort", "gather", "trace"], med[:4])}}
        extra["reorder_variants"] = variants
        best = max(variants, key=lambda k: variants[k]["mrays"])
        extra["best_reorder"] = {"variant": best, "mrays": variants[best]["mrays"],
                                 "vs_unsorted": round(variants[best]["mrays"] / unsorted, 3)}
        if rr.rr_device_error() != 0:
            raise RuntimeError("device error flag set during the reorder variants")

    if not args.no_extra:
        per_bounce = []
        for b, fr in enumerate(fronts, start=1):
            Bb = bounce_buffers(fr)
            st, pf = make_step(Bb, params_tp, False, sort="fused")
            k = 5
            tot_s, _, phb = timed(st, k, 3, pf)
            tot_uu, _, _ = timed(make_unsorted(Bb), k, 3)
            phb = np.median(np.array(phb), axis=0)
            per_bounce.append({"bounce": b, "rays": Bb["n"],
                               "sorted_e2e_mrays": round(Bb["n"] * k / (tot_s * 1e-3) / 1e6, 1),
                               "unsorted_trace_mrays": round(Bb["n"] * k / (tot_uu * 1e-3) / 1e6, 1),
                               "sorted_trace_mrays": round(Bb["n"] / (phb[3] * 1e-3) / 1e6, 1)})
            del Bb
        extra["per_bounce"] = per_bounce

    # end to end through the C ABI with page-locked host buffers: a stream of
    # bounces, two submissions in flight (the upload of step k+1 overlaps the
    # kernels of step k; every step's transfers are inside the timed region),
    # the L2 flush between steps enqueued between the submissions and counted
    pipe = rr.Pipeline(bvh, n, params_tp, RADIX_BITS)
    ho = torch.from_numpy(head.o_tmin).pin_memory()
    hd = torch.from_numpy(head.d_tmax).pin_memory()
    hp = torch.from_numpy(head.payload.view(np.int32)).pin_memory()
    outs = [(torch.empty(n, 4, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.int32).pin_memory())
            for _ in range(2)]
    for j in range(3):
        pipe.run_host(ho, hd, hp, *outs[j % 2])
    torch.cuda.synchronize()
    ke = max(3, args.steps)
    t1 = time.perf_counter()
    pending = []
    for k in range(ke):
        flush.zero_()
        pending.append(pipe.submit_host(ho, hd, hp, *outs[k % 2]))
        if len(pending) > 1:
            pipe.wait(pending.pop(0))
    pipe.wait(pending.pop(0))
    torch.cuda.synchronize()
    e2e = world * n * ke / (time.perf_counter() - t1) / 1e6
    pipe.close()

    hbm, peak_kind = peaks()
    # the dominant kernel (the trace, ~75% of a sorted step) alone, launched on
    # the sorted rays as in the step (L2 flushed before each launch), against
    # its algorithmic HBM floor: 48 B per ray (ray in, hit out) over the live
    # CUDA-event duration of the launch
    trace_hits = torch.empty(n, 4, device=dev)
    tot_tr, _, _ = timed(lambda: rr.rr_trace(bvh, B["so"], B["sd"], trace_hits), args.steps, args.warmup)
    trace_kernel_ms = tot_tr / args.steps
    del trace_hits
    trace_ach = BYTES_TRACE * n / (trace_kernel_ms * 1e-3) / 1e9
    traffic, inst = (None, None) if args.small else trace_ncu_counts()
    sm_mhz = clocks.get("sm_mhz") or MAX_SM_MHZ
    roofline = {"bound": "hbm", "kernel": "trace_kernel (closest hit, sorted rays)",
                "achieved": round(trace_ach, 1), "peak": hbm, "unit": "GB/s", "frac": round(trace_ach / hbm, 4),
                "traffic": traffic, "peak_kind": peak_kind + " (MEASURED_PEAKS hbm_gbs, copy bandwidth)",
                "algorithmic_bytes_per_ray": BYTES_TRACE, "units_per_launch": n,
                "launch_ms": round(trace_kernel_ms, 4)}
    if traffic is not None:
        roofline["traffic_over_algorithmic"] = round(traffic / (BYTES_TRACE * n), 2)
    if inst is not None:
        # what actually bounds the kernel: instruction issue (ncu warp instructions
        # per launch over the live launch time, against 4 issue slots x 152 SMs
        # x the sampled SM clock)
        issue_peak = SMS * ISSUE_PER_SM_CYCLE * sm_mhz * 1e6 / 1e9
        ach = inst / (trace_kernel_ms * 1e-3) / 1e9
        roofline["issue"] = {"achieved": round(ach, 1), "peak": round(issue_peak, 1),
                             "unit": "G warp-instructions/s", "frac": round(ach / issue_peak, 4),
                             "warp_instructions_per_launch": inst}
    sort_ach = BYTES_SORT * n / (phase_ms["sort"] * 1e-3) / 1e9
    gather_ach = BYTES_GATHER * n / (phase_ms["gather"] * 1e-3) / 1e9
    key_ach = BYTES_KEY * n / (phase_ms["key"] * 1e-3) / 1e9
    # fused: the key kernel's reads and writes plus the digit passes (the
    # counting pass's read of the keys is gone)
    bytes_key_sort = BYTES_KEY + BYTES_SORT - 8
    key_sort_ach = bytes_key_sort * n / (phase_ms["key_and_sort"] * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
        "data": "synthetic",
        "config": {"workload": ("path tracer 1920x1080 1spp, bounce-%d wavefront, %d-triangle terrain; "
                                "Two Point key (adaptive estimate) %d bits, radix %d" %
                                (args.bounce, info.n_tris, KEY_BITS, RADIX_BITS)) if not args.small
                   else "small profiling case",
                   "rays_per_step": n, "triangles": int(info.n_tris), "bounce": args.bounce,
                   "key": "two_point_adaptive", "key_bits": KEY_BITS, "radix_bits": RADIX_BITS,
                   "key_and_sort": "rr_key_sort (the sort's digit counting in the key kernel)",
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas" if world > 1 else "1 gpu"},
        "unsorted_mrays": round(unsorted, 2),
        "speedup_vs_unsorted": round(value / unsorted, 3),
        "phases_ms": {k: round(v, 4) for k, v in phase_ms.items()},
        "roofline": roofline,
        "phase_roofline": {
            "key": {"gbs": round(key_ach, 1), "frac": round(key_ach / hbm, 3), "bytes_per_ray": BYTES_KEY},
            "sort": {"gbs": round(sort_ach, 1), "frac": round(sort_ach / hbm, 3), "bytes_per_ray": BYTES_SORT,
                     "mkeys_s": round(n / (phase_ms["sort"] * 1e-3) / 1e6, 1)},
            "gather": {"gbs": round(gather_ach, 1), "frac": round(gather_ach / hbm, 3), "bytes_per_ray": BYTES_GATHER},
            "key_and_sort": {"gbs": round(key_sort_ach, 1), "frac": round(key_sort_ach / hbm, 3),
                             "bytes_per_ray": bytes_key_sort},
        },
        "e2e": {"value": round(e2e, 2), "unit": UNIT, "h2d_bytes_per_step": 36 * n,
                "d2h_bytes_per_step": 20 * n,
                "mode": "rr_pipeline_submit_host, two submissions in flight; L2 flush between steps counted"},
        "gpu_launches": int(launches_timed),
        "clocks": clocks,
        "bvh": {"nodes": int(info.n_nodes), "depth": int(info.depth), "build_s": round(info.build_seconds, 2),
                "bytes": int(info.node_bytes + info.tri_bytes)},
        "setup_s": round(setup_s, 1),
    }
    out.update(extra)
    out["coherence_capsule_m64"] = {k: {"mean_area": round(v, 4), "relative_to_unsorted":
                                        round(v / coherence["unsorted"], 3)} for k, v in coherence.items()}
    if not args.no_batched:
        out["batched"] = bench_batched(args, dev, flush)
    if not args.no_serving:
        out["serving"] = bench_serving(args, dev)
        mid = out["serving"]["loads"][-1]
        out["p99_latency_ms"] = mid["p99_ms"]
        out["p99_at_load"] = "%.0f%% of measured capacity (%.1f requests/s)" % (100 * mid["load_frac"],
                                                                                mid["offered_rps"])
    if rank == 0:
        out["cpu_baseline"] = cpu_baseline(tris, lo, hi, sample=20000 if args.small else 400000)
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- shadow rays

def bench_shadow(args, B, bvh, tris, lo, hi, flush, timed, stream):
    """Next-event shadow rays from the hit points of the bounce-3 wavefront (in
    wavefront order) to a square light of side 0.05 E above the scene (the
    paper's evaluation setup, Section 4), traced with the any-hit kernel:
    unsorted versus sorted by the Octahedron, Aila and Two Point keys (32 bits;
    Two Point with the known distance to the light as its estimate)."""
    import torch

    from paper_2506_11273_gb300 import rr
    from paper_2506_11273_gb300 import workloads as W

    h = B["hits"].cpu().numpy()  # unsorted hits, wavefront order
    o = B["o"].cpu().numpy()
    d = B["d"].cpu().numpy()
    hit = np.ascontiguousarray(h[:, 3]).view(np.uint32) != rr.MISS
    pts = o[hit, :3].astype(np.float64) + h[hit, 0:1].astype(np.float64) * d[hit, :3].astype(np.float64)
    E = float(np.max(hi - lo))
    center = ((lo[0] + hi[0]) / 2, hi[1] + 0.05 * E, (lo[2] + hi[2]) / 2)
    sr = W.shadow_rays_to_light(pts, center, 0.05 * E, seed=5)
    n = len(sr)
    so, sd, _ = rr.to_device_rays(sr, B["o"].device)
    hits = torch.empty(n, 4, device=so.device)
    perm = torch.empty(n, dtype=torch.int32, device=so.device)
    keys = torch.empty(n, dtype=torch.int32, device=so.device)
    go, gd = torch.empty_like(so), torch.empty_like(sd)
    ws = rr.sort_workspace(n, 32, RADIX_BITS, so.device)
    t_light = torch.linalg.norm(sd[:, :3], dim=1).contiguous()  # p = o + d^ |d| is the light point

    def unsorted():
        rr.rr_trace_ex(bvh, so, sd, hits, flags=rr.RR_TRACE_ANY_HIT)

    def variant(params):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

        def step():
            ev[0].record(stream)
            rr.rr_compute_keys(so, sd, params, keys)
            ev[1].record(stream)
            rr.rr_sort(keys, None, perm, n, 32, RADIX_BITS, ws)
            ev[2].record(stream)
            rr.rr_permute(so, sd, None, perm, go, gd, None)
            ev[3].record(stream)
            rr.rr_trace_ex(bvh, go, gd, hits, flags=rr.RR_TRACE_ANY_HIT)
            ev[4].record(stream)

        return step, lambda: [ev[i].elapsed_time(ev[i + 1]) for i in range(4)]

    K = max(3, args.steps // 2)
    tot_u, _, _ = timed(unsorted, K, 3)
    occluded = float(np.mean(np.ascontiguousarray(hits.cpu().numpy()[:, 3]).view(np.uint32) != rr.MISS))
    out = {"rays": n, "occluded_fraction": round(occluded, 3), "unsorted_mrays": round(n * K / (tot_u * 1e-3) / 1e6, 1)}
    for name, params in [("octahedron32", rr.key_params(rr.RR_KEY_OCTAHEDRON, 32, lo, hi)),
                         ("aila32", rr.key_params(rr.RR_KEY_AILA, 32, lo, hi)),
                         ("two_point32_light", rr.key_params(rr.RR_KEY_TWO_POINT, 32, lo, hi,
                                                             t_source=rr.RR_T_GIVEN, t_given=t_light))]:
        st, pf = variant(params)
        tot, _, ph = timed(st, K, 3, pf)
        med = np.median(np.array(ph), axis=0)
        out[name] = {"sorted_e2e_mrays": round(n * K / (tot * 1e-3) / 1e6, 1),
                     "trace_mrays": round(n / (float(med[3]) * 1e-3) / 1e6, 1),
                     "phases_ms": {k: round(float(v), 4) for k, v in zip(["key", "sort", "gather", "trace"], med)}}
    if rr.rr_device_error() != 0:
        raise RuntimeError("device error flag set during the shadow-ray measurement")
    return out


# ----------------------------------------------------------------------------- scale sweep

def run_sweep(args):
    """Key bits 16/32/48/64 x radix width 4/8 on the 4,674,304-triangle scene and
    its 3840x2160 bounce-2 wavefront (Two Point key, adaptive estimate): the
    phase split key / sort / gather / trace (+ table update) and MRays/s."""
    import torch

    from paper_2506_11273_gb300 import rr
    from paper_2506_11273_gb300 import workloads as W

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    if args.small:
        tris = W.scene_terrain(seed=3, cells_x=128, cells_z=256, n_boxes=1000)
        cam = W.Camera(width=960, height=540)
    else:
        tris = W.scene_terrain(seed=3, cells_x=1024, cells_z=2048, n_boxes=40000)
        cam = W.Camera(width=3840, height=2160)
    lo, hi = W.scene_aabb(tris)
    bvh = rr.BVH(tris)
    table = rr.LengthTable(lo, hi)
    rays = W.camera_rays(cam, seed=3)
    o, d, _ = rr.to_device_rays(rays, dev)
    h = torch.empty(len(rays), 4, device=dev)
    rr.rr_trace(bvh, o, d, h)
    table.accumulate(o, d, h)
    rays = W.next_bounce(tris, rays, h.cpu().numpy(), 1, seed=3)
    del o, d, h
    n = len(rays)
    o, d, p = rr.to_device_rays(rays, dev)
    so, sd, sp = torch.empty_like(o), torch.empty_like(d), torch.empty_like(p)
    hits = torch.empty(n, 4, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    setup_s = time.time() - t0

    def timed(fn, K, W_=3):
        evs = None
        for _ in range(W_):
            flush.zero_()
            fn(None)
        torch.cuda.synchronize()
        rows = []
        for _ in range(K):
            flush.zero_()
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            fn(evs)
            torch.cuda.synchronize()
            rows.append([evs[i].elapsed_time(evs[i + 1]) for i in range(4)])
        return np.median(np.array(rows), axis=0)

    def unsorted(evs):
        if evs:
            for e in evs[:4]:
                e.record(stream)
        rr.rr_trace(bvh, o, d, hits)
        if evs:
            evs[4].record(stream)

    t_uns = float(timed(unsorted, 5)[3])
    rows = []
    for bits in (16, 32, 48, 64):
        keys = torch.empty(n, dtype=rr.key_dtype(bits), device=dev)
        params = rr.key_params(rr.RR_KEY_TWO_POINT, bits, lo, hi, t_source=rr.RR_T_ADAPTIVE, table=table)
        for radix in (4, 8):
            ws = rr.sort_workspace(n, bits, radix, dev)

            def step(evs):
                if evs:
                    evs[0].record(stream)
                rr.rr_compute_keys(o, d, params, keys)
                if evs:
                    evs[1].record(stream)
                rr.rr_sort(keys, None, perm, n, bits, radix, ws)
                if evs:
                    evs[2].record(stream)
                rr.rr_permute(o, d, p, perm, so, sd, sp)
                if evs:
                    evs[3].record(stream)
                rr.rr_trace_accumulate(bvh, so, sd, hits, table)
                if evs:
                    evs[4].record(stream)

            ph = timed(step, 5)
            kb = 8 if bits > 32 else 4
            passes = -(-bits // radix)
            sort_bytes = n * (kb + passes * 2 * (kb + 4) - 4)
            hbm, _ = peaks()
            rows.append({"key_bits": bits, "radix_bits": radix,
                         "key_ms": round(float(ph[0]), 4), "sort_ms": round(float(ph[1]), 4),
                         "gather_ms": round(float(ph[2]), 4), "trace_accum_ms": round(float(ph[3]), 4),
                         "sorted_e2e_mrays": round(n / (float(ph.sum()) * 1e-3) / 1e6, 1),
                         "sort_gbs": round(sort_bytes / (float(ph[1]) * 1e-3) / 1e9, 1),
                         "sort_frac_hbm": round(sort_bytes / (float(ph[1]) * 1e-3) / 1e9 / hbm, 3)})
            del ws
        del keys
    # the direction-first Costa key (32 bits with the gather and with indirect
    # access; 24 bits with indirect access)
    keys32 = torch.empty(n, dtype=torch.int32, device=dev)
    ws32 = rr.sort_workspace(n, 32, 8, dev)
    extra_rows = {}
    for cbits, reorder in ((32, "gather"), (32, "indirect"), (24, "indirect")):
        params_c = rr.key_params(rr.RR_KEY_COSTA, cbits, lo, hi)

        def step_c(evs):
            if evs:
                evs[0].record(stream)
            rr.rr_compute_keys(o, d, params_c, keys32)
            if evs:
                evs[1].record(stream)
            rr.rr_sort(keys32, None, perm, n, cbits, 8, ws32)
            if evs:
                evs[2].record(stream)
            if reorder == "gather":
                rr.rr_permute(o, d, p, perm, so, sd, sp)
                if evs:
                    evs[3].record(stream)
                rr.rr_trace(bvh, so, sd, hits)
            else:
                if evs:
                    evs[3].record(stream)
                rr.rr_trace_ex(bvh, o, d, hits, order=perm)
            if evs:
                evs[4].record(stream)
        ph = timed(step_c, 5)
        extra_rows["costa%d_%s" % (cbits, reorder)] = {
            "key_ms": round(float(ph[0]), 4), "sort_ms": round(float(ph[1]), 4), "gather_ms": round(float(ph[2]), 4),
            "trace_ms": round(float(ph[3]), 4), "sorted_e2e_mrays": round(n / (float(ph.sum()) * 1e-3) / 1e6, 1)}
    if rr.rr_device_error() != 0:
        raise RuntimeError("device error flag set during the sweep")
    out = {"metric": METRIC, "sweep": rows, "costa": extra_rows, "unit": UNIT,
           "config": {"workload": "scale sweep: %d-triangle terrain, %dx%d bounce-2 wavefront (%d rays); Two Point "
                                  "key (adaptive estimate)" % (tris.shape[0], cam.width, cam.height, n),
                      "l2": "flushed between steps (256 MB write)"},
           "unsorted_trace_ms": round(t_uns, 4), "unsorted_mrays": round(n / (t_uns * 1e-3) / 1e6, 1),
           "setup_s": round(setup_s, 1)}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------- batched

# 4 resident scenes of ~50k, 250k, 1M and 2M triangles built like the path-tracer
# scene: (cells_x, cells_z, boxes) with 90% heightfield and 10% box triangles
BATCH_SCENES = [(112, 200, 417), (237, 475, 2083), (474, 949, 8333), (671, 1341, 16667)]
BATCH_WAVEFRONTS = 32


def bench_batched(args, dev, flush):
    """32 wavefronts of log-uniform 10k-2M rays over 4 resident scenes: the
    autotuned batch as one CUDA-graph launch versus the per-wavefront launch
    loop (same configuration), and the unsorted per-wavefront trace."""
    import torch

    from paper_2506_11273_gb300 import rr
    from paper_2506_11273_gb300 import workloads as W

    rng = np.random.default_rng(4)
    scale = 0.05 if args.small else 1.0
    sizes = np.exp(rng.uniform(np.log(1e4 * scale), np.log(2e6 * scale), BATCH_WAVEFRONTS)).astype(np.int64)
    which = rng.integers(0, len(BATCH_SCENES), BATCH_WAVEFRONTS)
    scenes, bvhs, boxes = [], [], []
    for k, (cx, cz, nb) in enumerate(BATCH_SCENES):
        if args.small:
            cx, cz, nb = max(8, cx // 8), max(16, cz // 8), max(10, nb // 64)
        t = W.scene_terrain(seed=40 + k, cells_x=cx, cells_z=cz, n_boxes=nb)
        scenes.append(t)
        bvhs.append(rr.BVH(t))
        boxes.append(W.scene_aabb(t))
    o_parts, d_parts, fronts = [], [], []
    for k in range(BATCH_WAVEFRONTS):
        s = int(which[k])
        r = W.surface_rays(scenes[s], int(sizes[k]), seed=500 + k)
        o_parts.append(r.o_tmin)
        d_parts.append(r.d_tmax)
        fronts.append((bvhs[s], None, boxes[s][0], boxes[s][1], int(sizes[k])))
    o = torch.from_numpy(np.concatenate(o_parts)).to(dev)
    d = torch.from_numpy(np.concatenate(d_parts)).to(dev)
    del o_parts, d_parts
    batch = rr.Batch(fronts, rr.RR_KEY_TWO_POINT, rr.RR_T_FIXED)
    n = batch.n
    hits = torch.empty(n, 4, device=dev)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    t0 = time.time()
    tuned, tuned_ms = batch.tune(o, d, hits)
    # the reordered batch: the tuner's choice, or the best sorted candidate
    # when the tuner found that not reordering was faster
    cfg = tuned if tuned.key_bits else rr.Batch.config(24, 8, tuned.trace_block)
    layout_names = {-1: "two_point (the batch's own)", rr.RR_KEY_COSTA: "costa",
                    rr.RR_KEY_AILA_COMPACT: "aila_compact"}
    tune_s = time.time() - t0
    stream = torch.cuda.current_stream()

    def timed(fn, K):
        for _ in range(3):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(K):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / K

    K = 5
    ms_graph = timed(lambda: batch.run(o, d, hits, cfg, perm), K)
    l0 = rr.rr_kernel_launch_count()
    ms_loop = timed(lambda: batch.run_loop(o, d, hits, cfg, perm), K)
    loop_launches = (rr.rr_kernel_launch_count() - l0) // (K + 3)
    offs = batch.offsets

    def unsorted():
        for k in range(BATCH_WAVEFRONTS):
            a, b_ = offs[k], offs[k + 1]
            rr.rr_trace(fronts[k][0], o[a:b_], d[a:b_], hits[a:b_])
    ms_uns = timed(unsorted, K)
    cfg0 = rr.Batch.config(0, 8, cfg.trace_block, cfg.layout)
    ms_graph0 = timed(lambda: batch.run(o, d, hits, cfg0), K)
    if rr.rr_device_error() != 0:
        raise RuntimeError("device error flag set during the batched measurement")
    out = {"workload": "%d wavefronts of log-uniform %d-%d rays over %d scenes of %s triangles; Two Point "
                       "key (fixed estimate)" % (BATCH_WAVEFRONTS, int(1e4 * scale), int(2e6 * scale),
                                                 len(scenes), "/".join(str(t.shape[0]) for t in scenes)),
           "rays": int(n), "autotuned": {"key_bits": tuned.key_bits, "radix_bits": tuned.radix_bits,
                                          "trace_block": tuned.trace_block,
                                          "layout": layout_names.get(tuned.layout, tuned.layout),
                                          "tuned_ms": round(tuned_ms, 3), "tune_s": round(tune_s, 2)},
           "sorted_config": {"key_bits": cfg.key_bits, "radix_bits": cfg.radix_bits,
                             "trace_block": cfg.trace_block, "layout": layout_names.get(cfg.layout, cfg.layout)},
           "graph_ms": round(ms_graph, 3), "graph_mrays": round(n / (ms_graph * 1e-3) / 1e6, 1),
           "graph_kernels": 3 + -(-(cfg.key_bits + batch.info()["seg_bits"]) // cfg.radix_bits),
           "loop_ms": round(ms_loop, 3), "loop_mrays": round(n / (ms_loop * 1e-3) / 1e6, 1),
           "loop_launches": int(loop_launches),
           "unsorted_graph_ms": round(ms_graph0, 3), "unsorted_graph_mrays": round(n / (ms_graph0 * 1e-3) / 1e6, 1),
           "unsorted_loop_ms": round(ms_uns, 3), "unsorted_loop_mrays": round(n / (ms_uns * 1e-3) / 1e6, 1)}
    batch.close()
    return out


# ----------------------------------------------------------------------------- serving

# 8 resident scenes of 50k..4M triangles built like the path-tracer scene
SERVE_SCENES = [(112, 200, 417), (158, 316, 833), (237, 475, 2083), (335, 670, 4167), (474, 949, 8333),
                (671, 1341, 16667), (822, 1643, 25000), (949, 1897, 33333)]
SERVE_BUDGET = 120 << 30
SERVE_POOL = 1 << 18    # distinct rays generated per scene and kind (requests tile them)
SERVE_MAX_REQ = 4 << 20


def bench_serving(args, dev, slots: int = 4, max_batch_rays: int = 1 << 23, fractions=(0.25, 0.5, 0.75, 0.9),
                  reserve: int = 8 << 30):
    """Poisson arrivals of requests of log-uniform 4k-4M rays (60% diffuse, 40%
    glossy) over 8 resident scenes, served with continuous batching under a
    120 GB budget; p50/p99 latency and throughput at several offered loads.
    Groups are capped at 8M rays (smaller groups finish sooner, so requests that
    share one wait less) and 8 GB of the memory pool is taken up front."""
    import threading

    import torch

    from paper_2506_11273_gb300 import rr
    from paper_2506_11273_gb300 import workloads as W

    small = args.small
    scale = 0.05 if small else 1.0
    lo_n, hi_n = int(4096 * scale) + 1, int(SERVE_MAX_REQ * scale)
    pool_n = max(1024, int(SERVE_POOL * scale))
    srv = rr.Server(budget_bytes=SERVE_BUDGET, slots=slots, max_batch_rays=max(max_batch_rays, hi_n), key_bits=24,
                    radix_bits=8, trace_block=128, reserve_bytes=reserve)
    scenes = []
    pools = {}
    t0 = time.time()
    for k, (cx, cz, nb) in enumerate(SERVE_SCENES):
        if small:
            cx, cz, nb = max(8, cx // 8), max(16, cz // 8), max(10, nb // 64)
        tris = W.scene_terrain(seed=60 + k, cells_x=cx, cells_z=cz, n_boxes=nb)
        bvh = rr.BVH(tris)
        lo, hi = W.scene_aabb(tris)
        sid = srv.add_scene(bvh, lo, hi)
        scenes.append((bvh, tris.shape[0]))
        for kind in ("diffuse", "glossy"):
            r = W.request_rays(tris, pool_n, kind, seed=700 + 2 * k + (kind == "glossy"))
            reps = -(-hi_n // pool_n)
            o = torch.from_numpy(np.tile(r.o_tmin, (reps, 1))).pin_memory()
            d = torch.from_numpy(np.tile(r.d_tmax, (reps, 1))).pin_memory()
            pools[(sid, kind)] = (o, d)
    setup_s = time.time() - t0
    hits_sink = torch.empty(hi_n, 4).pin_memory()  # results are written here and not read

    def link_gbs():
        # host-link copy rates of the request pools and the result buffer
        o = pools[(0, "diffuse")][0]
        dst = torch.empty(o.shape, dtype=o.dtype, device=dev)
        hs = torch.empty(hits_sink.shape, dtype=hits_sink.dtype, device=dev)
        rates = []
        for src, dd, h2d in ((o, dst, True), (hits_sink, hs, False)):
            best = 1e9
            for _ in range(3):
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                (dd.copy_(src, non_blocking=True) if h2d else src.copy_(dd, non_blocking=True))
                torch.cuda.synchronize()
                best = min(best, time.perf_counter() - t1)
            rates.append(round(src.numel() * src.element_size() / best / 1e9, 1))
        del dst, hs
        return rates
    link_before = link_gbs()

    def run_load(rate_rps, duration_s, seed):
        rng = np.random.default_rng(seed)
        n_req = max(8, int(rate_rps * duration_s))
        gaps = rng.exponential(1.0 / rate_rps, n_req)
        sizes = np.exp(rng.uniform(np.log(lo_n), np.log(hi_n), n_req)).astype(np.int64)
        which = rng.integers(0, len(scenes), n_req)
        kinds = np.where(rng.random(n_req) < 0.6, "diffuse", "glossy")
        tickets = []
        start = time.perf_counter()
        t_next = start
        for k in range(n_req):
            t_next += gaps[k]
            while True:
                dt = t_next - time.perf_counter()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.0005))
            o, d = pools[(int(which[k]), str(kinds[k]))]
            tickets.append((srv.submit(int(which[k]), o, d, hits_sink, n=int(sizes[k])), int(sizes[k])))
        lat, queued, service, rays, first, last = [], [], [], 0, None, None
        parts = {"enqueue": [], "device": [], "copy_in": [], "kernels": [], "copy_out": [], "device_start_and_host_fn": []}
        for t, n in tickets:
            tm = srv.wait(t)
            lat.append((tm["done_ns"] - tm["submit_ns"]) * 1e-6)
            queued.append((tm["start_ns"] - tm["submit_ns"]) * 1e-6)
            service.append((tm["done_ns"] - tm["start_ns"]) * 1e-6)
            parts["enqueue"].append((tm["enqueued_ns"] - tm["start_ns"]) * 1e-6)
            parts["device"].append(tm["device_ms"])
            parts["copy_in"].append(tm["copy_in_ms"])
            parts["kernels"].append(tm["kernels_ms"])
            parts["copy_out"].append(tm["copy_out_ms"])
            parts["device_start_and_host_fn"].append((tm["done_ns"] - tm["enqueued_ns"]) * 1e-6 - tm["device_ms"])
            rays += n
            first = tm["submit_ns"] if first is None else min(first, tm["submit_ns"])
            last = tm["done_ns"] if last is None else max(last, tm["done_ns"])
        span = (last - first) * 1e-9
        lat = np.array(lat)
        return {"offered_rps": round(rate_rps, 1), "offered_mrays": round(rate_rps * float(np.mean(sizes)) / 1e6, 1),
                "requests": n_req, "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "mean_ms": round(float(lat.mean()), 3),
                "queued_p50_p99_ms": [round(float(np.percentile(queued, q)), 3) for q in (50, 99)],
                "in_batch_p50_p99_ms": [round(float(np.percentile(service, q)), 3) for q in (50, 99)],
                "in_batch_split_p50_p99_ms": {k: [round(float(np.percentile(v, q)), 3) for q in (50, 99)]
                                              for k, v in parts.items()},
                "throughput_mrays": round(rays / span / 1e6, 1)}

    # capacity: bursts of 256 requests submitted at once (the better of two),
    # after one burst that warms the memory pool and the kernels
    mean_n = (hi_n - lo_n) / np.log(hi_n / lo_n)
    run_load(1e6, 64 / 1e6, seed=2)
    cap_mrays = max(run_load(1e6, 256 / 1e6, seed=s)["throughput_mrays"] for s in (1, 3))
    cap_rps = cap_mrays * 1e6 / mean_n
    loads = []
    with ClockSampler(dev.index or 0) as clk:
        for frac in fractions:
            loads.append(dict(run_load(frac * cap_rps, 1.5 if not small else 0.5, seed=int(frac * 100)),
                              load_frac=frac))
    st = srv.stats()
    srv.close()
    return {"workload": "Poisson arrivals of log-uniform %d-%d-ray requests (60%% diffuse, 40%% glossy) over 8 "
                        "scenes of %s triangles; budget %d GB, %d stream slots, groups of at most %d rays, "
                        "Two Point key 24 bits" % (lo_n, hi_n, "/".join(str(n) for _, n in scenes),
                                                   SERVE_BUDGET >> 30, slots, max(max_batch_rays, hi_n)),
            "capacity_mrays": cap_mrays, "loads": loads, "setup_s": round(setup_s, 1),
            "batches": st["batches"], "max_batch_requests": st["max_batch_requests"],
            "engine_slowdowns": st["engine_slowdowns"], "kernel_copy_groups": st["kernel_copy_groups"],
            "clocks": clk.summary(),
            "pool_h2d_result_d2h_gbs": link_before,
            "peak_reserved_gb": round(st["peak_reserved_bytes"] / 2**30, 2)}


# ----------------------------------------------------------------------------- oracle

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def stable_merge(a, b):
    """Stable merge of two sorted runs (keys, indices) where every index of `a`
    precedes every index of `b`: an element's output position is its position
    in its own run plus the number of elements of the other run that go before
    it (equal keys of `a` go first)."""
    ka, pa = a
    kb, pb = b
    pos_a = np.arange(ka.shape[0]) + np.searchsorted(kb, ka, side="left")
    pos_b = np.arange(kb.shape[0]) + np.searchsorted(ka, kb, side="right")
    k = np.empty(ka.shape[0] + kb.shape[0], ka.dtype)
    p = np.empty(k.shape[0], pa.dtype)
    k[pos_a], k[pos_b] = ka, kb
    p[pos_a], p[pos_b] = pa, pb
    return k, p


def oracle_bounce(lo, hi, rays, obvh, table, threads: int = 1):
    """One bounce through the oracle, as it stands: keys, stable sort, gather,
    trace (the oracle's BVH) and the length-table update.  With threads > 1 the
    same oracle functions run on contiguous ray ranges in parallel (ctypes
    releases the GIL around every C call): keys, gather and trace by range;
    the sort as a stable sort per range followed by stable pairwise merges of
    neighbouring ranges (equal keys keep the lower indices first: the stable
    order).  The table is
    updated once, after the trace, as in the single-threaded run.  Returns
    (keys, perm, hits)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    n = rays.o_tmin.shape[0]
    if threads <= 1:
        keys = oracle.compute_keys(oracle.TWO_POINT, KEY_BITS, rays.o_tmin, rays.d_tmax, lo, hi,
                                   tsrc=oracle.T_ADAPTIVE, table=table)
        perm, _ = oracle.stable_sort(keys)
        so, sd, sp = oracle.permute(rays.o_tmin, rays.d_tmax, rays.payload, perm)
        h, _ = obvh.trace(so, sd)
        table.accumulate(lo, hi, so, sd, h)
        return keys, perm, h
    cuts = [n * k // threads for k in range(threads + 1)]
    ranges = [(cuts[k], cuts[k + 1]) for k in range(threads) if cuts[k + 1] > cuts[k]]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(lambda r: oracle.compute_keys(oracle.TWO_POINT, KEY_BITS, rays.o_tmin[r[0]:r[1]],
                                                          rays.d_tmax[r[0]:r[1]], lo, hi,
                                                          tsrc=oracle.T_ADAPTIVE, table=table), ranges))
        keys = np.concatenate(parts)
        sorted_parts = list(ex.map(lambda r: oracle.stable_sort(keys[r[0]:r[1]]), ranges))
        runs = [(sk, p + np.uint32(r[0])) for (p, sk), r in zip(sorted_parts, ranges)]
        while len(runs) > 1:  # pairwise merges of neighbouring ranges, in parallel
            pairs = [(runs[k], runs[k + 1]) for k in range(0, len(runs) - 1, 2)]
            merged = list(ex.map(lambda ab: stable_merge(*ab), pairs))
            runs = merged + ([runs[-1]] if len(runs) % 2 else [])
        perm = runs[0][1]
        gathered = list(ex.map(lambda r: oracle.permute(rays.o_tmin, rays.d_tmax, rays.payload,
                                                        perm[r[0]:r[1]]), ranges))
        so = np.concatenate([g[0] for g in gathered])
        sd = np.concatenate([g[1] for g in gathered])
        hits = list(ex.map(lambda r: obvh.trace(so[r[0]:r[1]], sd[r[0]:r[1]])[0], ranges))
    h = np.concatenate(hits)
    table.accumulate(lo, hi, so, sd, h)
    return keys, perm, h


def oracle_bounce_time(lo, hi, rays, obvh, table, threads: int = 1):
    t0 = time.perf_counter()
    oracle_bounce(lo, hi, rays, obvh, table, threads)
    return time.perf_counter() - t0


def cpu_baseline(tris, lo, hi, sample: int):
    """The oracle on a bounded sample of the same scene (a trace-free stand-in
    secondary wavefront of `sample` rays), on every host core and on one."""
    import oracle
    from paper_2506_11273_gb300 import workloads as W
    rays = W.surface_rays(tris, sample, seed=77)
    obvh = oracle.BVH(tris)
    cores = host_cores()
    E = oracle.largest_extent(lo, hi)
    dt = oracle_bounce_time(lo, hi, rays, obvh, oracle.LengthTable(E), threads=cores)
    one = W.Rays(rays.o_tmin[: sample // 4], rays.d_tmax[: sample // 4], rays.payload[: sample // 4])
    dt1 = oracle_bounce_time(lo, hi, one, obvh, oracle.LengthTable(E), threads=1)
    return {"value": round(sample / dt / 1e6, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d stand-in secondary rays (origins on the scene by area, BSDF directions) of the "
                      "same scene; keys + sort + gather + trace (oracle BVH) + accumulate on %d threads "
                      "(ray ranges; per-range stable sorts and stable pairwise merges)" % (sample, cores),
            "seconds": round(dt, 2),
            "single_thread": {"value": round(one.o_tmin.shape[0] / dt1 / 1e6, 4), "unit": UNIT, "cores": 1,
                              "rays": int(one.o_tmin.shape[0]), "seconds": round(dt1, 2)}}


def run_reference(args):
    """The reference arm: the oracle as it stands on the host's cores, on a
    bounded sample of the same workload per step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2506_11273_gb300 import workloads as W
    import oracle
    tris, _ = build_workload(args.small, seed=2)
    lo, hi = W.scene_aabb(tris)
    obvh = oracle.BVH(tris)
    table = oracle.LengthTable(oracle.largest_extent(lo, hi))
    cores = host_cores()
    sample = 20000 if args.small else 200000
    rays = W.surface_rays(tris, sample, seed=77)
    for _ in range(args.warmup):
        oracle_bounce_time(lo, hi, rays, obvh, table, threads=cores)
    ts = [oracle_bounce_time(lo, hi, rays, obvh, table, threads=cores) for _ in range(args.steps)]
    value = sample * args.steps / sum(ts) / 1e6
    desc = ("%d stand-in secondary rays per step (same scene), oracle keys + sort + gather + trace + accumulate "
            "on %d threads (ray ranges; per-range stable sorts and stable pairwise merges)" % (sample, cores))
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(ts) / args.steps, 2),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+u64",
           "data": "synthetic",
           "config": {"workload": "path tracer 1920x1080 1spp scene, %d-ray sample per step" % sample,
                      "key": "two_point_adaptive", "key_bits": KEY_BITS},
           "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.sweep:
        run_sweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
