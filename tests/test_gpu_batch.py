"""GPU parity of batched execution: many wavefronts over several resident
scenes run as one captured CUDA graph (rr_batch_run), against the oracle run
wavefront by wavefront and against the per-wavefront launch loop.

Each wavefront's slice of the batch permutation must equal the oracle's stable
sort of that wavefront's keys (its own box and table) plus its offset; hits
follow the trace rule; graph and loop agree bit for bit (hits, tables); the
autotuner returns a valid configuration and leaves the tables as it found them.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2506_11273_gb300 import rr
from paper_2506_11273_gb300 import workloads as W

from hitcheck import compare

pytestmark = pytest.mark.gpu

SIZES = [1000, 0, 1, 33333, 4097, 70000, 5, 20000, 12345]


@pytest.fixture(scope="module")
def world():
    scenes = [W.scene_box_soup(seed=1),
              W.scene_terrain(seed=4, cells_x=64, cells_z=128, n_boxes=300),
              W.scene_terrain(seed=5, cells_x=32, cells_z=64, n_boxes=50)]
    bvhs = [rr.BVH(t) for t in scenes]
    obvhs = [oracle.BVH(t) for t in scenes]
    boxes = [W.scene_aabb(t) for t in scenes]
    which = [k % 3 for k in range(len(SIZES))]
    fronts = []
    for k, (cnt, s) in enumerate(zip(SIZES, which)):
        fronts.append(W.surface_rays(scenes[s], cnt, seed=100 + k) if cnt else None)
    o = np.concatenate([f.o_tmin for f in fronts if f is not None])
    d = np.concatenate([f.d_tmax for f in fronts if f is not None])
    return dict(scenes=scenes, bvhs=bvhs, obvhs=obvhs, boxes=boxes, which=which, fronts=fronts, o=o, d=d)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def make_batch(world, layout, tsrc=rr.RR_T_FIXED, tables=None):
    fronts = []
    for k, cnt in enumerate(SIZES):
        s = world["which"][k]
        lo, hi = world["boxes"][s]
        fronts.append((world["bvhs"][s], tables[s] if tables else None, lo, hi, cnt))
    return rr.Batch(fronts, layout, tsrc)


def oracle_batch(world, olayout, bits, otsrc=oracle.T_FIXED, otables=None):
    """Per wavefront: oracle keys, stable sort, closest hits (in input order)."""
    perms, hits, infos = [], [], []
    off = 0
    for k, cnt in enumerate(SIZES):
        if cnt == 0:
            continue
        s = world["which"][k]
        f = world["fronts"][k]
        lo, hi = world["boxes"][s]
        keys = oracle.compute_keys(olayout, bits, f.o_tmin, f.d_tmax, lo, hi, tsrc=otsrc,
                                   table=otables[s] if otables else None)
        perms.append(oracle.stable_sort(keys)[0] + np.uint32(off))
        h, info = world["obvhs"][s].trace(f.o_tmin, f.d_tmax)
        hits.append(h)
        infos.append(info)
        off += cnt
    return np.concatenate(perms), np.concatenate(hits), np.concatenate(infos)


def check_hits(world, g_hits, o_hits, o_info):
    off = 0
    for k, cnt in enumerate(SIZES):
        if cnt == 0:
            continue
        s = world["which"][k]
        f = world["fronts"][k]
        sl = slice(off, off + cnt)
        compare(world["scenes"][s], f.o_tmin, f.d_tmax, g_hits[sl], o_hits[sl], o_info[sl])
        off += cnt


def local_to_global(perm_loop):
    out = perm_loop.copy()
    off = 0
    for cnt in SIZES:
        out[off:off + cnt] += np.uint32(off)
        off += cnt
    return out


@pytest.mark.parametrize("layout,olayout,bits", [
    (rr.RR_KEY_TWO_POINT, oracle.TWO_POINT, 20),   # 24-bit batch keys (u32)
    (rr.RR_KEY_AILA, oracle.AILA, 60),             # 64-bit batch keys
    (rr.RR_KEY_OCTAHEDRON, oracle.OCTAHEDRON, 28),
])
def test_batch_graph_matches_oracle_and_loop(world, layout, olayout, bits):
    b = make_batch(world, layout)
    assert b.info()["seg_bits"] == 4 and b.n == len(world["o"])
    o, d = _dev(world["o"]), _dev(world["d"])
    n = b.n
    cfg = rr.Batch.config(bits, 8, 256)
    hits = torch.empty(n, 4, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    b.run(o, d, hits, cfg, perm)
    p_or, h_or, i_or = oracle_batch(world, olayout, bits)
    assert np.array_equal(rr.u32_to_numpy(perm), p_or)
    g = hits.cpu().numpy()
    check_hits(world, g, h_or, i_or)
    # replaying the graph gives the same result
    hits.zero_()
    b.run(o, d, hits, cfg, perm)
    assert np.array_equal(_bits(hits.cpu().numpy()), _bits(g))
    assert b.info()["graphs"] == 1
    # the per-wavefront launch loop gives the same hits and permutation
    h2 = torch.empty(n, 4, device="cuda")
    p2 = torch.empty(n, dtype=torch.int32, device="cuda")
    b.run_loop(o, d, h2, cfg, p2)
    assert np.array_equal(_bits(h2.cpu().numpy()), _bits(g))
    assert np.array_equal(local_to_global(rr.u32_to_numpy(p2)), p_or)
    # radix width and trace block change nothing in the results
    b.run(o, d, hits, rr.Batch.config(bits, 4, 128), perm)
    assert np.array_equal(rr.u32_to_numpy(perm), p_or)
    assert np.array_equal(_bits(hits.cpu().numpy()), _bits(g))
    b.run(o, d, hits, rr.Batch.config(bits, 8, 512), perm)
    assert np.array_equal(_bits(hits.cpu().numpy()), _bits(g))
    assert rr.rr_device_error() == 0
    b.close()


def test_batch_adaptive_tables(world):
    """Two Point ADAPTIVE: keys read each scene's table as it stood before the
    batch; the trace adds the batch's hits.  Tables are primed from the oracle."""
    from test_gpu_trace import check_table_close
    tables, otables = [], []
    for s, tris in enumerate(world["scenes"]):
        lo, hi = world["boxes"][s]
        prime = W.surface_rays(tris, 20000, seed=900 + s)
        ph, _ = world["obvhs"][s].trace(prime.o_tmin, prime.d_tmax)
        ot = oracle.LengthTable(oracle.largest_extent(lo, hi))
        ot.accumulate(lo, hi, prime.o_tmin, prime.d_tmax, ph)
        t = rr.LengthTable(lo, hi)
        t.write(ot.sum, ot.cnt)
        tables.append(t)
        otables.append(ot)
    b = make_batch(world, rr.RR_KEY_TWO_POINT, rr.RR_T_ADAPTIVE, tables)
    o, d = _dev(world["o"]), _dev(world["d"])
    n = b.n
    cfg = rr.Batch.config(40, 8, 256)
    before = [t.read() for t in tables]
    hits = torch.empty(n, 4, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    b.run(o, d, hits, cfg, perm)
    p_or, h_or, i_or = oracle_batch(world, oracle.TWO_POINT, 40, oracle.T_ADAPTIVE, otables)
    assert np.array_equal(rr.u32_to_numpy(perm), p_or)
    g = hits.cpu().numpy()
    check_hits(world, g, h_or, i_or)
    after_graph = [t.read() for t in tables]
    # the oracle's tables after the batch: its own hits added
    off = 0
    for k, cnt in enumerate(SIZES):
        if cnt:
            s = world["which"][k]
            lo, hi = world["boxes"][s]
            f = world["fronts"][k]
            otables[s].accumulate(lo, hi, f.o_tmin, f.d_tmax, h_or[off:off + cnt])
        off += cnt
    for s in range(3):
        check_table_close(tables[s], otables[s], ambiguous=16)
    # the launch loop from the same starting tables: same hits, same tables
    for t, (sm, cn) in zip(tables, before):
        t.write(sm, cn)
    h2 = torch.empty(n, 4, device="cuda")
    p2 = torch.empty(n, dtype=torch.int32, device="cuda")
    b.run_loop(o, d, h2, cfg, p2)
    assert np.array_equal(_bits(h2.cpu().numpy()), _bits(g))
    assert np.array_equal(local_to_global(rr.u32_to_numpy(p2)), p_or)
    for t, (sm, cn) in zip(tables, after_graph):
        s2, c2 = t.read()
        assert np.array_equal(s2, sm) and np.array_equal(c2, cn)
    # the autotuner leaves the tables as it found them and picks a valid config
    best, ms = b.tune(o, d, h2)
    assert best.radix_bits in (4, 8) and best.trace_block in (128, 256, 512)
    assert 0 <= best.key_bits <= 60 and ms > 0 and best.layout in (-1, rr.RR_KEY_COSTA, rr.RR_KEY_AILA_COMPACT)
    for t, (sm, cn) in zip(tables, after_graph):
        s2, c2 = t.read()
        assert np.array_equal(s2, sm) and np.array_equal(c2, cn)
    assert rr.rr_device_error() == 0
    b.close()


def test_batch_rejects_bad_arguments(world):
    o, d = _dev(world["o"]), _dev(world["d"])
    b = make_batch(world, rr.RR_KEY_AILA)
    h = torch.empty(b.n, 4, device="cuda")
    for cfg in [(61, 8, 256), (20, 5, 256), (20, 8, 64)]:
        with pytest.raises(rr.RRError):
            b.run(o, d, h, rr.Batch.config(*cfg))
    with pytest.raises(rr.RRError):
        make_batch(world, rr.RR_KEY_TWO_POINT, rr.RR_T_GIVEN)
    with pytest.raises(rr.RRError):  # ADAPTIVE without tables
        make_batch(world, rr.RR_KEY_TWO_POINT, rr.RR_T_ADAPTIVE)
    b.close()


def test_batch_without_reordering(world):
    """key_bits 0: no keys, no sort; every ray traced in input order, same hits."""
    b = make_batch(world, rr.RR_KEY_TWO_POINT)
    o, d = _dev(world["o"]), _dev(world["d"])
    h1 = torch.empty(b.n, 4, device="cuda")
    h2 = torch.empty(b.n, 4, device="cuda")
    h3 = torch.empty(b.n, 4, device="cuda")
    b.run(o, d, h1, rr.Batch.config(0, 8, 256))
    b.run_loop(o, d, h2, rr.Batch.config(0, 8, 256))
    b.run(o, d, h3, rr.Batch.config(24, 8, 256))
    g = _bits(h1.cpu().numpy())
    assert np.array_equal(g, _bits(h2.cpu().numpy()))
    assert np.array_equal(g, _bits(h3.cpu().numpy()))
    _, h_or, i_or = oracle_batch(world, oracle.TWO_POINT, 24)
    check_hits(world, h1.cpu().numpy(), h_or, i_or)
    assert rr.rr_device_error() == 0
    b.close()


def test_batch_degenerate_shapes(world):
    """One wavefront; wavefronts that are all empty but one; a batch with no rays."""
    o, d = _dev(world["o"]), _dev(world["d"])
    s = 0
    lo, hi = world["boxes"][s]
    f = world["fronts"][0]
    n0 = len(f)
    one = rr.Batch([(world["bvhs"][s], None, lo, hi, n0)], rr.RR_KEY_TWO_POINT)
    assert one.info()["seg_bits"] == 0
    h = torch.empty(n0, 4, device="cuda")
    p = torch.empty(n0, dtype=torch.int32, device="cuda")
    one.run(o[:n0].contiguous(), d[:n0].contiguous(), h, rr.Batch.config(32, 8, 256), p)
    keys = oracle.compute_keys(oracle.TWO_POINT, 32, f.o_tmin, f.d_tmax, lo, hi)
    assert np.array_equal(rr.u32_to_numpy(p), oracle.stable_sort(keys)[0])
    one.close()
    sparse = rr.Batch([(world["bvhs"][1], None, *world["boxes"][1], 0), (world["bvhs"][s], None, lo, hi, n0),
                       (world["bvhs"][2], None, *world["boxes"][2], 0)], rr.RR_KEY_TWO_POINT)
    h2 = torch.empty(n0, 4, device="cuda")
    sparse.run(o[:n0].contiguous(), d[:n0].contiguous(), h2, rr.Batch.config(30, 8, 256), p)
    assert np.array_equal(rr.u32_to_numpy(p), oracle.stable_sort(
        oracle.compute_keys(oracle.TWO_POINT, 30, f.o_tmin, f.d_tmax, lo, hi))[0])
    assert np.array_equal(_bits(h2.cpu().numpy()), _bits(h.cpu().numpy()))
    sparse.close()
    empty = rr.Batch([(world["bvhs"][s], None, lo, hi, 0)], rr.RR_KEY_AILA)
    assert empty.n == 0
    empty.run(o, d, h, rr.Batch.config(16, 8, 256))  # nothing to do
    empty.close()
    assert rr.rr_device_error() == 0


def test_batch_config_layout_overrides_the_key(world):
    """A configuration's layout orders the rays with another key family (Two
    Point falls back to the FIXED estimate); graph and loop agree; hits stay."""
    b = make_batch(world, rr.RR_KEY_TWO_POINT)
    o, d = _dev(world["o"]), _dev(world["d"])
    n = b.n
    base = torch.empty(n, 4, device="cuda")
    b.run(o, d, base, rr.Batch.config(24, 8, 256))
    for layout, olayout, bits in [(rr.RR_KEY_COSTA, oracle.COSTA, 28), (rr.RR_KEY_AILA_COMPACT, oracle.AILA_COMPACT, 40)]:
        hits = torch.empty(n, 4, device="cuda")
        perm = torch.empty(n, dtype=torch.int32, device="cuda")
        cfg = rr.Batch.config(bits, 8, 256, layout)
        b.run(o, d, hits, cfg, perm)
        p_or, _, _ = oracle_batch(world, olayout, bits)
        assert np.array_equal(rr.u32_to_numpy(perm), p_or)
        assert np.array_equal(_bits(hits.cpu().numpy()), _bits(base.cpu().numpy()))
        p2 = torch.empty(n, dtype=torch.int32, device="cuda")
        b.run_loop(o, d, hits, cfg, p2)
        assert np.array_equal(local_to_global(rr.u32_to_numpy(p2)), p_or)
    with pytest.raises(rr.RRError):
        b.run(o, d, base, rr.Batch.config(24, 8, 256, 9))
    best, _ = b.tune(o, d, base)
    assert best.layout in (-1, rr.RR_KEY_COSTA, rr.RR_KEY_AILA_COMPACT)
    assert rr.rr_device_error() == 0
    b.close()


def test_batch_tune_cached(world, tmp_path):
    """The first call tunes and writes the file; a second batch of the same
    kind takes the entry without timing; a batch of another size bucket is
    tuned again and its entry added; the file is JSON any reader can parse."""
    import json
    import time
    path = str(tmp_path / "tune.json")
    o, d = _dev(world["o"]), _dev(world["d"])
    b = make_batch(world, rr.RR_KEY_AILA)
    h = torch.empty(b.n, 4, device="cuda")
    best, ms, hit = b.tune_cached(o, d, h, path)
    assert not hit and ms > 0 and best.radix_bits in (4, 8) and best.trace_block in (128, 256, 512)
    doc = json.load(open(path))
    assert doc["format"] == "rr-batch-tune-cache" and len(doc["entries"]) == 1
    (key, entry), = doc["entries"].items()
    assert "rays2^" in key and entry["key_bits"] == best.key_bits and entry["trace_block"] == best.trace_block
    b2 = make_batch(world, rr.RR_KEY_AILA)
    t0 = time.perf_counter()
    best2, ms2, hit2 = b2.tune_cached(o, d, h, path)
    dt = time.perf_counter() - t0
    assert hit2 and dt < 0.05
    assert (best2.key_bits, best2.radix_bits, best2.trace_block, best2.layout) == \
        (best.key_bits, best.radix_bits, best.trace_block, best.layout)
    assert abs(ms2 - ms) <= 1e-3 * ms
    b2.run(o, d, h, best2)  # the cached configuration runs
    # another layout is another entry
    b3 = make_batch(world, rr.RR_KEY_COSTA)
    _, _, hit3 = b3.tune_cached(o, d, h, path)
    assert not hit3 and len(json.load(open(path))["entries"]) == 2
    # an entry the batch cannot run is tuned again and replaced
    doc = json.load(open(path))
    doc["entries"][key]["radix_bits"] = 5
    json.dump(doc, open(path, "w"))
    _, _, hit4 = b.tune_cached(o, d, h, path)
    assert not hit4 and json.load(open(path))["entries"][key]["radix_bits"] in (4, 8)
    with pytest.raises(rr.RRError):
        b.tune_cached(o, d, h, str(tmp_path / "no_such_dir" / "tune.json"))
    for x in (b, b2, b3):
        x.close()
    assert rr.rr_device_error() == 0
