// Batched execution: many wavefronts over several resident scenes keyed,
// sorted per wavefront and traced by one chain of launches that is captured
// once into a CUDA graph and replayed.  The per-wavefront sort is one global
// stable sort of keys that carry the wavefront number above the key's own
// bits, so each wavefront comes out sorted in place (Section 3.2's local
// sort with wavefront-sized segments); the trace reads the rays through the
// permutation (the indirect access of Section 4.4.1) and writes hits in input order.
// A small autotuner times candidate (key bits, radix width, trace block)
// configurations on the batch itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rr_batch.cuh"
#include "rr_tune_cache.h"
#include "rr_common.cuh"

using namespace rr;

namespace {

constexpr size_t kMaxGraphs = 32;  // captured graphs kept per batch

struct GraphEntry {
    rr_batch_config cfg;
    const float *o, *d;
    float *hits;
    uint32_t *perm;
    uint32_t *err;  // error word of the stream the graph reports to
    cudaGraphExec_t exec;
};

uint32_t bits_for(uint32_t n) {  // bits that number 0..n-1
    uint32_t b = 0;
    while ((1ull << b) < n) ++b;
    return b;
}

bool config_ok(const rr_batch_config *c, uint32_t seg_bits) {
    return c && c->key_bits + seg_bits <= 64 && (c->radix_bits == 4 || c->radix_bits == 8) &&
           c->layout >= -1 && c->layout <= (int32_t)RR_KEY_OCTAHEDRON &&
           (c->trace_block == 128 || c->trace_block == 256 || c->trace_block == 512);
}

bool same_cfg(const rr_batch_config &a, const rr_batch_config &b) {
    return a.key_bits == b.key_bits && a.radix_bits == b.radix_bits && a.trace_block == b.trace_block &&
           a.layout == b.layout;
}

}  // namespace

struct rr_batch {
    int device = 0;
    uint32_t n_fronts = 0, n_total = 0, seg_bits = 0;
    rr_key_layout layout = RR_KEY_TWO_POINT;
    rr_t_source tsrc = RR_T_FIXED;
    float ratio = 0.25f;
    std::vector<rr_wavefront> fronts;
    std::vector<uint32_t> offsets;           // host copy, n_fronts + 1
    std::vector<unsigned long long *> tables;  // distinct tables of the wavefronts
    unsigned char *mem = nullptr;            // one allocation for everything below
    BatchScene *d_segs = nullptr;
    uint32_t *d_offsets = nullptr;
    uint32_t *queue = nullptr;               // trace work-queue words of this batch
    void *keys = nullptr;                    // u64 [n_total]
    uint32_t *perm = nullptr;                // used when the caller passes no perm
    unsigned char *sort_ws = nullptr;
    size_t sort_ws_bytes = 0;
    cudaStream_t capture = nullptr;          // graphs are captured on this stream
    std::vector<GraphEntry> graphs;
};

namespace {

bool accumulating(const rr_batch *b) { return b->layout == RR_KEY_TWO_POINT && b->tsrc == RR_T_ADAPTIVE; }

// The layout and estimate a configuration keys with: the batch's own, or
// another layout that only orders the rays (Two Point with the FIXED estimate).
rr_key_layout run_layout(const rr_batch *b, const rr_batch_config &c) {
    return c.layout < 0 ? b->layout : (rr_key_layout)c.layout;
}
rr_t_source run_tsrc(const rr_batch *b, const rr_batch_config &c) {
    const rr_key_layout l = run_layout(b, c);
    return l == RR_KEY_TWO_POINT && l == b->layout ? b->tsrc : RR_T_FIXED;
}

// The whole chain on one stream: keys, sort, trace.  Device errors go to
// `err` (the word of the stream the chain is replayed on, not the capture
// stream's).
rr_status enqueue_batch(rr_batch *b, const float *o, const float *d, float *hits, uint32_t *perm,
                        const rr_batch_config &c, uint32_t *err, int sm_count, cudaStream_t s) {
    if (c.key_bits == 0)  // no reordering: every ray traced in input order
        return launch_trace_batch(b->d_segs, b->d_offsets, b->n_fronts, o, d, nullptr, b->n_total, hits,
                                  accumulating(b), c.trace_block, b->queue, err, s);
    rr_status st = launch_keys_batch(b->d_segs, b->d_offsets, b->n_fronts, run_layout(b, c), run_tsrc(b, c), b->ratio,
                                     c.key_bits,
                                     b->seg_bits, o, d, b->n_total, b->keys, s);
    if (st != RR_OK) return st;
    st = sort_enqueue(b->keys, nullptr, perm, b->n_total, c.key_bits + b->seg_bits, c.radix_bits, b->sort_ws, err,
                      sm_count, s);
    if (st != RR_OK) return st;
    return launch_trace_batch(b->d_segs, b->d_offsets, b->n_fronts, o, d, perm, b->n_total, hits, accumulating(b),
                              c.trace_block, b->queue, err, s);
}

rr_status check_run_args(const rr_batch *b, const float *o, const float *d, const float *hits,
                         const rr_batch_config *cfg, const char *what) {
    if (!b) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": NULL batch");
    if (!config_ok(cfg, b->seg_bits)) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": bad config");
    if (b->n_total == 0) return RR_OK;
    if (!o || !d || !hits) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": NULL buffer");
    if (!aligned16(o) || !aligned16(d) || !aligned16(hits))
        return fail(RR_ERR_INVALID_ARG, std::string(what) + ": buffers not 16-byte aligned");
    const size_t nb = 16ull * b->n_total;
    if (overlaps(hits, nb, o, nb) || overlaps(hits, nb, d, nb))
        return fail(RR_ERR_INVALID_ARG, std::string(what) + ": hits overlap the rays");
    return RR_OK;
}

}  // namespace

extern "C" rr_status rr_batch_create(const rr_wavefront *fronts, uint32_t n_fronts, rr_key_layout layout,
                                     rr_t_source t_source, float ratio, rr_batch **out) {
    if (!out) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: out is NULL");
    *out = nullptr;
    if (n_fronts == 0 || n_fronts > kMaxBatchSegments || !fronts)
        return fail(RR_ERR_INVALID_ARG, "rr_batch_create: need 1..1024 wavefronts");
    if (layout > RR_KEY_OCTAHEDRON) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: bad layout");
    const bool two_point = layout == RR_KEY_TWO_POINT;
    if (two_point && t_source == RR_T_GIVEN)
        return fail(RR_ERR_UNSUPPORTED, "rr_batch_create: GIVEN estimates are not batched");
    if (two_point && t_source > RR_T_GIVEN) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: bad t_source");
    if (two_point && t_source == RR_T_FIXED && !std::isfinite(ratio))
        return fail(RR_ERR_INVALID_ARG, "rr_batch_create: ratio not finite");
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    uint64_t next = 0;
    std::vector<float> boxes(6 * (size_t)n_fronts);
    for (uint32_t k = 0; k < n_fronts; ++k) {
        const rr_wavefront &f = fronts[k];
        if (!f.bvh) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: wavefront without a BVH");
        if (f.bvh->device != dev) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: BVH of another device");
        if (f.offset != next) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: wavefronts must be contiguous, in order");
        next += f.count;
        for (int c = 0; c < 3; ++c) {
            if (!std::isfinite(f.aabb_lo[c]) || !std::isfinite(f.aabb_hi[c]) || !(f.aabb_lo[c] <= f.aabb_hi[c]))
                return fail(RR_ERR_INVALID_ARG, "rr_batch_create: bad box");
            boxes[6 * k + c] = f.aabb_lo[c];
            boxes[6 * k + 3 + c] = f.aabb_hi[c];
        }
        if (two_point && t_source == RR_T_ADAPTIVE) {
            if (!f.table) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: ADAPTIVE needs a table per wavefront");
            if (std::memcmp(f.table->box.lo, f.aabb_lo, sizeof(float) * 3) ||
                std::memcmp(f.table->box.hi, f.aabb_hi, sizeof(float) * 3))
                return fail(RR_ERR_INVALID_ARG, "rr_batch_create: table was created for another box");
        }
    }
    if (next >= (1ull << 30)) return fail(RR_ERR_INVALID_ARG, "rr_batch_create: more than 2^30 rays");
    rr_batch *b = new rr_batch();
    b->device = dev;
    b->n_fronts = n_fronts;
    b->n_total = (uint32_t)next;
    b->seg_bits = bits_for(n_fronts);
    b->layout = layout;
    b->tsrc = two_point ? t_source : RR_T_FIXED;
    b->ratio = ratio;
    b->fronts.assign(fronts, fronts + n_fronts);
    b->offsets.resize(n_fronts + 1);
    for (uint32_t k = 0; k < n_fronts; ++k) b->offsets[k] = fronts[k].offset;
    b->offsets[n_fronts] = b->n_total;
    if (accumulating(b))
        for (uint32_t k = 0; k < n_fronts; ++k)
            if (std::find(b->tables.begin(), b->tables.end(), fronts[k].table->cells) == b->tables.end())
                b->tables.push_back(fronts[k].table->cells);
    // workspace for the widest sort any config can ask for
    size_t ws4 = 0, ws8 = 0;
    const uint32_t nsort = std::max(1u, b->n_total);
    rr_sort_workspace_size(nsort, 64, 4, &ws4);
    rr_sort_workspace_size(nsort, 64, 8, &ws8);
    b->sort_ws_bytes = std::max(ws4, ws8);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off = 0;
    const size_t o_segs = off;
    off = up(off + sizeof(BatchScene) * n_fronts);
    const size_t o_offs = off;
    off = up(off + sizeof(uint32_t) * (n_fronts + 1));
    const size_t o_queue = off;
    off = up(off + 2 * sizeof(uint32_t));
    const size_t o_boxes = off;
    off = up(off + sizeof(float) * boxes.size());
    const size_t o_keys = off;
    off = up(off + 8ull * nsort);
    const size_t o_perm = off;
    off = up(off + 4ull * nsort);
    const size_t o_ws = off;
    off = up(off + b->sort_ws_bytes);
    cudaError_t e = lib_malloc(reinterpret_cast<void **>(&b->mem), off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(RR_ERR_OOM, "rr_batch_create: cudaMalloc failed");
    }
    b->d_segs = reinterpret_cast<BatchScene *>(b->mem + o_segs);
    b->d_offsets = reinterpret_cast<uint32_t *>(b->mem + o_offs);
    b->queue = reinterpret_cast<uint32_t *>(b->mem + o_queue);
    b->keys = b->mem + o_keys;
    b->perm = reinterpret_cast<uint32_t *>(b->mem + o_perm);
    b->sort_ws = b->mem + o_ws;
    std::vector<BatchScene> segs(n_fronts);
    for (uint32_t k = 0; k < n_fronts; ++k) {
        const rr_bvh *h = fronts[k].bvh;
        segs[k].nodes = reinterpret_cast<const float4 *>(h->nodes);
        segs[k].tris = reinterpret_cast<const float4 *>(h->tris);
        segs[k].planes = h->planes;
        segs[k].n_nodes = h->n_nodes;
        segs[k].n_tris = h->n_tris;
        segs[k].table = accumulating(b) ? fronts[k].table->cells : nullptr;
        segs[k].invE = 0.0f;
        std::memset(&segs[k].frame, 0, sizeof(QuantFrame));
    }
    e = cudaMemcpy(b->d_segs, segs.data(), sizeof(BatchScene) * n_fronts, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_offsets, b->offsets.data(), sizeof(uint32_t) * (n_fronts + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->queue, 0, 2 * sizeof(uint32_t));
    float *d_boxes = reinterpret_cast<float *>(b->mem + o_boxes);
    if (e == cudaSuccess) e = cudaMemcpy(d_boxes, boxes.data(), sizeof(float) * boxes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_batch_frames(b->d_segs, d_boxes, n_fronts, nullptr);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(b->mem);
        if (b->capture) cudaStreamDestroy(b->capture);
        delete b;
        return fail_cuda(e, "rr_batch_create");
    }
    *out = b;
    return RR_OK;
}

extern "C" rr_status rr_batch_destroy(rr_batch *b) {
    if (!b) return RR_OK;
    for (GraphEntry &g : b->graphs) cudaGraphExecDestroy(g.exec);
    if (b->capture) cudaStreamDestroy(b->capture);
    cudaFree(b->mem);
    delete b;
    return RR_OK;
}

extern "C" rr_status rr_batch_info(const rr_batch *b, uint32_t *n_rays, uint32_t *seg_bits, uint32_t *n_graphs) {
    if (!b) return fail(RR_ERR_INVALID_ARG, "rr_batch_info: NULL batch");
    if (n_rays) *n_rays = b->n_total;
    if (seg_bits) *seg_bits = b->seg_bits;
    if (n_graphs) *n_graphs = (uint32_t)b->graphs.size();
    return RR_OK;
}

extern "C" rr_status rr_batch_run(rr_batch *b, const float *o_tmin, const float *d_tmax, float *hits_out,
                                  uint32_t *perm_out, const rr_batch_config *cfg, void *stream) {
    rr_status st = check_run_args(b, o_tmin, d_tmax, hits_out, cfg, "rr_batch_run");
    if (st != RR_OK || b->n_total == 0) return st;
    uint32_t *perm = perm_out ? perm_out : b->perm;
    if (!aligned(perm, 4)) return fail(RR_ERR_INVALID_ARG, "rr_batch_run: perm misaligned");
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    uint32_t *err = error_word(ds, as_stream(stream));
    GraphEntry *g = nullptr;
    for (GraphEntry &x : b->graphs)
        if (same_cfg(x.cfg, *cfg) && x.o == o_tmin && x.d == d_tmax && x.hits == hits_out && x.perm == perm &&
            x.err == err)
            g = &x;
    if (!g) {
        if (b->graphs.size() >= kMaxGraphs) {  // keep the cache bounded: drop the oldest graph
            cudaGraphExecDestroy(b->graphs.front().exec);
            b->graphs.erase(b->graphs.begin());
        }
        // capture the chain once for these buffers and this configuration
        cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return fail_cuda(e, "rr_batch_run: begin capture");
        st = enqueue_batch(b, o_tmin, d_tmax, hits_out, perm, *cfg, err, ds->sm_count, b->capture);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(b->capture, &graph);
        if (st != RR_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return fail_cuda(e, "rr_batch_run: end capture");
        cudaGraphExec_t exec = nullptr;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail_cuda(e, "rr_batch_run: instantiate");
        b->graphs.push_back(GraphEntry{*cfg, o_tmin, d_tmax, hits_out, perm, err, exec});
        g = &b->graphs.back();
    }
    const cudaError_t e = cudaGraphLaunch(g->exec, as_stream(stream));
    if (e != cudaSuccess) return fail_cuda(e, "rr_batch_run: graph launch");
    return RR_OK;
}

extern "C" rr_status rr_batch_run_loop(rr_batch *b, const float *o_tmin, const float *d_tmax, float *hits_out,
                                       uint32_t *perm_out, const rr_batch_config *cfg, void *stream) {
    rr_status st = check_run_args(b, o_tmin, d_tmax, hits_out, cfg, "rr_batch_run_loop");
    if (st != RR_OK || b->n_total == 0) return st;
    if (cfg->key_bits > 64) return fail(RR_ERR_INVALID_ARG, "rr_batch_run_loop: bad config");
    uint32_t *perm = perm_out ? perm_out : b->perm;
    const size_t kb = cfg->key_bits > 32 ? 8 : 4;
    unsigned char *keys = static_cast<unsigned char *>(b->keys);
    if (cfg->key_bits == 0) {
        for (uint32_t k = 0; k < b->n_fronts; ++k) {
            const rr_wavefront &f = b->fronts[k];
            if (f.count == 0) continue;
            st = rr_trace_ex(f.bvh, o_tmin + 4ull * f.offset, d_tmax + 4ull * f.offset, nullptr, f.count,
                             hits_out + 4ull * f.offset, 0u, accumulating(b) ? f.table : nullptr, stream);
            if (st != RR_OK) return st;
        }
        return RR_OK;
    }
    // as in the graph: every key is computed before any trace updates a table
    for (uint32_t k = 0; k < b->n_fronts; ++k) {
        const rr_wavefront &f = b->fronts[k];
        if (f.count == 0) continue;
        rr_key_params p{};
        p.layout = run_layout(b, *cfg);
        p.bits = cfg->key_bits;
        p.t_source = run_tsrc(b, *cfg);
        p.ratio = b->ratio;
        for (int c = 0; c < 3; ++c) {
            p.aabb_lo[c] = f.aabb_lo[c];
            p.aabb_hi[c] = f.aabb_hi[c];
        }
        p.table = p.t_source == RR_T_ADAPTIVE ? f.table : nullptr;
        st = rr_compute_keys(o_tmin + 4ull * f.offset, d_tmax + 4ull * f.offset, f.count, &p, keys + kb * f.offset,
                             stream);
        if (st != RR_OK) return st;
    }
    for (uint32_t k = 0; k < b->n_fronts; ++k) {
        const rr_wavefront &f = b->fronts[k];
        if (f.count == 0) continue;
        st = rr_sort(keys + kb * f.offset, nullptr, perm + f.offset, f.count, cfg->key_bits, cfg->radix_bits,
                     b->sort_ws, b->sort_ws_bytes, stream);
        if (st != RR_OK) return st;
    }
    for (uint32_t k = 0; k < b->n_fronts; ++k) {
        const rr_wavefront &f = b->fronts[k];
        if (f.count == 0) continue;
        st = rr_trace_ex(f.bvh, o_tmin + 4ull * f.offset, d_tmax + 4ull * f.offset, perm + f.offset, f.count,
                         hits_out + 4ull * f.offset, 0u, accumulating(b) ? f.table : nullptr, stream);
        if (st != RR_OK) return st;
    }
    return RR_OK;
}

extern "C" rr_status rr_batch_tune(rr_batch *b, const float *o_tmin, const float *d_tmax, float *hits_out,
                                   rr_batch_config *best, float *best_ms, void *stream) {
    if (!b || !best) return fail(RR_ERR_INVALID_ARG, "rr_batch_tune: NULL argument");
    rr_batch_config probe{16, 8, 256, -1};
    rr_status st = check_run_args(b, o_tmin, d_tmax, hits_out, &probe, "rr_batch_tune");
    if (st != RR_OK) return st;
    cudaStream_t s = as_stream(stream);
    // the tables change with every traced run: keep a copy and put it back
    std::vector<unsigned long long *> saved;
    const size_t tbytes = sizeof(unsigned long long) * 2 * kTableCells;
    for (unsigned long long *t : b->tables) {
        unsigned long long *c = nullptr;
        if (lib_malloc(reinterpret_cast<void **>(&c), tbytes) != cudaSuccess) {
            cudaGetLastError();
            for (unsigned long long *x : saved) cudaFree(x);
            return fail(RR_ERR_OOM, "rr_batch_tune: no room to save the length tables");
        }
        cudaMemcpyAsync(c, t, tbytes, cudaMemcpyDeviceToDevice, s);
        saved.push_back(c);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto time_cfg = [&](const rr_batch_config &c, float *ms) -> rr_status {
        rr_status r = rr_batch_run(b, o_tmin, d_tmax, hits_out, nullptr, &c, stream);  // capture + warm-up
        if (r != RR_OK) return r;
        float tot = 0.0f;
        const int reps = 3;
        for (int k = 0; k < reps; ++k) {
            cudaEventRecord(e0, s);
            r = rr_batch_run(b, o_tmin, d_tmax, hits_out, nullptr, &c, stream);
            if (r != RR_OK) return r;
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(RR_ERR_CUDA, "rr_batch_tune: timing");
            float x = 0.0f;
            cudaEventElapsedTime(&x, e0, e1);
            tot += x;
        }
        *ms = tot / reps;
        return RR_OK;
    };
    // key bits x radix width at the default block (0 bits: no reordering), then
    // the block for the winner
    const uint32_t cand_bits[] = {0, 12, 16, 20, 24, 32, 48, 64};
    std::vector<int32_t> cand_layouts{-1};
    for (rr_key_layout l : {RR_KEY_COSTA, RR_KEY_AILA_COMPACT})
        if (l != b->layout) cand_layouts.push_back((int32_t)l);
    rr_batch_config win{0, 0, 0, -1};
    float win_ms = -1.0f;
    st = RR_OK;
    for (int32_t lay : cand_layouts) {
        for (uint32_t kb : cand_bits) {
            if (kb == 0 && lay != -1) continue;  // no reordering is tried once
            const uint32_t bits = std::min(kb, 64u - b->seg_bits);
            for (uint32_t rb : {4u, 8u}) {
                if (kb == 0 && rb == 4) continue;  // nothing is sorted
                const rr_batch_config c{bits, rb, 256, lay};
                float ms = 0.0f;
                st = time_cfg(c, &ms);
                if (st != RR_OK) break;
                if (win_ms < 0.0f || ms < win_ms) {
                    win = c;
                    win_ms = ms;
                }
            }
            if (st != RR_OK) break;
        }
        if (st != RR_OK) break;
    }
    for (uint32_t blk : {128u, 512u}) {
        if (st != RR_OK) break;
        rr_batch_config c = win;
        c.trace_block = blk;
        float ms = 0.0f;
        st = time_cfg(c, &ms);
        if (st == RR_OK && ms < win_ms) {
            win = c;
            win_ms = ms;
        }
    }
    for (size_t k = 0; k < saved.size(); ++k) {
        cudaMemcpyAsync(b->tables[k], saved[k], tbytes, cudaMemcpyDeviceToDevice, s);
    }
    cudaStreamSynchronize(s);
    for (unsigned long long *x : saved) cudaFree(x);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != RR_OK) return st;
    *best = win;
    if (best_ms) *best_ms = win_ms;
    return RR_OK;
}

namespace {

uint32_t log2_floor(uint32_t x) {
    uint32_t r = 0;
    while (x > 1u) {
        x >>= 1;
        ++r;
    }
    return r;
}

// The cache key of a batch: what the tuner's choice depends on.  The GPU (name,
// SM count, compute capability), the batch's size to a power of two, its
// wavefront count to a power of two, the wavefront bits, and the layout and
// estimate of its keys.
std::string tune_key(const rr_batch *b) {
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, b->device);
    std::string name;
    for (const char *c = prop.name; *c; ++c)
        if (*c != '|' && *c != '"' && *c != '\\') name.push_back(*c);
    return name + "|sm" + std::to_string(prop.multiProcessorCount) + "|cc" + std::to_string(prop.major) + "." +
           std::to_string(prop.minor) + "|rays2^" + std::to_string(log2_floor(b->n_total)) + "|fronts2^" +
           std::to_string(log2_floor(b->n_fronts)) + "|seg" + std::to_string(b->seg_bits) + "|layout" +
           std::to_string((int)b->layout) + "|tsrc" + std::to_string((int)b->tsrc) + "|tuner1";
}

}  // namespace

extern "C" rr_status rr_batch_tune_cached(rr_batch *b, const float *o_tmin, const float *d_tmax, float *hits_out,
                                          const char *cache_path, rr_batch_config *best, float *best_ms,
                                          uint32_t *from_cache, void *stream) {
    if (!b || !best || !cache_path || !*cache_path)
        return fail(RR_ERR_INVALID_ARG, "rr_batch_tune_cached: NULL argument");
    rr_batch_config probe{16, 8, 256, -1};
    rr_status st = check_run_args(b, o_tmin, d_tmax, hits_out, &probe, "rr_batch_tune_cached");
    if (st != RR_OK) return st;
    const std::string key = tune_key(b);
    TuneEntry e;
    if (tune_cache_lookup(cache_path, key, &e)) {
        const rr_batch_config c{e.key_bits, e.radix_bits, e.trace_block, e.layout};
        // an entry this library could not run (a stale or edited file) is tuned again
        if (check_run_args(b, o_tmin, d_tmax, hits_out, &c, "rr_batch_tune_cached") == RR_OK) {
            *best = c;
            if (best_ms) *best_ms = (float)e.ms;
            if (from_cache) *from_cache = 1u;
            return RR_OK;
        }
    }
    float ms = 0.0f;
    st = rr_batch_tune(b, o_tmin, d_tmax, hits_out, best, &ms, stream);
    if (st != RR_OK) return st;
    if (best_ms) *best_ms = ms;
    if (from_cache) *from_cache = 0u;
    e.key_bits = best->key_bits;
    e.radix_bits = best->radix_bits;
    e.trace_block = best->trace_block;
    e.layout = best->layout;
    e.ms = ms;
    std::string err;
    if (!tune_cache_store(cache_path, key, e, &err)) return fail(RR_ERR_INVALID_ARG, "rr_batch_tune_cached: " + err);
    return RR_OK;
}
