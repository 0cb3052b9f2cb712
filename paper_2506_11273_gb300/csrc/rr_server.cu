// Serving loop: ray-batch requests against resident scenes, admitted under a
// device-memory budget and run with continuous batching.  A worker thread
// takes every request that has arrived (first come, first served, as far as
// the budget and a free stream slot allow), joins them into one multi-scene
// batch (keys in each request's own box, one stable sort with the request
// number above the key bits, one trace through the permutation), and enqueues
// copy-in, the batch and copy-out on the slot's stream.  Batches on different
// slots overlap on the device; requests that arrive meanwhile wait only for a
// slot and memory, not for earlier batches to finish.  Device memory comes
// from the stream-ordered pool (cudaMallocAsync / cudaFreeAsync on the slot's
// stream); the budget is enforced on the host before anything is enqueued.
// Completion is reported by a host function enqueued after the copy-out.
#include <algorithm>
#include <cmath>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "rr_batch.cuh"
#include "rr_common.cuh"

using namespace rr;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Request {
    uint64_t ticket;
    uint32_t scene;
    const float *o, *d;
    float *hits;
    // device addresses of the rays when they are page-locked host memory (then
    // they may be uploaded by the library's copy kernel), else null
    const float *o_dev = nullptr, *d_dev = nullptr;
    uint32_t n;
    rr_request_times times;
    rr_status status = RR_OK;
    bool done = false;
};

struct Group;

struct Slot {
    cudaStream_t stream = nullptr;
    uint32_t *queue = nullptr;       // trace work-queue words of this slot
    uint32_t *err = nullptr;         // device error word of the slot's stream
    uint32_t *h_err = nullptr;       // pinned: the flags of the slot's last group, read after its copy-out
    cudaEvent_t ev[4] = {};          // the group's stages: before copy-in, after it, after the trace, after copy-out
    BatchScene *h_segs = nullptr;    // pinned staging of the group's descriptors
    uint32_t *h_offs = nullptr;      // and offsets (one group in flight per slot)
    Group *busy = nullptr;
};

struct Group {
    rr_server *server = nullptr;
    uint32_t slot = 0;
    std::vector<Request *> reqs;
    size_t bytes = 0;    // charged against the budget
    bool timed = false;  // the slot's stage events were all recorded for this group
    bool kernel_copies = false;  // page-locked rays uploaded by the library's copy kernel
    uint64_t engine_bytes = 0;   // bytes uploaded by the copy engines
};

// Uploads of page-locked request rays normally go through the copy engines,
// which overlap other groups' kernels at no cost in SM time.  On GB300 the
// engines were measured to slow down to 11-20 GB/s for ~70 ms every ~0.5 s
// after an earlier process had used the GPU; a group whose engine upload runs
// below kSlowEngineGBs therefore switches uploads to the copy kernel (SM loads
// over the host link, unaffected) for kKernelCopyNs (the slowdowns persist
// for minutes once they start), after which the engines are tried again.
constexpr double kSlowEngineGBs = 40.0;
constexpr uint64_t kMinTimedUpload = 16ull << 20;
constexpr uint64_t kKernelCopyNs = 10000000000ull;

}  // namespace

struct rr_server {
    int device = 0;
    rr_server_config cfg{};
    std::vector<BatchScene> scenes;                 // descriptor of each resident scene
    std::vector<const rr_length_table *> tables;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> waiting;
    std::unordered_map<uint64_t, Request *> all;  // every request not yet released
    std::vector<Group *> finished;                // groups whose host function has run
    size_t reserved = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    uint64_t batches = 0, max_group = 0, peak_reserved = 0;
    std::string worker_error;
    int sm_count = 0;
    uint64_t kernel_copies_until = 0;  // steady-clock ns: uploads by the copy kernel until then
    uint64_t engine_slowdowns = 0, kernel_copy_groups = 0;
};

namespace {

bool adaptive(const rr_server *s) {
    return s->cfg.layout == RR_KEY_TWO_POINT && s->cfg.t_source == RR_T_ADAPTIVE;
}

// Device bytes a group of `n` rays in `g` requests needs: rays, hits, keys,
// permutation, sort workspace, descriptors.
size_t group_bytes(const rr_server *s, uint64_t n, uint32_t g, uint32_t total_bits) {
    size_t ws = 0;
    rr_sort_workspace_size((uint32_t)std::max<uint64_t>(n, 1), total_bits, s->cfg.radix_bits, &ws);
    return up256(16 * n) * 2 + up256(16 * n) + up256(8 * n) + up256(4 * n) + up256(ws) +
           up256(sizeof(BatchScene) * g) + up256(4 * (g + 1));
}

uint32_t bits_for(uint32_t n) {
    uint32_t b = 0;
    while ((1ull << b) < n) ++b;
    return b;
}

void CUDART_CB group_done(void *p) {
    Group *g = static_cast<Group *>(p);
    rr_server *s = g->server;
    const uint64_t t = now_ns();
    // the flags the group's kernels recorded on the slot's stream (taken from
    // its error word after the copy-out): they fail this group's requests only
    const uint32_t flags = *static_cast<volatile uint32_t *>(s->slots[g->slot].h_err);
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request *r : g->reqs) {
        r->times.done_ns = t;
        r->times.device_flags = flags;
        if (flags) r->status = RR_ERR_DEVICE;
    }
    s->finished.push_back(g);
    s->cv.notify_all();
}

// Enqueues one group on its slot; on failure marks its requests failed.
rr_status launch_group(rr_server *s, Group *g) {
    Slot &sl = s->slots[g->slot];
    cudaStream_t st = sl.stream;
    const uint32_t ng = (uint32_t)g->reqs.size();
    uint64_t n = 0;
    for (Request *r : g->reqs) n += r->n;
    const uint32_t seg_bits = bits_for(ng);
    const uint32_t key_bits = std::min(s->cfg.key_bits, 64u - seg_bits);
    const uint32_t total_bits = key_bits + seg_bits;
    size_t ws = 0;
    rr_sort_workspace_size((uint32_t)std::max<uint64_t>(n, 1), total_bits, s->cfg.radix_bits, &ws);
    unsigned char *mem = nullptr;
    cudaError_t e = cudaEventRecord(sl.ev[0], st);
    if (e == cudaSuccess) e = lib_malloc_async(reinterpret_cast<void **>(&mem), g->bytes, st);
    if (e == cudaErrorMemoryAllocation) return fail(RR_ERR_OOM, "rr_server: group memory could not be allocated");
    if (e != cudaSuccess) return fail_cuda(e, "rr_server: cudaMallocAsync");
    size_t off = 0;
    float *o = reinterpret_cast<float *>(mem + off);
    off += up256(16 * n);
    float *d = reinterpret_cast<float *>(mem + off);
    off += up256(16 * n);
    float *hits = reinterpret_cast<float *>(mem + off);
    off += up256(16 * n);
    void *keys = mem + off;
    off += up256(8 * n);
    uint32_t *perm = reinterpret_cast<uint32_t *>(mem + off);
    off += up256(4 * n);
    void *wsp = mem + off;
    off += up256(ws);
    BatchScene *segs = reinterpret_cast<BatchScene *>(mem + off);
    off += up256(sizeof(BatchScene) * ng);
    uint32_t *offs = reinterpret_cast<uint32_t *>(mem + off);
    uint64_t at = 0;
    rr_status cs = RR_OK;
    for (uint32_t k = 0; k < ng && e == cudaSuccess && cs == RR_OK; ++k) {
        Request *r = g->reqs[k];
        if (!(g->kernel_copies && r->o_dev && r->d_dev)) g->engine_bytes += 32ull * r->n;
        if (g->kernel_copies && r->o_dev && r->d_dev) {
            cs = enqueue_kernel_copy(o + 4 * at, r->o_dev, 16ull * r->n, s->sm_count, st);
            if (cs == RR_OK) cs = enqueue_kernel_copy(d + 4 * at, r->d_dev, 16ull * r->n, s->sm_count, st);
        } else {
            e = cudaMemcpyAsync(o + 4 * at, r->o, 16ull * r->n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d + 4 * at, r->d, 16ull * r->n, cudaMemcpyHostToDevice, st);
        }
        at += r->n;
    }
    if (cs != RR_OK) {
        cudaFreeAsync(mem, st);
        return cs;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(segs, sl.h_segs, sizeof(BatchScene) * ng, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(offs, sl.h_offs, 4ull * (ng + 1), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev[1], st);
    if (e != cudaSuccess) {
        cudaFreeAsync(mem, st);
        return fail_cuda(e, "rr_server: copy-in");
    }
    rr_status rs = RR_OK;
    if (n > 0) {
        rs = launch_keys_batch(segs, offs, ng, (rr_key_layout)s->cfg.layout, (rr_t_source)s->cfg.t_source,
                               s->cfg.ratio, key_bits, seg_bits, o, d, (uint32_t)n, keys, st);
        if (rs == RR_OK)
            rs = sort_enqueue(keys, nullptr, perm, (uint32_t)n, total_bits, s->cfg.radix_bits, wsp, sl.err,
                              s->sm_count, st);
        if (rs == RR_OK)
            rs = launch_trace_batch(segs, offs, ng, o, d, perm, (uint32_t)n, hits, adaptive(s),
                                    s->cfg.trace_block, sl.queue, sl.err, st);
    }
    if (rs == RR_OK) e = cudaEventRecord(sl.ev[2], st);
    at = 0;
    for (uint32_t k = 0; k < ng && rs == RR_OK && e == cudaSuccess; ++k) {
        Request *r = g->reqs[k];
        e = cudaMemcpyAsync(r->hits, hits + 4 * at, 16ull * r->n, cudaMemcpyDeviceToHost, st);
        at += r->n;
    }
    cudaFreeAsync(mem, st);
    if (rs != RR_OK) return rs;
    if (e != cudaSuccess) return fail_cuda(e, "rr_server: copy-out");
    rs = enqueue_take_error(sl.err, sl.h_err, st);
    if (rs != RR_OK) return rs;
    e = cudaEventRecord(sl.ev[3], st);
    if (e != cudaSuccess) return fail_cuda(e, "rr_server: event");
    e = cudaLaunchHostFunc(st, group_done, g);
    if (e != cudaSuccess) return fail_cuda(e, "rr_server: host function");
    return RR_OK;
}

void worker_main(rr_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lock(s->mu);
    while (true) {
        // retire finished groups: release their memory and slots
        for (Group *g : s->finished) {
            // the device time of the group's stages (its events have completed)
            const Slot &sl = s->slots[g->slot];
            float t[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (g->timed && cudaEventElapsedTime(&t[0], sl.ev[0], sl.ev[1]) == cudaSuccess &&
                cudaEventElapsedTime(&t[1], sl.ev[1], sl.ev[2]) == cudaSuccess &&
                cudaEventElapsedTime(&t[2], sl.ev[2], sl.ev[3]) == cudaSuccess &&
                cudaEventElapsedTime(&t[3], sl.ev[0], sl.ev[3]) == cudaSuccess) {
                for (Request *r : g->reqs) {
                    r->times.copy_in_ms = t[0];
                    r->times.kernels_ms = t[1];
                    r->times.copy_out_ms = t[2];
                    r->times.device_ms = t[3];
                    r->times.kernel_copies = g->kernel_copies ? 1u : 0u;
                }
                // a slow engine upload moves the next uploads to the copy kernel
                if (!g->kernel_copies && g->engine_bytes >= kMinTimedUpload && t[0] > 0.0f &&
                    (double)g->engine_bytes / (t[0] * 1e6) < kSlowEngineGBs) {
                    s->kernel_copies_until = now_ns() + kKernelCopyNs;
                    ++s->engine_slowdowns;
                }
            } else {
                cudaGetLastError();
            }
            for (Request *r : g->reqs) r->done = true;
            s->reserved -= g->bytes;
            s->slots[g->slot].busy = nullptr;
            delete g;
        }
        if (!s->finished.empty()) s->cv.notify_all();
        s->finished.clear();
        if (s->stop) {
            bool idle = true;
            for (const Slot &sl : s->slots) idle = idle && sl.busy == nullptr;
            if (idle && s->waiting.empty()) break;
        }
        // admit: everything that has arrived, in order, while a slot and memory allow
        int free_slot = -1;
        for (size_t k = 0; k < s->slots.size(); ++k)
            if (!s->slots[k].busy) {
                free_slot = (int)k;
                break;
            }
        if (free_slot >= 0 && !s->waiting.empty()) {
            Group *g = new Group();
            g->server = s;
            g->slot = (uint32_t)free_slot;
            g->kernel_copies = s->cfg.upload == RR_UPLOAD_KERNEL ||
                               (s->cfg.upload == RR_UPLOAD_ADAPTIVE && now_ns() < s->kernel_copies_until);
            if (g->kernel_copies) ++s->kernel_copy_groups;
            uint64_t n = 0;
            while (!s->waiting.empty() && g->reqs.size() < kMaxBatchSegments) {
                Request *r = s->waiting.front();
                const uint64_t n2 = n + r->n;
                if (!g->reqs.empty() && n2 > s->cfg.max_batch_rays) break;
                const uint32_t ng = (uint32_t)g->reqs.size() + 1;
                const size_t b = group_bytes(s, n2, ng, std::min(64u, s->cfg.key_bits + bits_for(ng)));
                if (s->reserved + b > s->cfg.budget_bytes) break;  // wait for memory (keeps arrival order)
                g->reqs.push_back(r);
                g->bytes = b;
                n = n2;
                s->waiting.pop_front();
            }
            if (g->reqs.empty()) {
                delete g;
            } else {
                const uint32_t ng = (uint32_t)g->reqs.size();
                s->reserved += g->bytes;
                s->peak_reserved = std::max<uint64_t>(s->peak_reserved, s->reserved);
                s->slots[g->slot].busy = g;
                ++s->batches;
                s->max_group = std::max<uint64_t>(s->max_group, ng);
                Slot &sl = s->slots[g->slot];
                uint64_t at = 0;
                const uint64_t t = now_ns();
                for (uint32_t k = 0; k < ng; ++k) {
                    sl.h_segs[k] = s->scenes[g->reqs[k]->scene];
                    sl.h_offs[k] = (uint32_t)at;
                    at += g->reqs[k]->n;
                    g->reqs[k]->times.start_ns = t;
                    g->reqs[k]->times.batch_requests = ng;
                }
                sl.h_offs[ng] = (uint32_t)at;
                lock.unlock();
                const rr_status st = launch_group(s, g);
                const uint64_t t_enq = now_ns();
                lock.lock();
                g->timed = st == RR_OK;
                for (Request *r : g->reqs) r->times.enqueued_ns = t_enq;
                if (st != RR_OK) {
                    s->worker_error = rr_last_error_message();
                    for (Request *r : g->reqs) {
                        r->status = st;
                        r->times.done_ns = now_ns();
                    }
                    // nothing after the failure point was enqueued: retire once the stream drains
                    lock.unlock();
                    cudaStreamSynchronize(s->slots[g->slot].stream);
                    cudaGetLastError();
                    lock.lock();
                    s->finished.push_back(g);
                }
                continue;
            }
        }
        s->cv.wait_for(lock, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" rr_status rr_server_create(const rr_server_config *cfg, rr_server **out) {
    if (!out || !cfg) return fail(RR_ERR_INVALID_ARG, "rr_server_create: NULL argument");
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64) return fail(RR_ERR_INVALID_ARG, "rr_server_create: slots must be 1..64");
    if (cfg->layout > RR_KEY_OCTAHEDRON || cfg->key_bits < 1 || cfg->key_bits > 64 ||
        (cfg->radix_bits != 4 && cfg->radix_bits != 8) ||
        (cfg->trace_block != 128 && cfg->trace_block != 256 && cfg->trace_block != 512))
        return fail(RR_ERR_INVALID_ARG, "rr_server_create: bad key, sort or trace settings");
    if (cfg->layout == RR_KEY_TWO_POINT && cfg->t_source == RR_T_GIVEN)
        return fail(RR_ERR_UNSUPPORTED, "rr_server_create: GIVEN estimates are not served");
    if (cfg->layout == RR_KEY_TWO_POINT && cfg->t_source > RR_T_GIVEN)
        return fail(RR_ERR_INVALID_ARG, "rr_server_create: bad t_source");
    if (cfg->max_batch_rays < 1 || cfg->max_batch_rays >= (1u << 30))
        return fail(RR_ERR_INVALID_ARG, "rr_server_create: max_batch_rays must be 1..2^30-1");
    if (cfg->upload > RR_UPLOAD_KERNEL) return fail(RR_ERR_INVALID_ARG, "rr_server_create: unknown upload policy");
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    rr_server *s = new rr_server();
    cudaGetDevice(&s->device);
    s->cfg = *cfg;
    s->sm_count = ds->sm_count;
    s->slots.resize(cfg->slots);
    cudaError_t e = cudaSuccess;
    for (Slot &sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) sl.err = error_word(ds, sl.stream);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl.h_err), sizeof(uint32_t));
        if (e == cudaSuccess) *sl.h_err = 0u;
        for (cudaEvent_t &ev : sl.ev)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
        if (e == cudaSuccess) e = lib_malloc(reinterpret_cast<void **>(&sl.queue), 2 * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMemset(sl.queue, 0, 2 * sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl.h_segs), sizeof(BatchScene) * kMaxBatchSegments);
        if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void **>(&sl.h_offs), 4ull * (kMaxBatchSegments + 1));
    }
    // keep freed pool memory cached for the next batches, up to the budget
    cudaMemPool_t pool = nullptr;
    if (e == cudaSuccess) e = cudaDeviceGetDefaultMemPool(&pool, s->device);
    if (e == cudaSuccess) {
        uint64_t thr = cfg->budget_bytes;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (e == cudaSuccess && cfg->reserve_bytes > 0) {
        // grow the pool once now; freed memory stays cached up to the threshold
        void *tmp = nullptr;
        const size_t bytes = (size_t)std::min<uint64_t>(cfg->reserve_bytes, cfg->budget_bytes);
        e = cudaMallocAsync(&tmp, bytes, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaFreeAsync(tmp, s->slots[0].stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->slots[0].stream);
    }
    if (e != cudaSuccess) {
        for (Slot &sl : s->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            cudaFree(sl.queue);
            cudaFreeHost(sl.h_segs);
            cudaFreeHost(sl.h_offs);
            cudaFreeHost(sl.h_err);
            for (cudaEvent_t ev : sl.ev)
                if (ev) cudaEventDestroy(ev);
        }
        delete s;
        return fail_cuda(e, "rr_server_create");
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return RR_OK;
}

extern "C" rr_status rr_server_add_scene(rr_server *s, const rr_bvh *bvh, rr_length_table *table,
                                         const float aabb_lo[3], const float aabb_hi[3], uint32_t *scene_id) {
    if (!s || !bvh || !aabb_lo || !aabb_hi || !scene_id)
        return fail(RR_ERR_INVALID_ARG, "rr_server_add_scene: NULL argument");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(aabb_lo[c]) || !std::isfinite(aabb_hi[c]) || !(aabb_lo[c] <= aabb_hi[c]))
            return fail(RR_ERR_INVALID_ARG, "rr_server_add_scene: bad box");
    if (adaptive(s)) {
        if (!table) return fail(RR_ERR_INVALID_ARG, "rr_server_add_scene: ADAPTIVE needs a table");
        if (std::memcmp(table->box.lo, aabb_lo, 12) || std::memcmp(table->box.hi, aabb_hi, 12))
            return fail(RR_ERR_INVALID_ARG, "rr_server_add_scene: table was created for another box");
    }
    // the descriptor, with the quantisation frame computed on the device
    BatchScene h{};
    h.nodes = reinterpret_cast<const float4 *>(bvh->nodes);
    h.tris = reinterpret_cast<const float4 *>(bvh->tris);
    h.planes = bvh->planes;
    h.n_nodes = bvh->n_nodes;
    h.n_tris = bvh->n_tris;
    h.table = adaptive(s) ? table->cells : nullptr;
    float box[6] = {aabb_lo[0], aabb_lo[1], aabb_lo[2], aabb_hi[0], aabb_hi[1], aabb_hi[2]};
    BatchScene *dseg = nullptr;
    float *dbox = nullptr;
    cudaError_t e = lib_malloc(reinterpret_cast<void **>(&dseg), sizeof(BatchScene));
    if (e == cudaSuccess) e = lib_malloc(reinterpret_cast<void **>(&dbox), sizeof(box));
    if (e == cudaSuccess) e = cudaMemcpy(dseg, &h, sizeof(BatchScene), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dbox, box, sizeof(box), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_batch_frames(dseg, dbox, 1, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&h, dseg, sizeof(BatchScene), cudaMemcpyDeviceToHost);
    cudaFree(dseg);
    cudaFree(dbox);
    if (e != cudaSuccess) return fail_cuda(e, "rr_server_add_scene");
    std::lock_guard<std::mutex> lock(s->mu);
    s->scenes.push_back(h);
    s->tables.push_back(table);
    *scene_id = (uint32_t)(s->scenes.size() - 1);
    return RR_OK;
}

extern "C" rr_status rr_server_submit(rr_server *s, uint32_t scene_id, const float *o_tmin_host,
                                      const float *d_tmax_host, uint32_t n, float *hits_host, uint64_t *ticket) {
    if (!s || !ticket) return fail(RR_ERR_INVALID_ARG, "rr_server_submit: NULL argument");
    if (n > 0 && (!o_tmin_host || !d_tmax_host || !hits_host))
        return fail(RR_ERR_INVALID_ARG, "rr_server_submit: NULL buffer");
    if (n > s->cfg.max_batch_rays) return fail(RR_ERR_INVALID_ARG, "rr_server_submit: n exceeds max_batch_rays");
    if (group_bytes(s, n, 1, s->cfg.key_bits) > s->cfg.budget_bytes)
        return fail(RR_ERR_INVALID_ARG, "rr_server_submit: request larger than the memory budget");
    Request *r = new Request();
    r->o = o_tmin_host;
    r->d = d_tmax_host;
    r->hits = hits_host;
    r->n = n;
    if (n > 0) {
        r->o_dev = static_cast<const float *>(mapped_host_range(o_tmin_host, 16ull * n));
        r->d_dev = static_cast<const float *>(mapped_host_range(d_tmax_host, 16ull * n));
        if (!aligned16(r->o_dev) || !aligned16(r->d_dev)) r->o_dev = r->d_dev = nullptr;
    }
    r->times = rr_request_times{};
    std::lock_guard<std::mutex> lock(s->mu);
    if (scene_id >= s->scenes.size()) {
        delete r;
        return fail(RR_ERR_INVALID_ARG, "rr_server_submit: unknown scene");
    }
    if (s->stop) {
        delete r;
        return fail(RR_ERR_INVALID_ARG, "rr_server_submit: server is shutting down");
    }
    r->scene = scene_id;
    r->ticket = s->next_ticket++;
    r->times.submit_ns = now_ns();
    s->waiting.push_back(r);
    s->all[r->ticket] = r;
    *ticket = r->ticket;
    s->cv.notify_all();
    return RR_OK;
}

extern "C" rr_status rr_server_wait(rr_server *s, uint64_t ticket, double timeout_s, rr_request_times *times) {
    if (!s) return fail(RR_ERR_INVALID_ARG, "rr_server_wait: NULL server");
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return fail(RR_ERR_INVALID_ARG, "rr_server_wait: unknown or released ticket");
    Request *r = it->second;
    if (fault_fires(Fault::Timeout)) return fail(RR_ERR_TIMEOUT, "rr_server_wait: injected time-out");
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (!r->done) {
        if (s->cv.wait_until(lock, until) == std::cv_status::timeout && !r->done)
            return fail(RR_ERR_TIMEOUT, "rr_server_wait: request not finished in time");
    }
    if (times) *times = r->times;
    const rr_status st = r->status;
    s->all.erase(it);
    delete r;
    if (st == RR_ERR_DEVICE) return fail(st, "rr_server_wait: a kernel of the request's group set a device error flag");
    if (st != RR_OK) return fail(st, "rr_server_wait: request failed: " + s->worker_error);
    return RR_OK;
}

extern "C" rr_status rr_server_stats(rr_server *s, rr_server_stats_t *out) {
    if (!s || !out) return fail(RR_ERR_INVALID_ARG, "rr_server_stats: NULL argument");
    std::lock_guard<std::mutex> lock(s->mu);
    out->batches = s->batches;
    out->max_batch_requests = s->max_group;
    out->peak_reserved_bytes = s->peak_reserved;
    out->reserved_bytes = s->reserved;
    out->waiting = s->waiting.size();
    out->engine_slowdowns = s->engine_slowdowns;
    out->kernel_copy_groups = s->kernel_copy_groups;
    return RR_OK;
}

extern "C" rr_status rr_server_destroy(rr_server *s) {
    if (!s) return RR_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    for (Slot &sl : s->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaFree(sl.queue);
        cudaFreeHost(sl.h_segs);
        cudaFreeHost(sl.h_offs);
        cudaFreeHost(sl.h_err);
        for (cudaEvent_t ev : sl.ev)
            if (ev) cudaEventDestroy(ev);
    }
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return RR_OK;
}
