// One bounce of the reordered path behind a single handle: keys -> sort ->
// reorder -> trace, then the length-table update when the Two Point key takes
// its estimate from the table (Section 3.1.6: accumulate after each trace).
#include "rr_common.cuh"

// Host-buffer submissions alternate between two staging slots, so the upload
// of one submission overlaps the kernels of the one before it.
struct HostSlot {
    float *o_in = nullptr, *d_in = nullptr;  // uploaded rays
    uint32_t *payload_in = nullptr, *payload_sorted = nullptr;
    float *hits = nullptr;  // hits staged here, then copied back on the side stream
    cudaEvent_t rays_up = nullptr, pay_up = nullptr;  // upload stream: rays, payloads arrived
    cudaEvent_t consumed = nullptr;  // main stream: the reorder has read this slot's inputs
    cudaEvent_t traced = nullptr;    // main stream: the trace has written this slot's hits
    cudaEvent_t pay_down = nullptr;  // side stream: sorted payloads returned
    cudaEvent_t done = nullptr;      // side stream: hits returned (the slot's hits buffer is free)
};

struct rr_pipeline {
    const rr_bvh *bvh;
    uint32_t max_n;
    rr_key_params params;
    uint32_t radix_bits;
    size_t ws_bytes;
    unsigned char *mem;  // one allocation holding every buffer below
    void *workspace;
    void *keys;
    uint32_t *perm;
    float *o_sorted, *d_sorted;
    HostSlot slot[2];
    cudaStream_t upload = nullptr, side = nullptr;
    uint64_t submitted = 0;
};

namespace {
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

using namespace rr;

extern "C" rr_status rr_pipeline_create(const rr_bvh *bvh, uint32_t max_n, const rr_key_params *params,
                                        uint32_t radix_bits, rr_pipeline **out) {
    if (!out || !bvh || !params) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_create: NULL argument");
    *out = nullptr;
    if (max_n == 0) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_create: max_n is 0");
    if (params->bits < 1 || params->bits > 64 || params->layout > RR_KEY_OCTAHEDRON)
        return fail(RR_ERR_INVALID_ARG, "rr_pipeline_create: bad key params");
    size_t ws = 0;
    rr_status st = rr_sort_workspace_size(max_n, params->bits, radix_bits, &ws);
    if (st != RR_OK) return st;
    const size_t kb = params->bits > 32 ? 8 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = up256(off + bytes);
        return at;
    };
    const size_t o_ws = take(ws), o_keys = take(kb * max_n), o_perm = take(4ull * max_n);
    const size_t o_os = take(16ull * max_n), o_ds = take(16ull * max_n);
    size_t o_slot[2][5];
    for (auto &sl : o_slot) {
        sl[0] = take(16ull * max_n);  // o_in
        sl[1] = take(16ull * max_n);  // d_in
        sl[2] = take(4ull * max_n);   // payload_in
        sl[3] = take(4ull * max_n);   // payload_sorted
        sl[4] = take(16ull * max_n);  // hits
    }
    rr_pipeline *p = new rr_pipeline();
    cudaError_t e = lib_malloc(reinterpret_cast<void **>(&p->mem), off);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return fail(RR_ERR_OOM, "rr_pipeline_create: cudaMalloc failed");
    }
    p->bvh = bvh;
    p->max_n = max_n;
    p->params = *params;
    p->radix_bits = radix_bits;
    p->ws_bytes = ws;
    p->workspace = p->mem + o_ws;
    p->keys = p->mem + o_keys;
    p->perm = reinterpret_cast<uint32_t *>(p->mem + o_perm);
    p->o_sorted = reinterpret_cast<float *>(p->mem + o_os);
    p->d_sorted = reinterpret_cast<float *>(p->mem + o_ds);
    for (int k = 0; k < 2; ++k) {
        HostSlot &h = p->slot[k];
        h.o_in = reinterpret_cast<float *>(p->mem + o_slot[k][0]);
        h.d_in = reinterpret_cast<float *>(p->mem + o_slot[k][1]);
        h.payload_in = reinterpret_cast<uint32_t *>(p->mem + o_slot[k][2]);
        h.payload_sorted = reinterpret_cast<uint32_t *>(p->mem + o_slot[k][3]);
        h.hits = reinterpret_cast<float *>(p->mem + o_slot[k][4]);
    }
    e = cudaStreamCreateWithFlags(&p->upload, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    for (HostSlot &h : p->slot)
        for (cudaEvent_t *ev : {&h.rays_up, &h.pay_up, &h.consumed, &h.traced, &h.pay_down, &h.done})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rr_pipeline_destroy(p);
        return fail_cuda(e, "rr_pipeline_create: streams or events");
    }
    *out = p;
    return RR_OK;
}

extern "C" rr_status rr_pipeline_destroy(rr_pipeline *p) {
    if (!p) return RR_OK;
    for (HostSlot &h : p->slot)
        for (cudaEvent_t ev : {h.rays_up, h.pay_up, h.consumed, h.traced, h.pay_down, h.done})
            if (ev) cudaEventSynchronize(ev);
    for (HostSlot &h : p->slot)
        for (cudaEvent_t ev : {h.rays_up, h.pay_up, h.consumed, h.traced, h.pay_down, h.done})
            if (ev) cudaEventDestroy(ev);
    if (p->upload) cudaStreamDestroy(p->upload);
    if (p->side) cudaStreamDestroy(p->side);
    cudaFree(p->mem);
    delete p;
    return RR_OK;
}

namespace {

// Events that order one host submission's bounce with its uploads and
// downloads; all null for rr_pipeline_run.
struct BounceSync {
    cudaEvent_t rays_ready = nullptr;    // wait before the keys
    cudaEvent_t payload_ready = nullptr; // wait before the reorder
    cudaEvent_t payload_free = nullptr;  // wait before the reorder (previous reader of payload_out)
    cudaEvent_t consumed = nullptr;      // record after the reorder
    cudaEvent_t hits_free = nullptr;     // wait before the trace (previous reader of hits_out)
};

rr_status wait_on(cudaStream_t s, cudaEvent_t ev) {
    if (!ev) return RR_OK;
    const cudaError_t e = cudaStreamWaitEvent(s, ev, 0);
    return e == cudaSuccess ? RR_OK : fail_cuda(e, "rr_pipeline: stream wait");
}

// The bounce on device buffers, enqueued on `stream`.
rr_status run_bounce(rr_pipeline *p, const float *o_tmin, const float *d_tmax, const uint32_t *payload_in,
                     uint32_t n, float *hits_out, uint32_t *payload_out, void *stream, const BounceSync &sync) {
    cudaStream_t s = as_stream(stream);
    rr_status st = wait_on(s, sync.rays_ready);
    if (st == RR_OK)
        st = rr_key_sort(o_tmin, d_tmax, n, &p->params, p->keys, p->perm, p->radix_bits, p->workspace, p->ws_bytes,
                         stream);
    if (st == RR_OK) st = wait_on(s, sync.payload_ready);
    if (st == RR_OK) st = wait_on(s, sync.payload_free);
    if (st == RR_OK)
        st = rr_permute(o_tmin, d_tmax, payload_in, p->perm, n, p->o_sorted, p->d_sorted, payload_out, stream);
    if (st != RR_OK) return st;
    if (sync.consumed) {
        const cudaError_t e = cudaEventRecord(sync.consumed, s);
        if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline: record");
    }
    st = wait_on(s, sync.hits_free);
    if (st != RR_OK) return st;
    if (p->params.layout == RR_KEY_TWO_POINT && p->params.t_source == RR_T_ADAPTIVE)
        return rr_trace_accumulate(p->bvh, p->o_sorted, p->d_sorted, n, hits_out,
                                   const_cast<rr_length_table *>(p->params.table), stream);
    return rr_trace(p->bvh, p->o_sorted, p->d_sorted, n, hits_out, stream);
}

}  // namespace

extern "C" rr_status rr_pipeline_run(rr_pipeline *p, const float *o_tmin, const float *d_tmax,
                                     const uint32_t *payload_in, uint32_t n, float *hits_out,
                                     uint32_t *payload_out, void *stream) {
    if (!p) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run: NULL pipeline");
    if (n > p->max_n) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run: n exceeds max_n");
    if (n == 0) return RR_OK;
    if ((payload_in == nullptr) != (payload_out == nullptr))
        return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run: payload_in and payload_out must both be set or both NULL");
    return run_bounce(p, o_tmin, d_tmax, payload_in, n, hits_out, payload_out, stream, BounceSync{});
}

// Host buffers, without waiting.  Submission k uses staging slot k mod 2: its
// rays and payloads go up on the upload stream (after submission k-2 has
// read the slot), the bounce runs on `stream` with the hits staged in the
// slot (after submission k-2's hits have gone back), and the sorted payloads
// and the hits come back on the side stream while the next submission
// computes.
extern "C" rr_status rr_pipeline_submit_host(rr_pipeline *p, const float *o_host, const float *d_host,
                                             const uint32_t *payload_host, uint32_t n, float *hits_host,
                                             uint32_t *payload_out_host, void *stream, uint64_t *ticket) {
    if (!p) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_submit_host: NULL pipeline");
    if (ticket) *ticket = 0;
    if (n > p->max_n) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_submit_host: n exceeds max_n");
    if (n == 0) return RR_OK;
    if (!o_host || !d_host || !hits_host) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_submit_host: NULL buffer");
    if ((payload_host == nullptr) != (payload_out_host == nullptr))
        return fail(RR_ERR_INVALID_ARG, "rr_pipeline_submit_host: payload in/out must both be set or both NULL");
    cudaStream_t s = as_stream(stream);
    const uint64_t k = p->submitted++;
    HostSlot &h = p->slot[k & 1];
    const bool pay = payload_host != nullptr;
    // uploads: after the reorder of submission k-2 has read this slot
    cudaError_t e = cudaStreamWaitEvent(p->upload, h.consumed, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.o_in, o_host, 16ull * n, cudaMemcpyHostToDevice, p->upload);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.d_in, d_host, 16ull * n, cudaMemcpyHostToDevice, p->upload);
    if (e == cudaSuccess) e = cudaEventRecord(h.rays_up, p->upload);
    if (pay) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.payload_in, payload_host, 4ull * n, cudaMemcpyHostToDevice, p->upload);
        if (e == cudaSuccess) e = cudaEventRecord(h.pay_up, p->upload);
    }
    if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_submit_host: upload");
    BounceSync sync;
    sync.rays_ready = h.rays_up;
    sync.payload_ready = pay ? h.pay_up : nullptr;
    sync.payload_free = pay ? h.pay_down : nullptr;
    sync.consumed = h.consumed;
    sync.hits_free = h.done;
    rr_status st = run_bounce(p, h.o_in, h.d_in, pay ? h.payload_in : nullptr, n, h.hits,
                              pay ? h.payload_sorted : nullptr, stream, sync);
    if (st != RR_OK) return st;
    if (pay) {
        e = cudaStreamWaitEvent(p->side, h.consumed, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(payload_out_host, h.payload_sorted, 4ull * n, cudaMemcpyDeviceToHost, p->side);
    }
    // recorded for every submission, so that it also covers the payload
    // downloads of earlier submissions still running on the side stream
    if (e == cudaSuccess) e = cudaEventRecord(h.pay_down, p->side);
    // the hits come back on the side stream while the next submission computes
    if (e == cudaSuccess) e = cudaEventRecord(h.traced, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, h.traced, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hits_host, h.hits, 16ull * n, cudaMemcpyDeviceToHost, p->side);
    if (e == cudaSuccess) e = cudaEventRecord(h.done, p->side);
    if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_submit_host: download");
    if (ticket) *ticket = k + 1;
    return RR_OK;
}

extern "C" rr_status rr_pipeline_wait(rr_pipeline *p, uint64_t ticket) {
    if (!p) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_wait: NULL pipeline");
    if (ticket == 0) return RR_OK;  // an empty submission
    if (ticket > p->submitted) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_wait: ticket was never issued");
    if (fault_fires(Fault::Timeout)) return fail(RR_ERR_TIMEOUT, "rr_pipeline_wait: injected time-out");
    // a slot's events are re-recorded by later submissions; those complete
    // after this one, so waiting on them is never too early.  `done` and
    // `pay_down` follow every earlier download on the side stream, and each
    // hit download follows its own submission's trace.
    HostSlot &h = p->slot[(ticket - 1) & 1];
    cudaError_t e = cudaEventSynchronize(h.done);
    if (e == cudaSuccess) e = cudaEventSynchronize(h.pay_down);
    if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_wait");
    return RR_OK;
}

extern "C" rr_status rr_pipeline_run_host(rr_pipeline *p, const float *o_host, const float *d_host,
                                          const uint32_t *payload_host, uint32_t n, float *hits_host,
                                          uint32_t *payload_out_host, void *stream) {
    uint64_t ticket = 0;
    rr_status st = rr_pipeline_submit_host(p, o_host, d_host, payload_host, n, hits_host, payload_out_host, stream,
                                           &ticket);
    if (st != RR_OK) {
        if (p) {
            cudaStreamSynchronize(p->upload);
            cudaStreamSynchronize(p->side);
        }
        return st;
    }
    return rr_pipeline_wait(p, ticket);
}
