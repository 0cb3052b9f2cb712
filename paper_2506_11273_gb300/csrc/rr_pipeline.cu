// One bounce of the reordered path behind a single handle: keys -> sort ->
// reorder -> trace, then the length-table update when the Two Point key takes
// its estimate from the table (Section 3.1.6: accumulate after each trace).
#include "rr_common.cuh"

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
    uint32_t *payload_sorted;
    float *o_in, *d_in;  // staging for rr_pipeline_run_host
    uint32_t *payload_in;
    float *hits;
    // rr_pipeline_run_host moves the payloads on a side stream, overlapped
    // with the key, sort and trace kernels of the main stream
    cudaStream_t side = nullptr;
    cudaEvent_t rays_in = nullptr, payload_in_done = nullptr, sorted = nullptr, payload_out_done = nullptr;
};

namespace {
size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of `bytes` of page-locked host memory at `host`, or null when
// either end of the range is not page-locked, mapped host memory (pageable
// memory takes the copy path).  Kernels then store into it directly over the
// host link.
void *mapped_host(void *host, size_t bytes) {
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess ||
        cudaPointerGetAttributes(&b, static_cast<char *>(host) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<char *>(b.devicePointer) - static_cast<char *>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}
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
    const size_t o_ws = off;
    off = up256(off + ws);
    const size_t o_keys = off;
    off = up256(off + kb * max_n);
    const size_t o_perm = off;
    off = up256(off + 4ull * max_n);
    const size_t o_os = off;
    off = up256(off + 16ull * max_n);
    const size_t o_ds = off;
    off = up256(off + 16ull * max_n);
    const size_t o_ps = off;
    off = up256(off + 4ull * max_n);
    const size_t o_oi = off;
    off = up256(off + 16ull * max_n);
    const size_t o_di = off;
    off = up256(off + 16ull * max_n);
    const size_t o_pi = off;
    off = up256(off + 4ull * max_n);
    const size_t o_h = off;
    off = up256(off + 16ull * max_n);
    rr_pipeline *p = new rr_pipeline();
    cudaError_t e = cudaMalloc(&p->mem, off);
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
    p->payload_sorted = reinterpret_cast<uint32_t *>(p->mem + o_ps);
    p->o_in = reinterpret_cast<float *>(p->mem + o_oi);
    p->d_in = reinterpret_cast<float *>(p->mem + o_di);
    p->payload_in = reinterpret_cast<uint32_t *>(p->mem + o_pi);
    p->hits = reinterpret_cast<float *>(p->mem + o_h);
    e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&p->rays_in, &p->payload_in_done, &p->sorted, &p->payload_out_done})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        rr_pipeline_destroy(p);
        return fail_cuda(e, "rr_pipeline_create: stream or events");
    }
    *out = p;
    return RR_OK;
}

extern "C" rr_status rr_pipeline_destroy(rr_pipeline *p) {
    if (!p) return RR_OK;
    for (cudaEvent_t ev : {p->rays_in, p->payload_in_done, p->sorted, p->payload_out_done})
        if (ev) cudaEventDestroy(ev);
    if (p->side) cudaStreamDestroy(p->side);
    cudaFree(p->mem);
    delete p;
    return RR_OK;
}

namespace {

// The bounce on device buffers.  When `payload_ready` is set, the stream waits
// for it before the reorder (the only step that reads payloads); when `sorted`
// is set, it is recorded after the reorder.
rr_status run_bounce(rr_pipeline *p, const float *o_tmin, const float *d_tmax, const uint32_t *payload_in,
                     uint32_t n, float *hits_out, uint32_t *payload_out, void *stream, cudaEvent_t payload_ready,
                     cudaEvent_t sorted) {
    rr_status st = rr_compute_keys(o_tmin, d_tmax, n, &p->params, p->keys, stream);
    if (st != RR_OK) return st;
    st = rr_sort(p->keys, nullptr, p->perm, n, p->params.bits, p->radix_bits, p->workspace, p->ws_bytes, stream);
    if (st != RR_OK) return st;
    cudaStream_t s = as_stream(stream);
    if (payload_ready) {
        const cudaError_t e = cudaStreamWaitEvent(s, payload_ready, 0);
        if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_run_host: wait for payloads");
    }
    st = rr_permute(o_tmin, d_tmax, payload_in, p->perm, n, p->o_sorted, p->d_sorted, payload_out, stream);
    if (st != RR_OK) return st;
    if (sorted) {
        const cudaError_t e = cudaEventRecord(sorted, s);
        if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_run_host: record");
    }
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
    return run_bounce(p, o_tmin, d_tmax, payload_in, n, hits_out, payload_out, stream, nullptr, nullptr);
}

// Host buffers.  The rays go up first (the keys need them); the payloads go up
// on the side stream while the keys and the sort run, and come back on it
// while the trace runs.  Hits in page-locked host memory are stored there by
// the trace kernel itself, so their transfer overlaps the trace; otherwise
// they are staged on the device and copied back after it.
extern "C" rr_status rr_pipeline_run_host(rr_pipeline *p, const float *o_host, const float *d_host,
                                          const uint32_t *payload_host, uint32_t n, float *hits_host,
                                          uint32_t *payload_out_host, void *stream) {
    if (!p) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run_host: NULL pipeline");
    if (n > p->max_n) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run_host: n exceeds max_n");
    if (n == 0) return RR_OK;
    if (!o_host || !d_host || !hits_host) return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run_host: NULL buffer");
    if ((payload_host == nullptr) != (payload_out_host == nullptr))
        return fail(RR_ERR_INVALID_ARG, "rr_pipeline_run_host: payload in/out must both be set or both NULL");
    cudaStream_t s = as_stream(stream);
    const bool pay = payload_host != nullptr;
    float *hits_direct = static_cast<float *>(mapped_host(hits_host, 16ull * n));
    if (hits_direct && !aligned(hits_direct, 16)) hits_direct = nullptr;
    cudaError_t e = cudaMemcpyAsync(p->o_in, o_host, 16ull * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->d_in, d_host, 16ull * n, cudaMemcpyHostToDevice, s);
    if (pay) {
        if (e == cudaSuccess) e = cudaEventRecord(p->rays_in, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->rays_in, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(p->payload_in, payload_host, 4ull * n, cudaMemcpyHostToDevice, p->side);
        if (e == cudaSuccess) e = cudaEventRecord(p->payload_in_done, p->side);
    }
    if (e != cudaSuccess) return fail_cuda(e, "rr_pipeline_run_host: upload");
    rr_status st = run_bounce(p, p->o_in, p->d_in, pay ? p->payload_in : nullptr, n, hits_direct ? hits_direct : p->hits,
                              pay ? p->payload_sorted : nullptr, stream, pay ? p->payload_in_done : nullptr,
                              pay ? p->sorted : nullptr);
    if (st != RR_OK) {
        cudaStreamSynchronize(p->side);
        return st;
    }
    if (pay) {
        e = cudaStreamWaitEvent(p->side, p->sorted, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(payload_out_host, p->payload_sorted, 4ull * n, cudaMemcpyDeviceToHost, p->side);
        if (e == cudaSuccess) e = cudaEventRecord(p->payload_out_done, p->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->payload_out_done, 0);
    }
    if (e == cudaSuccess && !hits_direct) e = cudaMemcpyAsync(hits_host, p->hits, 16ull * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(p->side);
        return fail_cuda(e, "rr_pipeline_run_host: download");
    }
    return RR_OK;
}
