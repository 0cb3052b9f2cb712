// The reorder pass of Section 3.2: rays are moved into sorted order.
// out[i] = in[perm[i]].  Reads of `in` are random (one 16-byte lane per field,
// i.e. half a sector); reads of perm and all writes are coalesced.
#include "rr_common.cuh"

namespace rr {

constexpr int kPermuteBlock = 256;
constexpr int kPermuteItems = 2;  // rays per thread: more loads in flight per thread

template <bool PAYLOAD>
__global__ void __launch_bounds__(kPermuteBlock) permute_kernel(const float4 *__restrict__ o_in,
                                                               const float4 *__restrict__ d_in,
                                                               const uint32_t *__restrict__ p_in,
                                                               const uint32_t *__restrict__ perm, uint32_t n,
                                                               float4 *__restrict__ o_out,
                                                               float4 *__restrict__ d_out,
                                                               uint32_t *__restrict__ p_out, uint32_t *err) {
    const uint32_t base = blockIdx.x * (kPermuteBlock * kPermuteItems) + threadIdx.x;
    uint32_t src[kPermuteItems];
#pragma unroll
    for (int j = 0; j < kPermuteItems; ++j) {
        const uint32_t i = base + j * kPermuteBlock;
        src[j] = i < n ? __ldcs(perm + i) : 0u;
    }
    float4 o[kPermuteItems], d[kPermuteItems];
    uint32_t p[kPermuteItems];
#pragma unroll
    for (int j = 0; j < kPermuteItems; ++j) {
        const uint32_t i = base + j * kPermuteBlock;
        if (i < n && index_ok(src[j], n, err)) {
            o[j] = __ldg(o_in + src[j]);
            d[j] = __ldg(d_in + src[j]);
            if (PAYLOAD) p[j] = __ldg(p_in + src[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < kPermuteItems; ++j) {
        const uint32_t i = base + j * kPermuteBlock;
        if (i < n && (!kChecked || src[j] < n)) {
            o_out[i] = o[j];
            d_out[i] = d[j];
            if (PAYLOAD) p_out[i] = p[j];
        }
    }
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_permute(const float *o_tmin_in, const float *d_tmax_in, const uint32_t *payload_in,
                                const uint32_t *perm, uint32_t n, float *o_tmin_out, float *d_tmax_out,
                                uint32_t *payload_out, void *stream) {
    if (n == 0) return RR_OK;
    if (!o_tmin_in || !d_tmax_in || !perm || !o_tmin_out || !d_tmax_out)
        return fail(RR_ERR_INVALID_ARG, "rr_permute: NULL buffer");
    if ((payload_in == nullptr) != (payload_out == nullptr))
        return fail(RR_ERR_INVALID_ARG, "rr_permute: payload_in and payload_out must both be set or both NULL");
    if (!aligned16(o_tmin_in) || !aligned16(d_tmax_in) || !aligned16(o_tmin_out) || !aligned16(d_tmax_out) ||
        !aligned(perm, 4) || (payload_in && (!aligned(payload_in, 4) || !aligned(payload_out, 4))))
        return fail(RR_ERR_INVALID_ARG, "rr_permute: misaligned buffer");
    const size_t rb = 16ull * n, pb = 4ull * n;
    if (overlaps(o_tmin_out, rb, o_tmin_in, rb) || overlaps(o_tmin_out, rb, d_tmax_in, rb) ||
        overlaps(d_tmax_out, rb, o_tmin_in, rb) || overlaps(d_tmax_out, rb, d_tmax_in, rb) ||
        overlaps(o_tmin_out, rb, d_tmax_out, rb) || overlaps(o_tmin_out, rb, perm, pb) ||
        overlaps(d_tmax_out, rb, perm, pb) ||
        (payload_in && (overlaps(payload_out, pb, payload_in, pb) || overlaps(payload_out, pb, perm, pb))))
        return fail(RR_ERR_INVALID_ARG, "rr_permute: buffers overlap");
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    const uint32_t per_block = kPermuteBlock * kPermuteItems;
    dim3 grid((n + per_block - 1) / per_block);
    cudaStream_t s = as_stream(stream);
    const float4 *oi = reinterpret_cast<const float4 *>(o_tmin_in);
    const float4 *di = reinterpret_cast<const float4 *>(d_tmax_in);
    float4 *oo = reinterpret_cast<float4 *>(o_tmin_out);
    float4 *dd = reinterpret_cast<float4 *>(d_tmax_out);
    uint32_t *err = error_word(ds, s);
    if (payload_in)
        permute_kernel<true><<<grid, kPermuteBlock, 0, s>>>(oi, di, payload_in, perm, n, oo, dd, payload_out, err);
    else
        permute_kernel<false><<<grid, kPermuteBlock, 0, s>>>(oi, di, nullptr, perm, n, oo, dd, nullptr, err);
    note_launches(1);
    return check_launch("rr_permute");
}
