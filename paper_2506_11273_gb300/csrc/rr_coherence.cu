// Capsule coherence measure (Section 4.3): for every run of `subset`
// consecutive rays, the surface area of a capsule around their origins and
// termination points.  One warp per run, two rays per lane, fp32.
#include <cmath>

#include "rr_common.cuh"

namespace rr {

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

__global__ void __launch_bounds__(256) capsule_kernel(const float4 *__restrict__ o_tmin,
                                                     const float4 *__restrict__ d_tmax,
                                                     const float4 *__restrict__ hits, uint32_t n,
                                                     uint32_t subset, uint32_t groups, float E,
                                                     float *__restrict__ out) {
    const uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31u;
    if (g >= groups) return;  // warp-uniform
    const uint32_t m = n < subset ? n : subset;
    const uint32_t first = g * subset;
    float po[2][3], pt[2][3];
    bool use[2];
    float co[3] = {0.f, 0.f, 0.f}, ct[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const uint32_t k = lane + 32u * r;
        use[r] = k < m;
        if (use[r]) {
            const float4 o = __ldg(o_tmin + first + k), d = __ldg(d_tmax + first + k), h = __ldg(hits + first + k);
            const float len = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            const float inv = len > 0.f ? 1.0f / len : 0.f;
            float t = h.x;
            if (__float_as_uint(h.w) == kMiss || !isfinite(t)) t = 4.0f * E;
            po[r][0] = o.x; po[r][1] = o.y; po[r][2] = o.z;
            pt[r][0] = o.x + d.x * inv * t;
            pt[r][1] = o.y + d.y * inv * t;
            pt[r][2] = o.z + d.z * inv * t;
        } else {
            po[r][0] = po[r][1] = po[r][2] = 0.f;
            pt[r][0] = pt[r][1] = pt[r][2] = 0.f;
        }
    }
    const float invm = 1.0f / (float)m;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        co[c] = warp_sum(po[0][c] + po[1][c]) * invm;
        ct[c] = warp_sum(pt[0][c] + pt[1][c]) * invm;
    }
    const float ax = ct[0] - co[0], ay = ct[1] - co[1], az = ct[2] - co[2];
    const float a2 = ax * ax + ay * ay + az * az;
    float so = 0.f, st = 0.f;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (!use[r]) continue;
#pragma unroll
        for (int which = 0; which < 2; ++which) {
            const float *x = which == 0 ? po[r] : pt[r];
            const float vx = x[0] - co[0], vy = x[1] - co[1], vz = x[2] - co[2];
            const float proj = a2 > 0.f ? (vx * ax + vy * ay + vz * az) / a2 : 0.f;
            const float wx = vx - proj * ax, wy = vy - proj * ay, wz = vz - proj * az;
            const float dist = sqrtf(wx * wx + wy * wy + wz * wz);
            if (which == 0)
                so += dist;
            else
                st += dist;
        }
    }
    const float ro = warp_sum(so) * invm, rt = warp_sum(st) * invm;
    if (lane == 0) {
        const float pi = 3.14159265358979f;
        const float h2 = a2, dr = ro - rt;
        out[g] = 2.f * pi * ro * ro + 2.f * pi * rt * rt + pi * (ro + rt) * sqrtf(h2 + dr * dr);
    }
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_coherence_capsule(const float *o_tmin, const float *d_tmax, const float *hits, uint32_t n,
                                          uint32_t subset, float E, float *areas_out, void *stream) {
    if (subset < 1 || subset > 64) return fail(RR_ERR_INVALID_ARG, "rr_coherence_capsule: subset must be 1..64");
    if (!std::isfinite(E) || !(E > 0.0f)) return fail(RR_ERR_INVALID_ARG, "rr_coherence_capsule: E must be > 0");
    if (n == 0) return RR_OK;
    if (!o_tmin || !d_tmax || !hits || !areas_out) return fail(RR_ERR_INVALID_ARG, "rr_coherence_capsule: NULL buffer");
    if (!aligned16(o_tmin) || !aligned16(d_tmax) || !aligned16(hits) || !aligned(areas_out, 4))
        return fail(RR_ERR_INVALID_ARG, "rr_coherence_capsule: misaligned buffer");
    rr_status st;
    if (!device_state(&st)) return st;
    const uint32_t groups = n < subset ? 1u : n / subset;
    const uint32_t blocks = (groups * 32u + 255u) / 256u;
    capsule_kernel<<<blocks, 256, 0, as_stream(stream)>>>(
        reinterpret_cast<const float4 *>(o_tmin), reinterpret_cast<const float4 *>(d_tmax),
        reinterpret_cast<const float4 *>(hits), n, subset, groups, E, areas_out);
    note_launches(1);
    return check_launch("rr_coherence_capsule");
}
