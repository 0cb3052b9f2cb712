// Device arithmetic of the sorting keys (Section 3.1, Figure 2).
//
// Every float operation is a correctly rounded binary32 intrinsic, so that the
// integer results (quantised coordinates, table cells, fixed-point lengths)
// do not depend on instruction selection (no multiply-add contraction).
#pragma once

#include <stdint.h>

namespace rr {

// x in [0,1] -> 32-bit cell by truncation; >= 1 -> all ones; <= 0 or NaN -> 0.
__device__ __forceinline__ uint32_t quantise_unit(float x) {
    if (!(x > 0.0f)) return 0u;
    if (x >= 1.0f) return 0xFFFFFFFFu;
    return __float2uint_rz(__fmul_rn(x, 4294967296.0f));  // times 2^32 is exact
}

struct QuantFrame {
    float lo[3];
    float inv[3];  // 1 / extent, or 0 for a flat axis
    float E;       // largest extent
};

__device__ __forceinline__ QuantFrame make_frame(const float lo[3], const float hi[3]) {
    QuantFrame f;
    float e = 0.0f;
    for (int c = 0; c < 3; ++c) {
        float ext = __fsub_rn(hi[c], lo[c]);
        f.lo[c] = lo[c];
        f.inv[c] = ext > 0.0f ? __fdiv_rn(1.0f, ext) : 0.0f;
        if (c == 0 || ext > e) e = ext;
    }
    f.E = e;
    return f;
}

__device__ __forceinline__ uint32_t quantise_coord(const QuantFrame &f, int c, float p) {
    return quantise_unit(__fmul_rn(__fsub_rn(p, f.lo[c]), f.inv[c]));
}

// |d| with the squares summed left to right.
__device__ __forceinline__ float length3(float x, float y, float z) {
    float s = __fmul_rn(x, x);
    s = __fadd_rn(s, __fmul_rn(y, y));
    s = __fadd_rn(s, __fmul_rn(z, z));
    return __fsqrt_rn(s);
}

// Spreads the low 11 bits of x so that bit i lands on bit 6i.
__host__ __device__ __forceinline__ uint64_t spread6(uint64_t x) {
    x &= 0x7FFull;
    x = (x | (x << 40)) & 0x00070000000000FFull;
    x = (x | (x << 20)) & 0x000700000F00000Full;
    x = (x | (x << 10)) & 0x1003003003003003ull;
    x = (x | (x << 5)) & 0x1041041041041041ull;
    return x;
}

// Spreads the low 3 bits of x so that bit i lands on bit 3i.
__host__ __device__ __forceinline__ uint32_t spread3_3(uint32_t x) {
    return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4);
}

// First 64 bits of the string whose level L (from the top) holds bit 31-L of
// c[0], c[1], ..., c[5] in that order (Aila with c[3..5] = q(d) >> 3, and Two
// Point with c[3..5] = q(p)).
__host__ __device__ __forceinline__ uint64_t interleave6_64(const uint32_t c[6]) {
    uint64_t hi = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) hi |= spread6(c[s] >> 22) << (5 - s);  // levels 0..9
    uint64_t tail = ((uint64_t)((c[0] >> 21) & 1u) << 3) | ((uint64_t)((c[1] >> 21) & 1u) << 2) |
                    ((uint64_t)((c[2] >> 21) & 1u) << 1) | (uint64_t)((c[3] >> 21) & 1u);
    return (hi << 4) | tail;  // level 10, first four slots
}

// The compact string: levels 0..2 carry only c[0..2] (the always-zero
// direction slots of the Aila string are dropped), later levels all six.
__host__ __device__ __forceinline__ uint64_t interleave_compact_64(const uint32_t c[6]) {
    uint32_t head = (spread3_3(c[0] >> 29) << 2) | (spread3_3(c[1] >> 29) << 1) |
                    spread3_3(c[2] >> 29);  // 9 bits, levels 0..2
    uint64_t body = 0;
#pragma unroll
    for (int s = 0; s < 6; ++s) body |= spread6((c[s] >> 20) & 0x1FFu) << (5 - s);  // levels 3..11
    return ((uint64_t)head << 55) | (body << 1) | (uint64_t)((c[0] >> 19) & 1u);  // + level 12, x
}

// Spreads the low 21 bits of x so that bit i lands on bit 3i.
__device__ __forceinline__ uint64_t spread3_21(uint64_t x) {
    x &= 0x1FFFFFull;
    x = (x | (x << 32)) & 0x1F00000000FFFFull;
    x = (x | (x << 16)) & 0x1F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// First 64 bits of the Morton string of three components (level L holds bit
// 31-L of c0, c1, c2): levels 0..20 and the first slot of level 21.
__device__ __forceinline__ uint64_t morton3_64(uint32_t c0, uint32_t c1, uint32_t c2) {
    const uint64_t m = (spread3_21(c0 >> 11) << 2) | (spread3_21(c1 >> 11) << 1) | spread3_21(c2 >> 11);
    return (m << 1) | ((c0 >> 10) & 1u);
}

// The first k bits of a 64-bit string (k = 0..64).
__device__ __forceinline__ uint64_t prefix64(uint64_t s, uint32_t k) { return k ? s >> (64 - k) : 0ull; }

// Spreads the low 10 bits of x so that bit i lands on bit 5i.
__device__ __forceinline__ uint64_t spread5_10(uint32_t x) {
    uint64_t r = 0;
#pragma unroll
    for (int i = 0; i < 10; ++i) r |= (uint64_t)((x >> i) & 1u) << (5 * i);
    return r;
}

// Octahedral parametrisation of a direction (Meyer et al. 2010) in [0,1]^2.
__device__ __forceinline__ void octahedral(float dx, float dy, float dz, float &u, float &v) {
    const float sum = __fadd_rn(__fadd_rn(fabsf(dx), fabsf(dy)), fabsf(dz));
    float px = 0.0f, py = 0.0f;
    if (sum > 0.0f) {
        px = __fdiv_rn(dx, sum);
        py = __fdiv_rn(dy, sum);
    }
    if (dz < 0.0f) {
        const float sx = px >= 0.0f ? 1.0f : -1.0f, sy = py >= 0.0f ? 1.0f : -1.0f;
        const float qx = __fmul_rn(__fsub_rn(1.0f, fabsf(py)), sx);
        const float qy = __fmul_rn(__fsub_rn(1.0f, fabsf(px)), sy);
        px = qx;
        py = qy;
    }
    u = __fmul_rn(__fadd_rn(px, 1.0f), 0.5f);
    v = __fmul_rn(__fadd_rn(py, 1.0f), 0.5f);
}

// Octahedron key string: levels 0..3 hold the origin only, later levels the
// origin and the two octahedral coordinates (c[3], c[4], each the quantised
// coordinate shifted right by 4).  First 64 bits: 12 + 5*10 + 2.
__device__ __forceinline__ uint64_t interleave_octa_64(const uint32_t c[5]) {
    const uint64_t head = (spread3_21(c[0] >> 28) << 2) | (spread3_21(c[1] >> 28) << 1) | spread3_21(c[2] >> 28);
    uint64_t body = 0;
#pragma unroll
    for (int s = 0; s < 5; ++s) body |= spread5_10((c[s] >> 18) & 0x3FFu) << (4 - s);  // levels 4..13
    return (head << 52) | (body << 2) | ((uint64_t)((c[0] >> 17) & 1u) << 1) | (uint64_t)((c[1] >> 17) & 1u);
}

// Quantised origin and direction of a ray (direction normalised, mapped to [0,1]).
__device__ __forceinline__ void quantise_ray(const QuantFrame &f, float4 o, float4 d, uint32_t qo[3],
                                             uint32_t qd[3], float dh[3]) {
    qo[0] = quantise_coord(f, 0, o.x);
    qo[1] = quantise_coord(f, 1, o.y);
    qo[2] = quantise_coord(f, 2, o.z);
    float len = length3(d.x, d.y, d.z);
    dh[0] = len > 0.0f ? __fdiv_rn(d.x, len) : 0.0f;
    dh[1] = len > 0.0f ? __fdiv_rn(d.y, len) : 0.0f;
    dh[2] = len > 0.0f ? __fdiv_rn(d.z, len) : 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) qd[c] = quantise_unit(__fmul_rn(__fadd_rn(dh[c], 1.0f), 0.5f));
}

// The frame of a box, computed once per block into shared memory by thread 0.
// Call from every thread of the block.
__device__ __forceinline__ QuantFrame block_frame(const float lo[3], const float hi[3]) {
    __shared__ QuantFrame s_frame;
    if (threadIdx.x == 0) s_frame = make_frame(lo, hi);
    __syncthreads();
    return s_frame;
}

// floor(sum / cnt) for cnt >= 1 and a quotient below 2^32: a float estimate,
// one refinement from the remainder, then exact integer correction of the
// remaining +-1 (instead of a 64-bit integer division).
__device__ __forceinline__ uint32_t div_floor_u64(unsigned long long sum, unsigned long long cnt) {
    const float inv = __frcp_rn(__ull2float_rn(cnt));
    long long q = (long long)(__ull2float_rn(sum) * inv);
    if (q < 0) q = 0;
    long long r = (long long)(sum - (unsigned long long)q * cnt);
    q += (long long)(__ll2float_rn(r) * inv);
    r = (long long)(sum - (unsigned long long)q * cnt);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (r < 0) {
            --q;
            r += (long long)cnt;
        } else if (r >= (long long)cnt) {
            ++q;
            r -= (long long)cnt;
        }
    }
    return (uint32_t)q;
}

// 20-bit compacted Aila code: the length-table cell (Section 3.1.6).  The
// first 20 bits of the compact string are o(12) d(3) o(3) d(2): levels 0..3
// of the origin, then the first direction level (bit 31 of each quantised
// direction, since the Aila direction is q >> 3), level 4 of the origin and
// the second direction level of x and y.
__host__ __device__ __forceinline__ uint32_t spread3_4(uint32_t x) {
    return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4) | ((x & 8u) << 6);
}
__host__ __device__ __forceinline__ uint32_t table_cell(const uint32_t qo[3], const uint32_t qd[3]) {
    const uint32_t o12 = (spread3_4(qo[0] >> 28) << 2) | (spread3_4(qo[1] >> 28) << 1) | spread3_4(qo[2] >> 28);
    const uint32_t d3 = ((qd[0] >> 31) << 2) | ((qd[1] >> 31) << 1) | (qd[2] >> 31);
    const uint32_t o3 = (((qo[0] >> 27) & 1u) << 2) | (((qo[1] >> 27) & 1u) << 1) | ((qo[2] >> 27) & 1u);
    const uint32_t d2 = (((qd[0] >> 30) & 1u) << 1) | ((qd[1] >> 30) & 1u);
    return (o12 << 8) | (d3 << 5) | (o3 << 2) | d2;
}

// Six-component interleave from a 64-entry table of 6-bit spreads (bit i of
// the index at bit 6i, values below 2^31), as interleave6_64 computes it: the
// first 30 bits of the string are levels 0..4 (bits 31..27 of every
// component), the next 34 bits levels 5..10 (bits 26..21) without the last
// two slots of level 10.
__host__ __device__ __forceinline__ uint32_t spread6_small(uint32_t x) {
    uint32_t r = 0;
    for (int i = 0; i < 6; ++i) r |= ((x >> i) & 1u) << (6 * i);
    return r;
}
__host__ __device__ __forceinline__ uint64_t interleave6_64_lut(const uint32_t c[6], const uint32_t *lut) {
    uint32_t P = 0;
    for (int s = 0; s < 6; ++s) P |= lut[c[s] >> 27] << (5 - s);
    uint32_t B[6];
    for (int s = 0; s < 6; ++s) B[s] = lut[(c[s] >> 21) & 63u];
    const uint32_t lo = (B[0] << 3) | (B[1] << 2) | (B[2] << 1) | B[3] | (B[4] >> 1) | (B[5] >> 2);
    const uint32_t hi = (P << 2) | ((B[0] >> 30) << 1) | (B[1] >> 30);
    return ((uint64_t)hi << 32) | lo;
}

// The table in shared memory, filled by the first 64 threads.  Call from
// every thread of the block.
__device__ __forceinline__ const uint32_t *block_spread6_lut() {
    __shared__ uint32_t s_lut[64];
    if (threadIdx.x < 64) s_lut[threadIdx.x] = spread6_small(threadIdx.x);
    return s_lut;
}

}  // namespace rr
