// Sorting keys (Section 3.1, Figure 2) and the adaptive ray-length table
// (Section 3.1.6).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "rr_batch.cuh"
#include "rr_common.cuh"
#include "rr_keymath.cuh"
#include "rr_tma.cuh"

namespace rr {

struct KeyArgs {
    uint32_t *err;  // device error word
    const float4 *o_tmin;
    const float4 *d_tmax;
    uint32_t n;
    uint32_t bits;
    float lo[3], hi[3];
    float ratio;
    const float *t_given;
    const ulonglong2 *table;  // cells {sum, count}
    void *keys;
    SortCountTarget count;    // the fused form only: where the digit counts go
};

// The key of one ray (Section 3.1): the first `bits` bits of its layout's
// string, in the frame of the quantisation box.  t_given: the GIVEN estimate;
// table: the ADAPTIVE cells.
template <int LAYOUT, int TSRC>
__device__ __forceinline__ uint64_t ray_key(const QuantFrame &f, float4 o, float4 d, uint32_t bits, float ratio,
                                            float t_given, const ulonglong2 *table, const uint32_t *lut) {
    uint32_t qo[3], qd[3];
    float dh[3];
    quantise_ray(f, o, d, qo, qd, dh);
    uint64_t key64;
    if (LAYOUT == RR_KEY_TWO_POINT) {
        float t;
        if (TSRC == RR_T_FIXED) {
            t = __fmul_rn(ratio, f.E);
        } else if (TSRC == RR_T_GIVEN) {
            t = t_given;
        } else {
            // mean length of the ray's cell, in units of E / 2^24
            ulonglong2 cell = __ldg(table + table_cell(qo, qd));
            if (cell.y == 0ull) {
                t = __fmul_rn(0.25f, f.E);
            } else {
                const uint32_t mean = div_floor_u64(cell.x, cell.y);
                t = __fmul_rn(__fmul_rn(__uint2float_rn(mean), 5.9604644775390625e-8f), f.E);
            }
        }
        if (!isfinite(t)) t = __fmul_rn(4.0f, f.E);
        uint32_t c[6];
        c[0] = qo[0];
        c[1] = qo[1];
        c[2] = qo[2];
        c[3] = quantise_coord(f, 0, __fadd_rn(o.x, __fmul_rn(dh[0], t)));
        c[4] = quantise_coord(f, 1, __fadd_rn(o.y, __fmul_rn(dh[1], t)));
        c[5] = quantise_coord(f, 2, __fadd_rn(o.z, __fmul_rn(dh[2], t)));
        key64 = interleave6_64_lut(c, lut);
    } else if (LAYOUT == RR_KEY_AILA || LAYOUT == RR_KEY_AILA_COMPACT) {
        uint32_t c[6] = {qo[0], qo[1], qo[2], qd[0] >> 3, qd[1] >> 3, qd[2] >> 3};
        key64 = LAYOUT == RR_KEY_AILA ? interleave6_64_lut(c, lut) : interleave_compact_64(c);
    } else if (LAYOUT == RR_KEY_ORIGIN) {
        key64 = morton3_64(qo[0], qo[1], qo[2]);
    } else if (LAYOUT == RR_KEY_REIS || LAYOUT == RR_KEY_COSTA) {
        // two prefixes of their own Morton strings; the 32-bit split of Figure 2
        // (22 + 10 and 8 + 24) scaled to `bits`
        const uint32_t db = LAYOUT == RR_KEY_REIS ? (bits * 10u) / 32u : (bits * 8u) / 32u;
        const uint32_t ob = bits - db;
        const uint64_t ko = prefix64(morton3_64(qo[0], qo[1], qo[2]), ob);
        const uint64_t kd = prefix64(morton3_64(qd[0], qd[1], qd[2]), db);
        return LAYOUT == RR_KEY_REIS ? (db ? (ko << db) | kd : ko) : (ob ? (kd << ob) | ko : kd);
    } else {
        float u, v;
        octahedral(d.x, d.y, d.z, u, v);
        const uint32_t c[5] = {qo[0], qo[1], qo[2], quantise_unit(u) >> 4, quantise_unit(v) >> 4};
        key64 = interleave_octa_64(c);
    }
    return key64 >> (64 - bits);
}

// Persistent blocks walk over tiles of 256 rays.  Each tile's origins and
// directions arrive in shared memory by two bulk asynchronous copies completed
// on an mbarrier, issued one tile ahead into the other of two buffers, so the
// loads of the next tile overlap the key arithmetic of this one.  One ray per
// thread per tile: quantisation, interleave, one store.
constexpr int kKeyTile = 256;
constexpr uint32_t kCopySpinLimit = 1u << 22;  // polls of a copy's barrier before giving up

// Digit-count entries of the fused form: passes x 2^radix_bits <= 2048 for
// every key width with 4- or 8-bit digits.
constexpr int kCountEntries = 2048;

// COUNT (the fused key + sort form): each block also counts the digits of
// every sort pass of its keys (shared atomics into two copies, even and odd
// warps), adds its counts to the sort's digit counts once at the end, and
// clears the sort's look-back words and tile counters, so the separate
// counting kernel of the sort is not needed.
template <int LAYOUT, int TSRC, typename KeyT, bool COUNT>
__global__ void __launch_bounds__(kKeyTile, 6) key_kernel(KeyArgs a) {
    __shared__ __align__(128) float4 s_o[2][kKeyTile];
    __shared__ __align__(128) float4 s_d[2][kKeyTile];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_cnt[COUNT ? 2 : 1][COUNT ? kCountEntries : 1];
    const uint32_t tid = threadIdx.x;
    const uint32_t tiles = (a.n + kKeyTile - 1) / kKeyTile;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init_fence();
    }
    if (COUNT)
        for (uint32_t i = tid; i < 2u * kCountEntries; i += kKeyTile) (&s_cnt[0][0])[i] = 0u;
    const uint32_t *lut = block_spread6_lut();
    const QuantFrame f = block_frame(a.lo, a.hi);  // synchronises: barriers, counters and table published
    auto issue = [&](uint32_t t, uint32_t buf) {
        const uint32_t first = t * kKeyTile;
        const uint32_t bytes = min((uint32_t)kKeyTile, a.n - first) * (uint32_t)sizeof(float4);
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&s_bar[buf], 2 * bytes);
        bulk_copy_g2s(s_o[buf], a.o_tmin + first, bytes, &s_bar[buf]);
        bulk_copy_g2s(s_d[buf], a.d_tmax + first, bytes, &s_bar[buf]);
    };
    if (tid == 0 && blockIdx.x < tiles) issue(blockIdx.x, 0);
    uint32_t k = 0;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x, ++k) {
        const uint32_t buf = k & 1u, parity = (k >> 1) & 1u;
        const uint32_t next = t + gridDim.x;
        if (tid == 0 && next < tiles) issue(next, buf ^ 1u);
        const bool ok = mbar_wait_bounded(&s_bar[buf], parity, kCopySpinLimit);
        if (!__syncthreads_and(ok)) {
            // give up on this launch; let the copies in flight (the late one
            // into `buf` and the one already issued for the next tile) land
            // before the block's shared memory goes away
            if (tid == 0) {
                atomicOr(a.err, RR_DEVERR_COPY_TIMEOUT);
                mbar_wait_bounded(&s_bar[buf], parity, kCopySpinLimit);
                if (next < tiles) mbar_wait_bounded(&s_bar[buf ^ 1u], ((k + 1) >> 1) & 1u, kCopySpinLimit);
            }
            break;
        }
        const uint32_t i = t * kKeyTile + tid;
        if (i < a.n) {
            const float tg = TSRC == RR_T_GIVEN ? __ldg(a.t_given + i) : 0.0f;
            const KeyT key =
                (KeyT)ray_key<LAYOUT, TSRC>(f, s_o[buf][tid], s_d[buf][tid], a.bits, a.ratio, tg, a.table, lut);
            static_cast<KeyT *>(a.keys)[i] = key;
            if (COUNT) {
                // bits above a.bits are zero, so the last pass's digit needs no narrower mask
                uint32_t *mine = s_cnt[(tid >> 5) & 1u];
                const uint32_t rb = a.count.radix_bits, mask = (1u << rb) - 1u;
                KeyT x = key;
                for (uint32_t p = 0; p < a.count.passes; ++p) {
                    atomicAdd(&mine[(p << rb) + ((uint32_t)x & mask)], 1u);
                    x >>= rb;
                }
            }
        }
        __syncthreads();  // every thread is done with `buf` before it is refilled
    }
    if (COUNT) {
        __syncthreads();
        const uint32_t entries = a.count.passes << a.count.radix_bits;
        for (uint32_t i = tid; i < entries; i += kKeyTile) {
            const uint32_t c = s_cnt[0][i] + s_cnt[1][i];
            if (c) atomicAdd(a.count.hist + i, c);
        }
        if (blockIdx.x == 0 && tid < a.count.passes) a.count.counters[tid] = 0u;
        for (size_t w = (size_t)blockIdx.x * kKeyTile + tid; w < a.count.zero_count; w += (size_t)gridDim.x * kKeyTile)
            a.count.zero_words[w] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Batches: the key of ray i in the frame (and table) of its segment, with the
// segment number above the key's bits.
template <int LAYOUT, int TSRC, typename KeyT>
__global__ void __launch_bounds__(256) key_batch_kernel(const BatchScene *__restrict__ segs,
                                                        const uint32_t *__restrict__ seg_offsets, uint32_t n_segs,
                                                        const float4 *__restrict__ o_tmin,
                                                        const float4 *__restrict__ d_tmax, uint32_t n,
                                                        uint32_t bits, float ratio, KeyT *__restrict__ keys) {
    __shared__ uint32_t s_off[kMaxBatchSegments + 1];
    const uint32_t *lut = block_spread6_lut();
    for (uint32_t k = threadIdx.x; k <= n_segs; k += blockDim.x) s_off[k] = seg_offsets[k];
    __syncthreads();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t lo = 0, hi = n_segs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    const QuantFrame f = segs[lo].frame;
    const ulonglong2 *table = reinterpret_cast<const ulonglong2 *>(segs[lo].table);
    const uint64_t k =
        ray_key<LAYOUT, TSRC>(f, __ldg(o_tmin + i), __ldg(d_tmax + i), bits, ratio, 0.0f, table, lut);
    keys[i] = (KeyT)(((uint64_t)lo << bits) | k);
}

__global__ void batch_frame_kernel(BatchScene *segs, const float *boxes, uint32_t n) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const QuantFrame f = make_frame(boxes + 6 * k, boxes + 6 * k + 3);
    segs[k].frame = f;
    segs[k].invE = __fdiv_rn(1.0f, f.E);
}

// Blocks of one key-kernel variant that fit on the device at once (its
// occupancy is queried once per variant).
template <int LAYOUT, int TSRC, typename KeyT, bool COUNT>
static uint32_t key_grid(uint32_t tiles, int sm_count) {
    static int bps = 0;
    if (bps == 0) {
        int v = 0;
        const cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, key_kernel<LAYOUT, TSRC, KeyT, COUNT>, kKeyTile, 0);
        bps = (e == cudaSuccess && v > 0) ? v : 1;
    }
    return std::max(1u, std::min(tiles, (uint32_t)(sm_count * bps)));
}

template <int LAYOUT, int TSRC, bool COUNT>
static void launch_keys_t(const KeyArgs &a, bool wide, int sm_count, cudaStream_t s) {
    const uint32_t tiles = (a.n + kKeyTile - 1) / kKeyTile;
    if (wide)
        key_kernel<LAYOUT, TSRC, unsigned long long, COUNT>
            <<<key_grid<LAYOUT, TSRC, unsigned long long, COUNT>(tiles, sm_count), kKeyTile, 0, s>>>(a);
    else
        key_kernel<LAYOUT, TSRC, uint32_t, COUNT>
            <<<key_grid<LAYOUT, TSRC, uint32_t, COUNT>(tiles, sm_count), kKeyTile, 0, s>>>(a);
}

template <int LAYOUT, int TSRC>
static void launch_keys(const KeyArgs &a, bool wide, bool count, int sm_count, cudaStream_t s) {
    if (count)
        launch_keys_t<LAYOUT, TSRC, true>(a, wide, sm_count, s);
    else
        launch_keys_t<LAYOUT, TSRC, false>(a, wide, sm_count, s);
}

__global__ void table_init_kernel(ulonglong2 *cells) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kTableCells) cells[i] = make_ulonglong2(4194304ull /* 0.25 * 2^24 */, 1ull);
}

// After a trace: rays that hit add their fixed-point length to their cell.
// Lanes of a warp that share a cell combine first (match_any + warp reduce),
// then one lane issues the two 64-bit atomics.
__global__ void __launch_bounds__(256) table_accumulate_kernel(unsigned long long *cells, float lo0,
                                                               float lo1, float lo2, float hi0, float hi1,
                                                               float hi2, const float4 *o_tmin,
                                                               const float4 *d_tmax, const float4 *hits,
                                                               uint32_t n) {
    const float lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    const QuantFrame f = block_frame(lo, hi);
    const float invE = __fdiv_rn(1.0f, f.E);
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u;  // warp-uniform
    uint32_t i = base + lane;
    bool valid = false;
    uint32_t cell = 0, lq = 0;
    if (i < n) {
        float4 h = __ldg(hits + i);
        uint32_t tri = __float_as_uint(h.w);
        if (tri != kMiss && isfinite(h.x)) {
            float4 o = __ldg(o_tmin + i);
            float4 d = __ldg(d_tmax + i);
            uint32_t qo[3], qd[3];
            float dh[3];
            quantise_ray(f, o, d, qo, qd, dh);
            cell = table_cell(qo, qd);
            float len = __fmul_rn(h.x, length3(d.x, d.y, d.z));
            float x = __fmul_rn(len, invE);
            if (!(x > 0.0f)) x = 0.0f;
            if (x > 64.0f) x = 64.0f;
            lq = __float2uint_rz(__fmul_rn(x, 16777216.0f));
            valid = true;
        }
    }
    uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
    if (!valid) return;
    uint32_t peers = __match_any_sync(vmask, cell);
    uint32_t s_hi = __reduce_add_sync(peers, lq >> 16);
    uint32_t s_lo = __reduce_add_sync(peers, lq & 0xFFFFu);
    if (lane == (uint32_t)(__ffs(peers) - 1)) {
        unsigned long long sum = ((unsigned long long)s_hi << 16) + s_lo;
        atomicAdd(cells + 2 * (size_t)cell, sum);
        atomicAdd(cells + 2 * (size_t)cell + 1, (unsigned long long)__popc(peers));
    }
}

static bool box_ok(const float lo[3], const float hi[3]) {
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(lo[c]) || !std::isfinite(hi[c]) || !(lo[c] <= hi[c])) return false;
    return true;
}

static float largest_extent_host(const Box &b) {
    float e = b.hi[0] - b.lo[0];
    for (int c = 1; c < 3; ++c) {
        float x = b.hi[c] - b.lo[c];
        if (x > e) e = x;
    }
    return e;
}

cudaError_t launch_batch_frames(BatchScene *segs, const float *boxes, uint32_t n, cudaStream_t s) {
    batch_frame_kernel<<<(n + 127) / 128, 128, 0, s>>>(segs, boxes, n);
    note_launches(1);
    return cudaGetLastError();
}

template <int LAYOUT, int TSRC>
static void launch_keys_batch_t(const BatchScene *segs, const uint32_t *offs, uint32_t n_segs, const float4 *o,
                                const float4 *d, uint32_t n, uint32_t bits, float ratio, void *keys, bool wide,
                                cudaStream_t s) {
    dim3 grid((n + 255) / 256);
    if (wide)
        key_batch_kernel<LAYOUT, TSRC, unsigned long long><<<grid, 256, 0, s>>>(
            segs, offs, n_segs, o, d, n, bits, ratio, static_cast<unsigned long long *>(keys));
    else
        key_batch_kernel<LAYOUT, TSRC, uint32_t><<<grid, 256, 0, s>>>(segs, offs, n_segs, o, d, n, bits, ratio,
                                                                     static_cast<uint32_t *>(keys));
}

rr_status launch_keys_batch(const BatchScene *segs, const uint32_t *seg_offsets, uint32_t n_segs,
                            rr_key_layout layout, rr_t_source tsrc, float ratio, uint32_t key_bits,
                            uint32_t seg_bits, const float *o_tmin, const float *d_tmax, uint32_t n, void *keys,
                            cudaStream_t s) {
    if (n == 0) return RR_OK;
    const bool wide = key_bits + seg_bits > 32;
    const float4 *o = reinterpret_cast<const float4 *>(o_tmin);
    const float4 *d = reinterpret_cast<const float4 *>(d_tmax);
#define RR_KB(L, T) launch_keys_batch_t<L, T>(segs, seg_offsets, n_segs, o, d, n, key_bits, ratio, keys, wide, s)
    switch (layout) {
        case RR_KEY_AILA: RR_KB(RR_KEY_AILA, 0); break;
        case RR_KEY_AILA_COMPACT: RR_KB(RR_KEY_AILA_COMPACT, 0); break;
        case RR_KEY_ORIGIN: RR_KB(RR_KEY_ORIGIN, 0); break;
        case RR_KEY_REIS: RR_KB(RR_KEY_REIS, 0); break;
        case RR_KEY_COSTA: RR_KB(RR_KEY_COSTA, 0); break;
        case RR_KEY_OCTAHEDRON: RR_KB(RR_KEY_OCTAHEDRON, 0); break;
        default:
            if (tsrc == RR_T_ADAPTIVE)
                RR_KB(RR_KEY_TWO_POINT, RR_T_ADAPTIVE);
            else
                RR_KB(RR_KEY_TWO_POINT, RR_T_FIXED);
    }
#undef RR_KB
    note_launches(1);
    return check_launch("rr_batch keys");
}

}  // namespace rr

using namespace rr;

namespace {

// The checks of rr_compute_keys (and of the key half of rr_key_sort); fills
// the kernel arguments.  RR_OK with a->n == 0 means nothing to do.
rr_status key_setup(const char *what, const float *o_tmin, const float *d_tmax, uint32_t n, const rr_key_params *p,
                    void *keys_out, KeyArgs *a) {
    const std::string w(what);
    if (!p) return fail(RR_ERR_INVALID_ARG, w + ": params is NULL");
    if (p->layout > RR_KEY_OCTAHEDRON) return fail(RR_ERR_INVALID_ARG, w + ": bad layout");
    if (p->bits < 1 || p->bits > 64) return fail(RR_ERR_INVALID_ARG, w + ": bits not in 1..64");
    if (p->layout == RR_KEY_TWO_POINT && p->t_source > RR_T_GIVEN)
        return fail(RR_ERR_INVALID_ARG, w + ": bad t_source");
    if (!box_ok(p->aabb_lo, p->aabb_hi)) return fail(RR_ERR_INVALID_ARG, w + ": bad box");
    *a = KeyArgs{};
    if (n == 0) return RR_OK;
    if (!o_tmin || !d_tmax || !keys_out) return fail(RR_ERR_INVALID_ARG, w + ": NULL buffer");
    if (!aligned16(o_tmin) || !aligned16(d_tmax))
        return fail(RR_ERR_INVALID_ARG, w + ": rays not 16-byte aligned");
    const bool wide = p->bits > 32;
    if (!aligned(keys_out, wide ? 8 : 4)) return fail(RR_ERR_INVALID_ARG, w + ": keys misaligned");
    const size_t kbytes = (wide ? 8ull : 4ull) * n;
    if (overlaps(keys_out, kbytes, o_tmin, 16ull * n) || overlaps(keys_out, kbytes, d_tmax, 16ull * n))
        return fail(RR_ERR_INVALID_ARG, w + ": keys overlap the rays");
    if (p->layout == RR_KEY_TWO_POINT) {
        if (p->t_source == RR_T_FIXED && !std::isfinite(p->ratio))
            return fail(RR_ERR_INVALID_ARG, w + ": ratio not finite");
        if (p->t_source == RR_T_GIVEN && (!p->t_given || !aligned(p->t_given, 4)))
            return fail(RR_ERR_INVALID_ARG, w + ": t_given missing or misaligned");
        if (p->t_source == RR_T_ADAPTIVE) {
            const rr_length_table *t = p->table;
            if (!t) return fail(RR_ERR_INVALID_ARG, w + ": ADAPTIVE needs a table");
            if (std::memcmp(t->box.lo, p->aabb_lo, sizeof(float) * 3) ||
                std::memcmp(t->box.hi, p->aabb_hi, sizeof(float) * 3))
                return fail(RR_ERR_INVALID_ARG, w + ": table was created for another box");
            a->table = reinterpret_cast<const ulonglong2 *>(t->cells);
        }
    }
    a->o_tmin = reinterpret_cast<const float4 *>(o_tmin);
    a->d_tmax = reinterpret_cast<const float4 *>(d_tmax);
    a->n = n;
    a->bits = p->bits;
    for (int c = 0; c < 3; ++c) {
        a->lo[c] = p->aabb_lo[c];
        a->hi[c] = p->aabb_hi[c];
    }
    a->ratio = p->ratio;
    a->t_given = p->t_given;
    a->keys = keys_out;
    return RR_OK;
}

// Launches the key kernel of the params' layout and estimate.
void launch_layout(const rr_key_params *p, const KeyArgs &a, bool count, int sms, cudaStream_t s) {
    const bool wide = p->bits > 32;
    switch (p->layout) {
        case RR_KEY_AILA: launch_keys<RR_KEY_AILA, 0>(a, wide, count, sms, s); break;
        case RR_KEY_AILA_COMPACT: launch_keys<RR_KEY_AILA_COMPACT, 0>(a, wide, count, sms, s); break;
        case RR_KEY_ORIGIN: launch_keys<RR_KEY_ORIGIN, 0>(a, wide, count, sms, s); break;
        case RR_KEY_REIS: launch_keys<RR_KEY_REIS, 0>(a, wide, count, sms, s); break;
        case RR_KEY_COSTA: launch_keys<RR_KEY_COSTA, 0>(a, wide, count, sms, s); break;
        case RR_KEY_OCTAHEDRON: launch_keys<RR_KEY_OCTAHEDRON, 0>(a, wide, count, sms, s); break;
        default:
            if (p->t_source == RR_T_FIXED)
                launch_keys<RR_KEY_TWO_POINT, RR_T_FIXED>(a, wide, count, sms, s);
            else if (p->t_source == RR_T_GIVEN)
                launch_keys<RR_KEY_TWO_POINT, RR_T_GIVEN>(a, wide, count, sms, s);
            else
                launch_keys<RR_KEY_TWO_POINT, RR_T_ADAPTIVE>(a, wide, count, sms, s);
    }
}

}  // namespace

extern "C" rr_status rr_compute_keys(const float *o_tmin, const float *d_tmax, uint32_t n,
                                     const rr_key_params *p, void *keys_out, void *stream) {
    KeyArgs a;
    rr_status st = key_setup("rr_compute_keys", o_tmin, d_tmax, n, p, keys_out, &a);
    if (st != RR_OK || n == 0) return st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    cudaStream_t s = as_stream(stream);
    a.err = error_word(ds, s);
    launch_layout(p, a, false, ds->sm_count, s);
    note_launches(1);
    return check_launch("rr_compute_keys");
}

extern "C" rr_status rr_key_sort(const float *o_tmin, const float *d_tmax, uint32_t n, const rr_key_params *p,
                                 void *keys_out, uint32_t *perm_out, uint32_t radix_bits, void *workspace,
                                 size_t workspace_bytes, void *stream) {
    KeyArgs a;
    rr_status st = key_setup("rr_key_sort", o_tmin, d_tmax, n, p, keys_out, &a);
    if (st != RR_OK) return st;
    st = sort_check("rr_key_sort", keys_out, nullptr, perm_out, n, p->bits, radix_bits, workspace, workspace_bytes);
    if (st != RR_OK || n == 0) return st;
    if (overlaps(perm_out, 4ull * n, o_tmin, 16ull * n) || overlaps(perm_out, 4ull * n, d_tmax, 16ull * n) ||
        overlaps(workspace, workspace_bytes, o_tmin, 16ull * n) || overlaps(workspace, workspace_bytes, d_tmax, 16ull * n))
        return fail(RR_ERR_INVALID_ARG, "rr_key_sort: buffers overlap the rays");
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    cudaStream_t s = as_stream(stream);
    a.err = error_word(ds, s);
    a.count = sort_count_target(n, p->bits, radix_bits, workspace);
    const cudaError_t e = cudaMemsetAsync(a.count.hist, 0, sizeof(uint32_t) * (a.count.passes << radix_bits), s);
    if (e != cudaSuccess) return fail_cuda(e, "rr_key_sort: memset");
    launch_layout(p, a, true, ds->sm_count, s);
    note_launches(1);
    st = check_launch("rr_key_sort");
    if (st != RR_OK) return st;
    return sort_enqueue_passes(keys_out, nullptr, perm_out, n, p->bits, radix_bits, workspace, a.err, ds->sm_count, s);
}

extern "C" rr_status rr_length_table_create(const float lo[3], const float hi[3], rr_length_table **out,
                                            void *stream) {
    if (!out || !lo || !hi) return fail(RR_ERR_INVALID_ARG, "rr_length_table_create: NULL argument");
    *out = nullptr;
    if (!box_ok(lo, hi)) return fail(RR_ERR_INVALID_ARG, "rr_length_table_create: bad box");
    rr_status st;
    if (!device_state(&st)) return st;
    rr_length_table *t = new rr_length_table();
    cudaGetDevice(&t->device);
    for (int c = 0; c < 3; ++c) {
        t->box.lo[c] = lo[c];
        t->box.hi[c] = hi[c];
    }
    t->E = largest_extent_host(t->box);
    if (!(t->E > 0.0f)) {
        delete t;
        return fail(RR_ERR_INVALID_ARG, "rr_length_table_create: box has zero extent");
    }
    cudaError_t e = lib_malloc(reinterpret_cast<void **>(&t->cells), sizeof(unsigned long long) * 2 * kTableCells);
    if (e != cudaSuccess) {
        delete t;
        cudaGetLastError();
        return fail(RR_ERR_OOM, "rr_length_table_create: cudaMalloc failed");
    }
    *out = t;
    return rr_length_table_reset(t, stream);
}

extern "C" rr_status rr_length_table_reset(rr_length_table *t, void *stream) {
    if (!t) return fail(RR_ERR_INVALID_ARG, "rr_length_table_reset: NULL table");
    table_init_kernel<<<kTableCells / 256, 256, 0, as_stream(stream)>>>(reinterpret_cast<ulonglong2 *>(t->cells));
    note_launches(1);
    return check_launch("rr_length_table_reset");
}

extern "C" rr_status rr_length_table_accumulate(rr_length_table *t, const float *o_tmin, const float *d_tmax,
                                                const float *hits, uint32_t n, void *stream) {
    if (!t) return fail(RR_ERR_INVALID_ARG, "rr_length_table_accumulate: NULL table");
    if (n == 0) return RR_OK;
    if (!o_tmin || !d_tmax || !hits) return fail(RR_ERR_INVALID_ARG, "rr_length_table_accumulate: NULL buffer");
    if (!aligned16(o_tmin) || !aligned16(d_tmax) || !aligned16(hits))
        return fail(RR_ERR_INVALID_ARG, "rr_length_table_accumulate: buffers not 16-byte aligned");
    dim3 grid((n + 255) / 256);
    table_accumulate_kernel<<<grid, 256, 0, as_stream(stream)>>>(
        t->cells, t->box.lo[0], t->box.lo[1], t->box.lo[2], t->box.hi[0], t->box.hi[1], t->box.hi[2],
        reinterpret_cast<const float4 *>(o_tmin), reinterpret_cast<const float4 *>(d_tmax),
        reinterpret_cast<const float4 *>(hits), n);
    note_launches(1);
    return check_launch("rr_length_table_accumulate");
}

extern "C" rr_status rr_length_table_read(const rr_length_table *t, uint64_t *sum_host, uint32_t *cnt_host) {
    if (!t || !sum_host || !cnt_host) return fail(RR_ERR_INVALID_ARG, "rr_length_table_read: NULL argument");
    unsigned long long *tmp = new (std::nothrow) unsigned long long[2 * (size_t)kTableCells];
    if (!tmp) return fail(RR_ERR_OOM, "rr_length_table_read: host allocation failed");
    cudaError_t e = cudaMemcpy(tmp, t->cells, sizeof(unsigned long long) * 2 * kTableCells, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] tmp;
        return fail_cuda(e, "rr_length_table_read");
    }
    for (uint32_t i = 0; i < kTableCells; ++i) {
        sum_host[i] = tmp[2 * (size_t)i];
        cnt_host[i] = (uint32_t)tmp[2 * (size_t)i + 1];
    }
    delete[] tmp;
    return RR_OK;
}

extern "C" rr_status rr_length_table_write(rr_length_table *t, const uint64_t *sum_host, const uint32_t *cnt_host) {
    if (!t || !sum_host || !cnt_host) return fail(RR_ERR_INVALID_ARG, "rr_length_table_write: NULL argument");
    unsigned long long *tmp = new (std::nothrow) unsigned long long[2 * (size_t)kTableCells];
    if (!tmp) return fail(RR_ERR_OOM, "rr_length_table_write: host allocation failed");
    for (uint32_t i = 0; i < kTableCells; ++i) {
        tmp[2 * (size_t)i] = sum_host[i];
        tmp[2 * (size_t)i + 1] = cnt_host[i];
    }
    cudaError_t e = cudaMemcpy(t->cells, tmp, sizeof(unsigned long long) * 2 * kTableCells, cudaMemcpyHostToDevice);
    delete[] tmp;
    if (e != cudaSuccess) return fail_cuda(e, "rr_length_table_write");
    return RR_OK;
}

extern "C" rr_status rr_length_table_destroy(rr_length_table *t) {
    if (!t) return RR_OK;
    cudaFree(t->cells);
    delete t;
    return RR_OK;
}
