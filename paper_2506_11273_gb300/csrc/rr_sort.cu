// Stable LSD radix sort of (key, index) pairs (Section 3.2), onesweep style:
// one upfront pass counts the digits of every pass; then each digit pass is a
// single kernel in which a tile counts its digits and publishes the counts,
// ranks its keys (peer masks from warp votes), resolves its global offsets by
// a decoupled look-back over the preceding tiles (pointer jumping over
// published spans), and scatters through shared memory so that global writes
// come out in runs.  Consecutive passes overlap launch and drain
// (programmatic dependent launch).
#include <algorithm>
#include <mutex>

#include "rr_batch.cuh"
#include "rr_common.cuh"

namespace rr {

// Look-back word of (tile t, digit d): ready bit | first tile s of the span it
// covers | count of digit d in tiles s..t.  A span starting at tile 0 is the
// inclusive prefix.
constexpr unsigned long long kReady = 1ull << 63;
constexpr uint32_t kSpinLimit = 1u << 20;   // bounded wait on a predecessor's word
constexpr int kSortBlock = 256;
constexpr int kSortWarps = kSortBlock / 32;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long lookback_word(uint32_t start, uint32_t count) {
    return kReady | ((unsigned long long)start << 32) | count;
}
__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Programmatic dependent launch: a pass lets the next kernel of its stream
// start its blocks once all of its own have started, and waits (before it
// touches global memory) until the kernel before it has finished and its
// writes are visible.  Both are no-ops for a kernel launched without the
// programmatic-serialisation attribute.
__device__ __forceinline__ void allow_dependent_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void wait_for_prerequisite() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename K>
struct SortTile;
template <>
struct SortTile<uint32_t> {
    static constexpr int kItems = 16;
};
template <>
struct SortTile<unsigned long long> {
    static constexpr int kItems = 12;
};

template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, uint32_t shift, uint32_t mask) {
    return (uint32_t)(k >> shift) & mask;
}

// Lanes of `among` whose digit equals this lane's digit: one warp vote per
// digit bit (votes are cheap; a match instruction per key is not).  Every lane
// of the warp must call it; lanes outside `among` get an unspecified result.
template <int RBITS>
__device__ __forceinline__ uint32_t digit_peers(uint32_t dg, uint32_t among) {
    uint32_t peers = among;
#pragma unroll
    for (int b = 0; b < RBITS; ++b) {
        const uint32_t bit = (dg >> b) & 1u;
        const uint32_t vote = __ballot_sync(0xFFFFFFFFu, bit);
        peers &= bit ? vote : ~vote;
    }
    return peers;
}

// Exclusive scan of one value per thread over the first `RADIX` threads
// (threads beyond contribute zero).  Called by every thread of the block.
template <int RADIX>
__device__ __forceinline__ uint32_t scan_digits(uint32_t v, uint32_t *s_warp) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (RADIX > 32) {
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        uint32_t add = 0;
        for (uint32_t w = 0; w < warp; ++w) add += s_warp[w];
        __syncthreads();
        x += add;
    }
    return x - v;
}

// ------------------------------------------------------------------ upfront histograms

// Counts the digits of every pass over all keys.  Plain shared atomics into
// two copies of the block's counters (even and odd warps): one atomic per key
// and pass, far fewer instructions than building warp peer masks.
template <typename K, int RBITS>
__global__ void __launch_bounds__(kSortBlock) sort_histogram_kernel(const K *__restrict__ keys, uint32_t n,
                                                                   uint32_t bits, uint32_t passes,
                                                                   uint32_t *__restrict__ hist,
                                                                   uint4 *__restrict__ zero_words,
                                                                   size_t zero_count, uint32_t *counters,
                                                                   uint32_t *zero_err) {
    constexpr int RADIX = 1 << RBITS;
    constexpr int PMAX = (64 + RBITS - 1) / RBITS;
    constexpr int KPT = 4;  // keys per thread per round
    __shared__ uint32_t sh[2][PMAX * RADIX];
    allow_dependent_launch();
    for (uint32_t i = threadIdx.x; i < 2 * PMAX * RADIX; i += kSortBlock) (&sh[0][0])[i] = 0;
    if (blockIdx.x == 0) {
        if (threadIdx.x < passes) counters[threadIdx.x] = 0u;  // tile counters of every pass
        if (threadIdx.x == 0 && zero_err) *zero_err = 0u;
    }
    __syncthreads();
    uint32_t *mine = sh[(threadIdx.x >> 5) & 1u];
    const uint32_t stride = gridDim.x * kSortBlock * KPT;
    for (uint32_t base = blockIdx.x * kSortBlock * KPT + threadIdx.x; base < n; base += stride) {
        K k[KPT];
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            const uint32_t i = base + q * kSortBlock;
            k[q] = i < n ? keys[i] : (K)0;
        }
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            if (base + q * kSortBlock < n) {
                K x = k[q];
                uint32_t left = bits;
                for (uint32_t p = 0; p < passes; ++p) {
                    const uint32_t nb = min((uint32_t)RBITS, left);
                    atomicAdd(&mine[p * RADIX + ((uint32_t)x & ((1u << nb) - 1u))], 1u);
                    x >>= RBITS;
                    left -= nb;
                }
            }
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < passes * RADIX; i += kSortBlock) {
        const uint32_t c = sh[0][i] + sh[1][i];
        if (c) atomicAdd(&hist[i], c);
    }
    // the look-back words of every pass start at zero
    for (size_t i = (size_t)blockIdx.x * kSortBlock + threadIdx.x; i < zero_count; i += (size_t)gridDim.x * kSortBlock)
        zero_words[i] = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------------ one digit pass

template <typename K>
struct PassArgs {
    const K *keys_in;
    const uint32_t *vals_in;  // null on the first pass: the value is the input index
    K *keys_out;              // null: keys are not written
    uint32_t *vals_out;
    uint32_t n;
    uint32_t shift;
    uint32_t mask;
    const uint32_t *hist;     // RADIX counts of this pass's digit over all keys
    unsigned long long *lookback;  // [tiles][RADIX] look-back words
    uint32_t *tile_counter;
    uint32_t *err;
};

// Shared-memory layout of one digit pass.
template <typename K, int RBITS>
struct PassSmem {
    static constexpr int RADIX = 1 << RBITS;
    static constexpr int TILE = kSortBlock * SortTile<K>::kItems;
    // keys [TILE] | values [TILE] | per-warp counters [warps][RADIX] | tile-local
    // digit starts [RADIX] | global base per digit [RADIX] | tile counts
    // [RADIX] | misc [16]: [0] tile id, [8..15] scan scratch
    static constexpr size_t bytes =
        sizeof(K) * TILE + sizeof(uint32_t) * (TILE + kSortWarps * RADIX + 3 * RADIX + 16);
};
static_assert(PassSmem<unsigned long long, 8>::bytes <= 48 * 1024 && PassSmem<uint32_t, 8>::bytes <= 48 * 1024,
              "a digit pass must fit the default dynamic shared-memory limit");

// One tile of a digit pass.  FULL tiles skip every bounds check; only the
// last tile of a pass can be partial.  LATE loads the values after the
// ranking (their loads then overlap the look-back), which keeps the ranking's
// registers low enough for four blocks per SM.
template <typename K, int RBITS, bool FULL, bool LATE>
__device__ __forceinline__ void onesweep_tile(const PassArgs<K> &a, uint32_t tile, unsigned char *smem) {
    constexpr int RADIX = 1 << RBITS;
    constexpr int ITEMS = SortTile<K>::kItems;
    constexpr int TILE = kSortBlock * ITEMS;
    constexpr int WTILE = 32 * ITEMS;
    K *s_keys = reinterpret_cast<K *>(smem);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + TILE);
    uint32_t *s_wh = s_vals + TILE;                  // [warps][RADIX]: counts, then prefix over warps
    uint32_t *s_lstart = s_wh + kSortWarps * RADIX;  // tile-local start of each digit
    uint32_t *s_gbase = s_lstart + RADIX;            // global position minus tile-local position
    uint32_t *s_cnt = s_gbase + RADIX;               // the tile's count of each digit
    uint32_t *s_misc = s_cnt + RADIX;

    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t base = tile * TILE;
    const uint32_t wbase = base + warp * WTILE;

    K k[ITEMS];
    uint32_t v[ITEMS], r[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        if (FULL || idx < a.n) {
            k[j] = a.keys_in[idx];
            if (!LATE) v[j] = a.vals_in ? a.vals_in[idx] : idx;
        } else {
            k[j] = 0;
            if (!LATE) v[j] = 0;
        }
    }
    // The tile's digit counts, published before the ranking so that later
    // tiles looking back wait on this tile's loads only, not on its ranking.
#pragma unroll
    for (int j = 0; j < ITEMS; ++j)
        if (FULL || wbase + j * 32 + lane < a.n) atomicAdd(&s_cnt[digit_of(k[j], a.shift, a.mask)], 1u);
    __syncthreads();
    const uint32_t cnt = tid < RADIX ? s_cnt[tid] : 0u;
    if (tid < RADIX) st_relaxed(a.lookback + (size_t)tile * RADIX + tid, lookback_word(tile, cnt));

    // stable rank inside the warp: items in index order (j, then lane).  The
    // peer masks of every row are independent; only the per-digit counters chain.
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t among = FULL ? 0xFFFFFFFFu : __ballot_sync(0xFFFFFFFFu, wbase + j * 32 + lane < a.n);
        r[j] = digit_peers<RBITS>(digit_of(k[j], a.shift, a.mask), among);
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const bool valid = FULL || wbase + j * 32 + lane < a.n;
        const uint32_t dg = digit_of(k[j], a.shift, a.mask);
        const uint32_t peers = r[j];
        const uint32_t cur = valid ? s_wh[warp * RADIX + dg] : 0u;
        __syncwarp();
        if (valid && lane == 31u - __clz(peers)) s_wh[warp * RADIX + dg] = cur + __popc(peers);
        __syncwarp();
        r[j] = cur + __popc(peers & lt);
    }
    __syncthreads();
    if (LATE) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t idx = wbase + j * 32 + lane;
            v[j] = (FULL || idx < a.n) ? (a.vals_in ? a.vals_in[idx] : idx) : 0u;
        }
    }

    // per digit: prefix over warps
    if (tid < RADIX) {
        uint32_t acc = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = s_wh[w * RADIX + tid];
            s_wh[w * RADIX + tid] = acc;
            acc += c;
        }
    }
    const uint32_t dstart = scan_digits<RADIX>(tid < RADIX ? a.hist[tid] : 0u, s_misc + 8);
    const uint32_t lstart = scan_digits<RADIX>(cnt, s_misc + 8);
    uint32_t excl = 0;
    if (tid < RADIX) {
        if (tile > 0) {
            // decoupled look-back by pointer jumping: add the span the nearest
            // uncovered predecessor has published and continue before its
            // start; republish the wider span so successors can jump over it.
            // Spans grow as tiles finish, so a tile needs few hops even when
            // every tile of the pass runs at the same time.
            uint32_t start = tile, sum = cnt, spins = 0;
            while (start > 0) {
                const unsigned long long w = ld_relaxed(a.lookback + (size_t)(start - 1) * RADIX + tid);
                if (!(w & kReady)) {
                    if (++spins > kSpinLimit) {
                        atomicOr(a.err, RR_DEVERR_LOOKBACK_TIMEOUT);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                sum += (uint32_t)w;
                start = (uint32_t)(w >> 32) & 0x7FFFFFFFu;
                st_relaxed(a.lookback + (size_t)tile * RADIX + tid, lookback_word(start, sum));
            }
            excl = sum - cnt;
        }
        s_lstart[tid] = lstart;
        s_gbase[tid] = dstart + excl - lstart;
    }
    __syncthreads();

    // scatter into shared memory in digit order (stable)
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        if (FULL || wbase + j * 32 + lane < a.n) {
            const uint32_t dg = digit_of(k[j], a.shift, a.mask);
            const uint32_t pos = s_lstart[dg] + s_wh[warp * RADIX + dg] + r[j];
            s_keys[pos] = k[j];
            s_vals[pos] = v[j];
        }
    }
    __syncthreads();
    // global writes in tile order: runs of equal digits land contiguously
    if (FULL) {
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t i = j * kSortBlock + tid;
            const K key = s_keys[i];
            const uint32_t gpos = s_gbase[digit_of(key, a.shift, a.mask)] + i;
            if (!index_ok(gpos, a.n, a.err)) continue;
            if (a.keys_out) a.keys_out[gpos] = key;
            a.vals_out[gpos] = s_vals[i];
        }
    } else {
        const uint32_t tile_n = min((uint32_t)TILE, a.n - base);
        for (uint32_t i = tid; i < tile_n; i += kSortBlock) {
            const K key = s_keys[i];
            const uint32_t gpos = s_gbase[digit_of(key, a.shift, a.mask)] + i;
            if (!index_ok(gpos, a.n, a.err)) continue;
            if (a.keys_out) a.keys_out[gpos] = key;
            a.vals_out[gpos] = s_vals[i];
        }
    }
}

// MINB blocks per SM: 3 for passes of one wave or less (shortest tile
// latency), 4 with late values for longer passes (more tiles in flight).
template <typename K, int RBITS, int MINB>
__global__ void __launch_bounds__(kSortBlock, MINB) onesweep_kernel(PassArgs<K> a) {
    using L = PassSmem<K, RBITS>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *s_wh = reinterpret_cast<uint32_t *>(smem_raw + sizeof(K) * L::TILE) + L::TILE;
    uint32_t *s_cnt = s_wh + kSortWarps * L::RADIX + 2 * L::RADIX;
    uint32_t *s_misc = s_cnt + L::RADIX;
    allow_dependent_launch();
    for (uint32_t i = threadIdx.x; i < kSortWarps * L::RADIX; i += kSortBlock) s_wh[i] = 0;
    for (uint32_t i = threadIdx.x; i < (uint32_t)L::RADIX; i += kSortBlock) s_cnt[i] = 0;
    wait_for_prerequisite();
    if (threadIdx.x == 0) s_misc[0] = atomicAdd(a.tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_misc[0];
    if ((tile + 1) * (uint32_t)L::TILE <= a.n)
        onesweep_tile<K, RBITS, true, (MINB > 3)>(a, tile, smem_raw);
    else
        onesweep_tile<K, RBITS, false, (MINB > 3)>(a, tile, smem_raw);
}

// ------------------------------------------------------------------ local (segment) sort

// One block sorts one segment of SEG = 256 * ITEMS consecutive keys entirely in
// shared memory: an LSD pass per 8-bit digit, each ranking the keys in
// position order (warp, item, lane) with the same warp-vote peer masks as the
// global passes, then scattering them back to shared memory.  The tail segment
// is padded with all-ones keys placed after the real keys, so stability keeps
// the padding last.  perm receives global indices.
template <typename K, int ITEMS>
__global__ void __launch_bounds__(kSortBlock) segment_sort_kernel(const K *__restrict__ keys_in,
                                                                 K *__restrict__ keys_out,
                                                                 uint32_t *__restrict__ perm_out, uint32_t n,
                                                                 uint32_t bits) {
    constexpr int RBITS = 8, RADIX = 256;
    constexpr int SEG = kSortBlock * ITEMS;
    constexpr int WSEG = 32 * ITEMS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K *s_keys = reinterpret_cast<K *>(smem_raw);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_keys + SEG);
    uint32_t *s_wh = s_vals + SEG;                 // [warps][RADIX]
    uint32_t *s_dstart = s_wh + kSortWarps * RADIX;  // [RADIX]
    uint32_t *s_scan = s_dstart + RADIX;           // scan scratch

    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t base = blockIdx.x * (uint32_t)SEG;
    const uint32_t m = min((uint32_t)SEG, n - base);
    const uint32_t lt = lanemask_lt();
    K k[ITEMS];
    uint32_t v[ITEMS], r[ITEMS];
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t pos = warp * WSEG + j * 32 + lane;
        k[j] = pos < m ? keys_in[base + pos] : ~(K)0;
        v[j] = pos;
    }
    const uint32_t passes = (bits + RBITS - 1) / RBITS;
    for (uint32_t p = 0; p < passes; ++p) {
        const uint32_t shift = p * RBITS;
        const uint32_t mask = (1u << min((uint32_t)RBITS, bits - shift)) - 1u;
        for (uint32_t i = tid; i < kSortWarps * RADIX; i += kSortBlock) s_wh[i] = 0;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) r[j] = digit_peers<RBITS>(digit_of(k[j], shift, mask), 0xFFFFFFFFu);
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t dg = digit_of(k[j], shift, mask);
            const uint32_t peers = r[j];
            const uint32_t cur = s_wh[warp * RADIX + dg];
            __syncwarp();
            if (lane == 31u - __clz(peers)) s_wh[warp * RADIX + dg] = cur + __popc(peers);
            __syncwarp();
            r[j] = cur + __popc(peers & lt);
        }
        __syncthreads();
        uint32_t cnt = 0;
        if (tid < RADIX) {
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_wh[w * RADIX + tid];
                s_wh[w * RADIX + tid] = cnt;
                cnt += c;
            }
        }
        const uint32_t start = scan_digits<RADIX>(cnt, s_scan);
        if (tid < RADIX) s_dstart[tid] = start;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t dg = digit_of(k[j], shift, mask);
            const uint32_t pos = s_dstart[dg] + s_wh[warp * RADIX + dg] + r[j];
            s_keys[pos] = k[j];
            s_vals[pos] = v[j];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < ITEMS; ++j) {
            const uint32_t pos = warp * WSEG + j * 32 + lane;
            k[j] = s_keys[pos];
            v[j] = s_vals[pos];
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < ITEMS; ++j) {
        const uint32_t pos = warp * WSEG + j * 32 + lane;
        if (pos < m) {
            perm_out[base + pos] = base + v[j];
            if (keys_out) keys_out[base + pos] = k[j];
        }
    }
}

template <typename K, int ITEMS>
static size_t segment_smem() {
    return (sizeof(K) + sizeof(uint32_t)) * kSortBlock * ITEMS + sizeof(uint32_t) * (kSortWarps * 256 + 256 + 16);
}

template <typename K, int ITEMS>
static cudaError_t launch_segment_sort(const K *keys_in, K *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                                       cudaStream_t s) {
    const size_t smem = segment_smem<K, ITEMS>();
    static bool configured = false;
    if (!configured) {
        const cudaError_t e = cudaFuncSetAttribute(segment_sort_kernel<K, ITEMS>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const uint32_t seg = kSortBlock * ITEMS;
    segment_sort_kernel<K, ITEMS><<<(n + seg - 1) / seg, kSortBlock, smem, s>>>(keys_in, keys_out, perm_out, n, bits);
    return cudaGetLastError();
}

template <typename K>
static cudaError_t dispatch_segment_sort(const K *ki, K *ko, uint32_t *perm, uint32_t n, uint32_t bits,
                                         uint32_t segment, cudaStream_t s) {
    switch (segment) {
        case 256: return launch_segment_sort<K, 1>(ki, ko, perm, n, bits, s);
        case 512: return launch_segment_sort<K, 2>(ki, ko, perm, n, bits, s);
        case 1024: return launch_segment_sort<K, 4>(ki, ko, perm, n, bits, s);
        case 2048: return launch_segment_sort<K, 8>(ki, ko, perm, n, bits, s);
        default: return launch_segment_sort<K, 16>(ki, ko, perm, n, bits, s);
    }
}

// ------------------------------------------------------------------ host side

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SortPlan {
    uint32_t passes, radix, tiles, kb;
    size_t off_hist, off_counters, off_lookback, off_keys_a, off_keys_b, off_vals, total;
};

// Workspace layout: digit counts [pass][radix], tile counters [pass],
// 64-bit look-back words [pass][tile][radix], two key buffers, one value buffer.
constexpr SortPlan plan_sort(uint32_t n, uint32_t bits, uint32_t radix_bits) {
    SortPlan p{};
    p.passes = (bits + radix_bits - 1) / radix_bits;
    p.radix = 1u << radix_bits;
    p.kb = bits > 32 ? 8u : 4u;
    const uint32_t tile = kSortBlock * (bits > 32 ? SortTile<unsigned long long>::kItems : SortTile<uint32_t>::kItems);
    p.tiles = (n + tile - 1) / tile;
    size_t off = 0;
    p.off_hist = off;
    off = align256(off + sizeof(uint32_t) * p.passes * p.radix);
    p.off_counters = off;
    off = align256(off + sizeof(uint32_t) * p.passes);
    p.off_lookback = off;
    off = align256(off + sizeof(unsigned long long) * (size_t)p.passes * p.tiles * p.radix);
    p.off_keys_a = off;
    off = align256(off + (size_t)p.kb * n);
    p.off_keys_b = off;
    off = align256(off + (size_t)p.kb * n);
    p.off_vals = off;
    off = align256(off + sizeof(uint32_t) * (size_t)n);
    p.total = off;
    return p;
}

template <typename K, int RBITS>
static size_t pass_smem() {
    return PassSmem<K, RBITS>::bytes;
}

// One digit pass, launched so that it may start while the kernel before it
// drains (programmatic dependent launch; the pass waits in the kernel).
// Passes of at least two waves at four blocks per SM take the four-block form.
template <typename K, int RBITS>
static cudaError_t launch_pass(const PassArgs<K> &a, uint32_t tiles, int sm_count, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(tiles);
    cfg.blockDim = dim3(kSortBlock);
    cfg.dynamicSmemBytes = pass_smem<K, RBITS>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (tiles >= 8u * (uint32_t)sm_count) return cudaLaunchKernelEx(&cfg, onesweep_kernel<K, RBITS, 4>, a);
    return cudaLaunchKernelEx(&cfg, onesweep_kernel<K, RBITS, 3>, a);
}

// The counting stage of a sort: the digit counts of every pass start at zero
// (a memset) and one counting kernel fills them, clearing the look-back words
// and tile counters.  zero_err (may be null) is a device word cleared too.
template <typename K, int RBITS>
static cudaError_t enqueue_count(const SortPlan &pl, const K *keys_in, uint32_t n, uint32_t bits, unsigned char *ws,
                                 uint32_t *zero_err, int sm_count, cudaStream_t s) {
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + pl.off_hist);
    uint32_t *counters = reinterpret_cast<uint32_t *>(ws + pl.off_counters);
    unsigned long long *lookback = reinterpret_cast<unsigned long long *>(ws + pl.off_lookback);
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * pl.passes * pl.radix, s);
    if (e != cudaSuccess) return e;
    const size_t zero_count = (size_t)pl.passes * pl.tiles * pl.radix / 2;  // uint4 = two words
    const uint32_t per_block = kSortBlock * 4u;
    // counting-pass grid: two blocks per SM up to ~2M keys, then one block per
    // 8 rounds of keys up to eight per SM (more blocks in flight hide the
    // loads; each block adds its counters to the global histogram once)
    const uint32_t sms = (uint32_t)sm_count;
    const uint32_t hist_blocks = std::max(
        1u, std::min({(n + per_block - 1) / per_block, std::max(2u * sms, n / (8u * per_block)), 8u * sms}));
    sort_histogram_kernel<K, RBITS><<<hist_blocks, kSortBlock, 0, s>>>(
        keys_in, n, bits, pl.passes, hist, reinterpret_cast<uint4 *>(lookback), zero_count, counters, zero_err);
    note_launches(1);
    return cudaGetLastError();
}

// The digit passes of a sort whose counting stage has run (by enqueue_count
// or fused into the key kernel): one onesweep kernel per pass.  Allocates
// nothing.
template <typename K, int RBITS>
static cudaError_t enqueue_passes(const SortPlan &pl, const K *keys_in, K *keys_out, uint32_t *perm_out,
                                  uint32_t n, uint32_t bits, unsigned char *ws, uint32_t *err, int sm_count,
                                  cudaStream_t s) {
    uint32_t *hist = reinterpret_cast<uint32_t *>(ws + pl.off_hist);
    uint32_t *counters = reinterpret_cast<uint32_t *>(ws + pl.off_counters);
    unsigned long long *lookback = reinterpret_cast<unsigned long long *>(ws + pl.off_lookback);
    K *keys_a = reinterpret_cast<K *>(ws + pl.off_keys_a);
    K *keys_b = reinterpret_cast<K *>(ws + pl.off_keys_b);
    uint32_t *vals_ws = reinterpret_cast<uint32_t *>(ws + pl.off_vals);
    const K *kin = keys_in;
    const uint32_t *vin = nullptr;
    for (uint32_t p = 0; p < pl.passes; ++p) {
        const bool final_slot = ((pl.passes - 1 - p) & 1u) == 0;
        K *kout;
        if (p == pl.passes - 1)
            kout = keys_out;
        else
            kout = final_slot ? (keys_out ? keys_out : keys_b) : keys_a;
        uint32_t *vout = final_slot ? perm_out : vals_ws;
        PassArgs<K> a;
        a.keys_in = kin;
        a.vals_in = vin;
        a.keys_out = kout;
        a.vals_out = vout;
        a.n = n;
        a.shift = p * RBITS;
        const uint32_t nb = std::min<uint32_t>(RBITS, bits - p * RBITS);
        a.mask = (1u << nb) - 1u;
        a.hist = hist + p * pl.radix;
        a.lookback = lookback + (size_t)p * pl.tiles * pl.radix;
        a.tile_counter = counters + p;
        a.err = err;
        const cudaError_t e = launch_pass<K, RBITS>(a, pl.tiles, sm_count, s);
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
    }
    note_launches(pl.passes);
    return cudaGetLastError();
}

// Enqueues the whole sort: counting stage, one kernel per digit pass.
// Allocates nothing.  zero_err (may be null) is a device word cleared
// before the passes run.
template <typename K, int RBITS>
static cudaError_t enqueue_sort(const SortPlan &pl, const K *keys_in, K *keys_out, uint32_t *perm_out,
                                uint32_t n, uint32_t bits, unsigned char *ws, uint32_t *err, uint32_t *zero_err,
                                int sm_count, cudaStream_t s) {
    const cudaError_t e = enqueue_count<K, RBITS>(pl, keys_in, n, bits, ws, zero_err, sm_count, s);
    if (e != cudaSuccess) return e;
    return enqueue_passes<K, RBITS>(pl, keys_in, keys_out, perm_out, n, bits, ws, err, sm_count, s);
}

template <typename K, int RBITS>
static rr_status run_sort(const SortPlan &pl, const K *keys_in, K *keys_out, uint32_t *perm_out, uint32_t n,
                          uint32_t bits, unsigned char *ws, uint32_t *err, int sm_count, cudaStream_t s) {
    const cudaError_t e = enqueue_sort<K, RBITS>(pl, keys_in, keys_out, perm_out, n, bits, ws, err, nullptr,
                                                 sm_count, s);
    if (e != cudaSuccess) return fail_cuda(e, "rr_sort");
    if (fault_fires(Fault::Launch)) return fail(RR_ERR_CUDA, "rr_sort: injected launch failure");
    return RR_OK;
}

// The sort of rr_sort (arguments already checked) with device errors going to
// `err`: batches captured on one stream and replayed on another report to the
// word of the stream they run on.
rr_status sort_enqueue(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                       uint32_t radix_bits, void *workspace, uint32_t *err, int sm_count, cudaStream_t s) {
    const SortPlan pl = plan_sort(n, bits, radix_bits);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    if (pl.kb == 4) {
        const uint32_t *ki = static_cast<const uint32_t *>(keys_in);
        uint32_t *ko = static_cast<uint32_t *>(keys_out);
        return radix_bits == 8 ? run_sort<uint32_t, 8>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s)
                               : run_sort<uint32_t, 4>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s);
    }
    const unsigned long long *ki = static_cast<const unsigned long long *>(keys_in);
    unsigned long long *ko = static_cast<unsigned long long *>(keys_out);
    return radix_bits == 8 ? run_sort<unsigned long long, 8>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s)
                           : run_sort<unsigned long long, 4>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s);
}

SortCountTarget sort_count_target(uint32_t n, uint32_t bits, uint32_t radix_bits, void *workspace) {
    const SortPlan pl = plan_sort(n, bits, radix_bits);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    SortCountTarget t;
    t.hist = reinterpret_cast<uint32_t *>(ws + pl.off_hist);
    t.counters = reinterpret_cast<uint32_t *>(ws + pl.off_counters);
    t.zero_words = reinterpret_cast<uint4 *>(ws + pl.off_lookback);
    t.zero_count = (size_t)pl.passes * pl.tiles * pl.radix / 2;
    t.passes = pl.passes;
    t.radix_bits = radix_bits;
    return t;
}

rr_status sort_enqueue_passes(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                              uint32_t radix_bits, void *workspace, uint32_t *err, int sm_count, cudaStream_t s) {
    const SortPlan pl = plan_sort(n, bits, radix_bits);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaError_t e;
    if (pl.kb == 4) {
        const uint32_t *ki = static_cast<const uint32_t *>(keys_in);
        uint32_t *ko = static_cast<uint32_t *>(keys_out);
        e = radix_bits == 8 ? enqueue_passes<uint32_t, 8>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s)
                            : enqueue_passes<uint32_t, 4>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s);
    } else {
        const unsigned long long *ki = static_cast<const unsigned long long *>(keys_in);
        unsigned long long *ko = static_cast<unsigned long long *>(keys_out);
        e = radix_bits == 8
                ? enqueue_passes<unsigned long long, 8>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s)
                : enqueue_passes<unsigned long long, 4>(pl, ki, ko, perm_out, n, bits, ws, err, sm_count, s);
    }
    if (e != cudaSuccess) return fail_cuda(e, "sort passes");
    if (fault_fires(Fault::Launch)) return fail(RR_ERR_CUDA, "sort passes: injected launch failure");
    return RR_OK;
}

rr_status sort_check(const char *what, const void *keys_in, const void *keys_out, const uint32_t *perm_out,
                     uint32_t n, uint32_t bits, uint32_t radix_bits, const void *workspace,
                     size_t workspace_bytes) {
    const std::string w(what);
    if (bits < 1 || bits > 64) return fail(RR_ERR_INVALID_ARG, w + ": bits not in 1..64");
    if (radix_bits != 4 && radix_bits != 8) return fail(RR_ERR_INVALID_ARG, w + ": radix_bits must be 4 or 8");
    if (n >= (1u << 30)) return fail(RR_ERR_INVALID_ARG, w + ": n must be < 2^30");
    if (n == 0) return RR_OK;
    if (!keys_in || !perm_out || !workspace) return fail(RR_ERR_INVALID_ARG, w + ": NULL buffer");
    const SortPlan pl = plan_sort(n, bits, radix_bits);
    if (workspace_bytes < pl.total) return fail(RR_ERR_INVALID_ARG, w + ": workspace too small");
    if (!aligned(workspace, 256)) return fail(RR_ERR_INVALID_ARG, w + ": workspace not 256-byte aligned");
    const size_t kbytes = (size_t)pl.kb * n;
    if (!aligned(keys_in, pl.kb) || (keys_out && !aligned(keys_out, pl.kb)) || !aligned(perm_out, 4))
        return fail(RR_ERR_INVALID_ARG, w + ": misaligned buffer");
    if (overlaps(keys_in, kbytes, perm_out, 4ull * n) ||
        (keys_out && (overlaps(keys_out, kbytes, keys_in, kbytes) || overlaps(keys_out, kbytes, perm_out, 4ull * n))) ||
        overlaps(workspace, pl.total, keys_in, kbytes) || overlaps(workspace, pl.total, perm_out, 4ull * n) ||
        (keys_out && overlaps(workspace, pl.total, keys_out, kbytes)))
        return fail(RR_ERR_INVALID_ARG, w + ": buffers overlap");
    return RR_OK;
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_sort_workspace_size(uint32_t n, uint32_t bits, uint32_t radix_bits, size_t *bytes) {
    if (!bytes) return fail(RR_ERR_INVALID_ARG, "rr_sort_workspace_size: bytes is NULL");
    if (bits < 1 || bits > 64) return fail(RR_ERR_INVALID_ARG, "rr_sort_workspace_size: bits not in 1..64");
    if (radix_bits != 4 && radix_bits != 8)
        return fail(RR_ERR_INVALID_ARG, "rr_sort_workspace_size: radix_bits must be 4 or 8");
    if (n >= (1u << 30)) return fail(RR_ERR_INVALID_ARG, "rr_sort_workspace_size: n must be < 2^30");
    *bytes = plan_sort(n, bits, radix_bits).total;
    return RR_OK;
}

extern "C" rr_status rr_sort(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                             uint32_t radix_bits, void *workspace, size_t workspace_bytes, void *stream) {
    rr_status st = sort_check("rr_sort", keys_in, keys_out, perm_out, n, bits, radix_bits, workspace, workspace_bytes);
    if (st != RR_OK || n == 0) return st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    cudaStream_t s = as_stream(stream);
    return sort_enqueue(keys_in, keys_out, perm_out, n, bits, radix_bits, workspace, error_word(ds, s),
                        ds->sm_count, s);
}

extern "C" rr_status rr_sort_segments(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n,
                                      uint32_t bits, uint32_t segment, void *stream) {
    if (bits < 1 || bits > 64) return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: bits not in 1..64");
    if (segment != 256 && segment != 512 && segment != 1024 && segment != 2048 && segment != 4096)
        return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: segment must be 256, 512, 1024, 2048 or 4096");
    if (n >= (1u << 30)) return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: n must be < 2^30");
    if (n == 0) return RR_OK;
    if (!keys_in || !perm_out) return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: NULL buffer");
    const size_t kb = bits > 32 ? 8 : 4, kbytes = kb * n;
    if (!aligned(keys_in, kb) || (keys_out && !aligned(keys_out, kb)) || !aligned(perm_out, 4))
        return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: misaligned buffer");
    if (overlaps(keys_in, kbytes, perm_out, 4ull * n) ||
        (keys_out && (overlaps(keys_out, kbytes, keys_in, kbytes) || overlaps(keys_out, kbytes, perm_out, 4ull * n))))
        return fail(RR_ERR_INVALID_ARG, "rr_sort_segments: buffers overlap");
    rr_status st;
    if (!device_state(&st)) return st;
    cudaStream_t s = as_stream(stream);
    const cudaError_t e =
        kb == 4 ? dispatch_segment_sort(static_cast<const uint32_t *>(keys_in), static_cast<uint32_t *>(keys_out),
                                        perm_out, n, bits, segment, s)
                : dispatch_segment_sort(static_cast<const unsigned long long *>(keys_in),
                                        static_cast<unsigned long long *>(keys_out), perm_out, n, bits, segment, s);
    if (e != cudaSuccess) return fail_cuda(e, "rr_sort_segments");
    note_launches(1);
    return RR_OK;
}

// ------------------------------------------------------------------ failure detection self-test
//
// One digit pass over two tiles of which only the second is launched: its
// look-back waits for the first tile's word, which nothing publishes, until
// the bounded spin gives up and records RR_DEVERR_LOOKBACK_TIMEOUT.  Without
// its predecessor's counts the tile scatters below its true offsets, which
// stay inside the output (all keys are zero: digit 0, positions 0..tile-1).

extern "C" rr_status rr_selftest_lookback_timeout(void *stream) {
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    using K = uint32_t;
    constexpr uint32_t tile = kSortBlock * SortTile<K>::kItems;
    const uint32_t n = 2 * tile;
    const SortPlan pl = plan_sort(n, 8, 8);
    unsigned char *ws = nullptr;
    K *keys = nullptr, *keys_out = nullptr;
    uint32_t *perm = nullptr;
    cudaError_t e = cudaMalloc(&ws, pl.total);
    if (e == cudaSuccess) e = cudaMalloc(&keys, sizeof(K) * n);
    if (e == cudaSuccess) e = cudaMalloc(&keys_out, sizeof(K) * n);
    if (e == cudaSuccess) e = cudaMalloc(&perm, sizeof(uint32_t) * n);
    cudaStream_t s = as_stream(stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws, 0, pl.total, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(keys, 0, sizeof(K) * n, s);
    const uint32_t one = 1u;  // the tile counter hands the only block tile 1
    uint32_t *counter = reinterpret_cast<uint32_t *>(ws + pl.off_counters);
    if (e == cudaSuccess) e = cudaMemcpyAsync(counter, &one, sizeof(one), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        PassArgs<K> a;
        a.keys_in = keys;
        a.vals_in = nullptr;
        a.keys_out = keys_out;
        a.vals_out = perm;
        a.n = n;
        a.shift = 0;
        a.mask = 0xFFu;
        a.hist = reinterpret_cast<const uint32_t *>(ws + pl.off_hist);
        a.lookback = reinterpret_cast<unsigned long long *>(ws + pl.off_lookback);
        a.tile_counter = counter;
        a.err = error_word(ds, s);
        onesweep_kernel<K, 8, 3><<<1, kSortBlock, pass_smem<K, 8>(), s>>>(a);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(ws);
    cudaFree(keys);
    cudaFree(keys_out);
    cudaFree(perm);
    if (e != cudaSuccess) return fail_cuda(e, "rr_selftest_lookback_timeout");
    return RR_OK;
}

// ------------------------------------------------------------------ sort without allocation
//
// rr_sort_noalloc: the same sort with its scratch in a file-scope device array
// instead of a caller-supplied workspace, for callers that cannot allocate
// device memory when they sort.  Nothing here allocates: not the array (it is
// part of the loaded module), not the per-device set-up, not the launches.

namespace rr {

constexpr size_t cx_max(size_t a, size_t b) { return a > b ? a : b; }

constexpr size_t kNoAllocHeader = 256;  // device error word of this entry point
constexpr size_t kNoAllocScratchBytes =
    kNoAllocHeader + cx_max(cx_max(plan_sort(RR_SORT_NOALLOC_MAX_N, 64, 8).total,
                                   plan_sort(RR_SORT_NOALLOC_MAX_N, 64, 4).total),
                            cx_max(plan_sort(RR_SORT_NOALLOC_MAX_N, 32, 8).total,
                                   plan_sort(RR_SORT_NOALLOC_MAX_N, 32, 4).total));
static_assert(kNoAllocScratchBytes <= RR_SORT_NOALLOC_SCRATCH_BYTES, "scratch bound in rr.h is too small");

static __device__ __align__(256) unsigned char g_sort_scratch[RR_SORT_NOALLOC_SCRATCH_BYTES];

struct NoAllocDevice {
    unsigned char *scratch = nullptr;  // device address of g_sort_scratch on this device
    int sm_count = 0;
};
constexpr int kNoAllocMaxDevices = 64;
static NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Per-device set-up, done by the first call on each device with that device
// current: look up the array's device address (host code may not use the
// symbol itself) and the SM count.
static rr_status noalloc_device(NoAllocDevice **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RR_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return RR_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocDevice &d = g_noalloc_dev[dev];
    if (d.scratch == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_sort_scratch) != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return RR_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            return RR_ERR_CUDA;
        }
        d.sm_count = sms;
        d.scratch = static_cast<unsigned char *>(p);
    }
    *out = &d;
    return RR_OK;
}

template <typename K, int RBITS>
static rr_status launch_sort_noalloc(const SortPlan &pl, const K *keys_in, K *keys_out, uint32_t *perm_out,
                                     uint32_t n, uint32_t bits, unsigned char *scratch, int sm_count,
                                     cudaStream_t s) {
    // the array keeps the last call's contents: the counting kernel clears the
    // tile counters and the look-back words before the passes.  The error word
    // at the head of the array is not cleared: its flags stay until
    // rr_device_error reads them (take_noalloc_error).
    uint32_t *err = reinterpret_cast<uint32_t *>(scratch);
    const cudaError_t e = enqueue_sort<K, RBITS>(pl, keys_in, keys_out, perm_out, n, bits, scratch + kNoAllocHeader,
                                                 err, nullptr, sm_count, s);
    return e == cudaSuccess ? RR_OK : RR_ERR_CUDA;
}

// Reads and clears the error word of rr_sort_noalloc on the current device
// (synchronous copies of four bytes; used by rr_device_error).
uint32_t take_noalloc_error() {
    uint32_t v = 0;
    const uint32_t zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_sort_scratch, sizeof(v), 0, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpyToSymbol(g_sort_scratch, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

}  // namespace rr

extern "C" rr_status rr_sort_noalloc(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n,
                                     uint32_t bits, uint32_t radix_bits, void *stream) {
    if (bits < 1 || bits > 64 || (radix_bits != 4 && radix_bits != 8)) return RR_ERR_INVALID_ARG;
    if (n > RR_SORT_NOALLOC_MAX_N) return RR_ERR_TOO_LARGE;
    if (n == 0) return RR_OK;
    if (!keys_in || !perm_out) return RR_ERR_INVALID_ARG;
    const SortPlan pl = plan_sort(n, bits, radix_bits);
    if (kNoAllocHeader + pl.total > sizeof(g_sort_scratch)) return RR_ERR_TOO_LARGE;
    const size_t kbytes = (size_t)pl.kb * n;
    if (!aligned(keys_in, pl.kb) || (keys_out && !aligned(keys_out, pl.kb)) || !aligned(perm_out, 4))
        return RR_ERR_INVALID_ARG;
    if (overlaps(keys_in, kbytes, perm_out, 4ull * n) ||
        (keys_out && (overlaps(keys_out, kbytes, keys_in, kbytes) || overlaps(keys_out, kbytes, perm_out, 4ull * n))))
        return RR_ERR_INVALID_ARG;
    NoAllocDevice *d = nullptr;
    const rr_status st = noalloc_device(&d);
    if (st != RR_OK) return st;
    cudaStream_t s = as_stream(stream);
    if (pl.kb == 4) {
        const uint32_t *ki = static_cast<const uint32_t *>(keys_in);
        uint32_t *ko = static_cast<uint32_t *>(keys_out);
        return radix_bits == 8 ? launch_sort_noalloc<uint32_t, 8>(pl, ki, ko, perm_out, n, bits, d->scratch, d->sm_count, s)
                               : launch_sort_noalloc<uint32_t, 4>(pl, ki, ko, perm_out, n, bits, d->scratch, d->sm_count, s);
    }
    const unsigned long long *ki = static_cast<const unsigned long long *>(keys_in);
    unsigned long long *ko = static_cast<unsigned long long *>(keys_out);
    return radix_bits == 8
               ? launch_sort_noalloc<unsigned long long, 8>(pl, ki, ko, perm_out, n, bits, d->scratch, d->sm_count, s)
               : launch_sort_noalloc<unsigned long long, 4>(pl, ki, ko, perm_out, n, bits, d->scratch, d->sm_count, s);
}
