// Closest-hit traversal of the compressed 8-wide BVH.
//
// Persistent warps take batches of consecutive rays from a global queue, so
// which rays share a warp is decided by the order of the ray buffer: the
// coherence that reordering is meant to create (Section 4.2 measures its
// effect on control-flow and cache efficiency).  Each thread walks the
// compressed 8-wide BVH with a stack of node groups (the hit children of a
// node that remain to be visited, in the near-to-far order given by the ray's
// direction octant); the leaves a node's children hit are tested at once.
// Triangles are intersected with Moller-Trumbore in fp32 and the winning
// distance is refined in compensated fp32.
//
// Two variants serve the reordering study: indirect access (the queue hands
// out positions of an index buffer, so sorted rays are traced without being
// gathered first, Section 4.4.1) and any-hit traversal for shadow rays (the first
// triangle found inside the interval ends the ray, Section 4).
#include <chrono>
#include <cmath>

#include "rr_batch.cuh"
#include "rr_common.cuh"
#include "rr_keymath.cuh"
#include "rr_trace.h"

namespace rr {

constexpr int kTraceBlock = 128;

// The BVH arrays of one scene.
struct SceneRef {
    const float4 *nodes;   // RRNode8 as five float4
    const float4 *tris;    // RRTri as three float4
    const float4 *planes;  // two float4 per triangle: normal hi.xyz, lo.x | lo.y, lo.z
    uint32_t n_nodes;
    uint32_t n_tris;
};

struct TraceArgs {
    SceneRef scene;  // single-scene kernels
    const float4 *o_tmin;
    const float4 *d_tmax;
    float4 *hits;
    const uint32_t *order;  // NULL: position k traces ray k; else ray order[k]
    uint32_t n;
    uint32_t *queue;  // [0] next ray, [1] finished blocks
    uint32_t *err;
    unsigned long long *table;  // length-table cells {sum, count} (accumulating kernel only)
    float tlo[3], thi[3];       // the table's box
    // batches: ray i belongs to the segment s with seg_offsets[s] <= i < seg_offsets[s + 1]
    const BatchScene *segs;
    const uint32_t *seg_offsets;
    uint32_t n_segs;
};

__device__ __forceinline__ float safe_inv(float x) {
    const float m = fabsf(x) > 1e-18f ? x : copysignf(1e-18f, x);
    return __frcp_rn(m);
}

// Error-free transformations (Knuth's TwoSum, FMA-based TwoProd).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Distance along the ray to the plane of BVH-ordered triangle k, evaluated in
// compensated fp32: t = ((v0 - o) . n) / (d . n) with n the triangle normal
// stored as hi + lo floats and v0 - o split exactly into hi + lo.  Plain fp32
// loses relative accuracy when the hit is close to the origin compared with
// |v0 - o|; this form keeps it at a few ulps.
__device__ __forceinline__ float refine_t(const SceneRef &a, uint32_t k, float4 o, float4 d) {
    const float4 v0 = __ldg(a.tris + 3 * (size_t)k);
    const float4 p0 = __ldg(a.planes + 2 * (size_t)k), p1 = __ldg(a.planes + 2 * (size_t)k + 1);
    const float nh[3] = {p0.x, p0.y, p0.z}, nl[3] = {p0.w, p1.x, p1.y};
    const float vo[3] = {v0.x, v0.y, v0.z}, oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
    float num_hi = 0.0f, num_lo = 0.0f, den_hi = 0.0f, den_lo = 0.0f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float w, wl, p, pe, s, se;
        two_sum(vo[c], -oo[c], w, wl);  // v0 - o exactly
        two_prod(w, nh[c], p, pe);
        two_sum(num_hi, p, s, se);
        num_hi = s;
        num_lo = __fadd_rn(num_lo, __fadd_rn(__fadd_rn(se, pe), __fmaf_rn(w, nl[c], __fmul_rn(wl, nh[c]))));
        two_prod(dd[c], nh[c], p, pe);
        two_sum(den_hi, p, s, se);
        den_hi = s;
        den_lo = __fadd_rn(den_lo, __fadd_rn(__fadd_rn(se, pe), __fmul_rn(dd[c], nl[c])));
    }
    return __fdiv_rn(__fadd_rn(num_hi, num_lo), __fadd_rn(den_hi, den_lo));
}

// Byte k of a 32-bit word as the float 2^23 + byte: one byte permute puts the
// byte in the mantissa of 2^23 (no integer-to-float conversion).
template <int K>
__device__ __forceinline__ float byte_plus_2p23(uint32_t w) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, (uint32_t)K | 0x7540u));
}

// Traversal state of the ray a lane is tracing.  Node groups (child base,
// remaining hit mask in the near-to-far order of the ray's direction octant,
// inner-child mask) are the stack entries: one push per level descended.
struct RayState {
    float4 o, d;
    float idx, idy, idz;
    uint32_t negmask;
    float best, bu, bv;
    uint32_t best_tri, best_k;
    uint32_t g_base, g_hits, g_imask;
    uint32_t t_base, t_hits, t_all;  // pending triangle group: base, bits to test, node's tribits
    int sp;
};

__device__ __forceinline__ void ray_begin(RayState &r, const SceneRef &a, float4 o, float4 d) {
    r.o = o;
    r.d = d;
    r.idx = safe_inv(d.x);
    r.idy = safe_inv(d.y);
    r.idz = safe_inv(d.z);
    r.negmask = (r.idx < 0.0f ? 1u : 0u) | (r.idy < 0.0f ? 2u : 0u) | (r.idz < 0.0f ? 4u : 0u);
    r.best = d.w;
    r.bu = 0.0f;
    r.bv = 0.0f;
    r.best_tri = kMiss;
    r.best_k = 0u;
    // the current node group starts as a virtual group holding only the root
    r.g_base = 0u;
    r.g_hits = (a.n_nodes > 0 && o.w <= d.w) ? 1u : 0u;
    r.g_imask = 1u << r.negmask;
    r.t_base = 0u;
    r.t_hits = 0u;
    r.t_all = 0u;
    r.sp = 0;
}

// Stack entries are node groups: (child base, remaining hit mask in octant
// order | inner-child mask << 8).

__device__ __forceinline__ float max3f(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Node part of a traversal round: visit the nearest node of the current group
// (its hit inner children become the current group, its hit leaves the
// pending triangle group).
__device__ __forceinline__ bool ray_visit_node(RayState &r, uint2 *stack, const SceneRef &a, uint32_t *err) {
    const float tmin = r.o.w;
    const uint32_t pos = __ffs(r.g_hits) - 1u;
    r.g_hits &= r.g_hits - 1u;
    const uint32_t slot = pos ^ r.negmask;
    const uint32_t node = r.g_base + __popc(r.g_imask & ((1u << slot) - 1u));
    if (!index_ok(node, a.n_nodes, err)) {  // checked build: end the ray as a miss
        r.best_tri = kMiss;
        r.g_hits = 0u;
        r.t_hits = 0u;
        r.sp = 0;
        return true;
    }
    if (r.g_hits != 0u) {
        if (r.sp >= (int)kTraceStack) return false;
        stack[r.sp++] = make_uint2(r.g_base, r.g_hits | (r.g_imask << 8));
    }
    const float4 *np = a.nodes + 5 * (size_t)node;
    const float4 f0 = __ldg(np), f1 = __ldg(np + 1), f2 = __ldg(np + 2), f3 = __ldg(np + 3), f4 = __ldg(np + 4);
    const uint32_t ew = __float_as_uint(f0.w);
    const float sx = __uint_as_float((ew & 0xFFu) << 23);
    const float sy = __uint_as_float(((ew >> 8) & 0xFFu) << 23);
    const float sz = __uint_as_float(((ew >> 16) & 0xFFu) << 23);
    // plane of quantised value q: t = q*b + a.  The byte arrives as 2^23 + q, so
    // the offset moves into a: a' = a - 2^23*b.  Rounding a' costs at most half
    // a quantisation step, and every stored box is one step larger than the
    // child it bounds.
    const float bx = sx * r.idx, by = sy * r.idy, bz = sz * r.idz;
    const float ax = fmaf(-8388608.0f, bx, (f0.x - r.o.x) * r.idx);
    const float ay = fmaf(-8388608.0f, by, (f0.y - r.o.y) * r.idy);
    const float az = fmaf(-8388608.0f, bz, (f0.z - r.o.z) * r.idz);
    uint32_t nxl = __float_as_uint(f2.x), nxh = __float_as_uint(f2.y);
    uint32_t nyl = __float_as_uint(f2.z), nyh = __float_as_uint(f2.w);
    uint32_t nzl = __float_as_uint(f3.x), nzh = __float_as_uint(f3.y);
    uint32_t fxl = __float_as_uint(f3.z), fxh = __float_as_uint(f3.w);
    uint32_t fyl = __float_as_uint(f4.x), fyh = __float_as_uint(f4.y);
    uint32_t fzl = __float_as_uint(f4.z), fzh = __float_as_uint(f4.w);
    // for a negative direction the near plane is the box's high side
    if (r.negmask & 1u) {
        const uint32_t t0 = nxl, t1 = nxh;
        nxl = fxl; nxh = fxh; fxl = t0; fxh = t1;
    }
    if (r.negmask & 2u) {
        const uint32_t t0 = nyl, t1 = nyh;
        nyl = fyl; nyh = fyh; fyl = t0; fyh = t1;
    }
    if (r.negmask & 4u) {
        const uint32_t t0 = nzl, t1 = nzh;
        nzl = fzl; nzh = fzh; fzl = t0; fzh = t1;
    }
    uint32_t hm = 0u;  // slot s: the ray meets the child's box within [tmin, best]
    const float best = r.best;
#define RR_SLOT(S)                                                                                      \
    {                                                                                                   \
        const uint32_t w_nx = (S) < 4 ? nxl : nxh, w_ny = (S) < 4 ? nyl : nyh, w_nz = (S) < 4 ? nzl : nzh; \
        const uint32_t w_fx = (S) < 4 ? fxl : fxh, w_fy = (S) < 4 ? fyl : fyh, w_fz = (S) < 4 ? fzl : fzh; \
        const float t0 = max3f(fmaf(byte_plus_2p23<(S) & 3>(w_nx), bx, ax),                              \
                               fmaf(byte_plus_2p23<(S) & 3>(w_ny), by, ay),                              \
                               fmaxf(fmaf(byte_plus_2p23<(S) & 3>(w_nz), bz, az), tmin));                \
        const float t1 = min3f(fmaf(byte_plus_2p23<(S) & 3>(w_fx), bx, ax),                              \
                               fmaf(byte_plus_2p23<(S) & 3>(w_fy), by, ay),                              \
                               fminf(fmaf(byte_plus_2p23<(S) & 3>(w_fz), bz, az), best));                \
        if (t0 <= t1) hm |= 1u << (S);                                                                  \
    }
    RR_SLOT(0) RR_SLOT(1) RR_SLOT(2) RR_SLOT(3) RR_SLOT(4) RR_SLOT(5) RR_SLOT(6) RR_SLOT(7)
#undef RR_SLOT
    const uint32_t imask = (ew >> 24) & 0xFFu, tribits = __float_as_uint(f1.z);
    hm &= __float_as_uint(f1.w);  // used slots only
    // inner children to octant positions: bit s -> bit s ^ negmask
    uint32_t hits = hm & imask;
    if (r.negmask & 1u) hits = ((hits & 0x55u) << 1) | ((hits >> 1) & 0x55u);
    if (r.negmask & 2u) hits = ((hits & 0x33u) << 2) | ((hits >> 2) & 0x33u);
    if (r.negmask & 4u) hits = ((hits & 0x0Fu) << 4) | (hits >> 4);
    // leaves: slot bit s -> nibble s, keeping the triangles the nibble holds
    uint32_t x = hm & ~imask;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    const uint32_t tris = (x * 15u) & tribits;
    r.g_base = __float_as_uint(f1.x);
    r.g_hits = hits;
    r.g_imask = imask;
    r.t_base = __float_as_uint(f1.y);
    r.t_hits = tris;
    r.t_all = tribits;
    return true;
}

// Tests the nearest-slot triangle of the pending group (one triangle per
// traversal step).  ANY: a hit ends the ray (the pending group, the current
// node group and the stack are dropped).
template <bool ANY>
__device__ __forceinline__ void test_one_triangle(RayState &r, const SceneRef &a, uint32_t *err) {
    const float tmin = r.o.w;
    const uint32_t b = __ffs(r.t_hits) - 1u;
    r.t_hits &= r.t_hits - 1u;
    const uint32_t k = r.t_base + __popc(r.t_all & ((1u << b) - 1u));
    if (!index_ok(k, a.n_tris, err)) return;
    const float4 *tp = a.tris + 3 * (size_t)k;
    const float4 v0 = __ldg(tp), e1 = __ldg(tp + 1), e2 = __ldg(tp + 2);
    const float4 d = r.d, o = r.o;
    const float pvx = d.y * e2.z - d.z * e2.y;
    const float pvy = d.z * e2.x - d.x * e2.z;
    const float pvz = d.x * e2.y - d.y * e2.x;
    const float det = e1.x * pvx + e1.y * pvy + e1.z * pvz;
    if (det == 0.0f) return;
    const float inv = __frcp_rn(det);
    const float tvx = o.x - v0.x, tvy = o.y - v0.y, tvz = o.z - v0.z;
    const float u = (tvx * pvx + tvy * pvy + tvz * pvz) * inv;
    if (!(u >= 0.0f && u <= 1.0f)) return;
    const float qvx = tvy * e1.z - tvz * e1.y;
    const float qvy = tvz * e1.x - tvx * e1.z;
    const float qvz = tvx * e1.y - tvy * e1.x;
    const float v = (d.x * qvx + d.y * qvy + d.z * qvz) * inv;
    if (!(v >= 0.0f && u + v <= 1.0f)) return;
    const float t = (e2.x * qvx + e2.y * qvy + e2.z * qvz) * inv;
    if (t > tmin && t < r.best) {
        r.best = t;
        r.bu = u;
        r.bv = v;
        r.best_tri = __float_as_uint(v0.w);
        r.best_k = k;
        if (ANY) {
            r.t_hits = 0u;
            r.g_hits = 0u;
            r.sp = 0;
        }
    }
}

__device__ __forceinline__ float4 ray_result(const RayState &r, const SceneRef &a) {
    if (r.best_tri == kMiss) return make_float4(__int_as_float(0x7f800000), 0.0f, 0.0f, __uint_as_float(kMiss));
    const float tr = refine_t(a, r.best_k, r.o, r.d);
    return make_float4(isfinite(tr) ? tr : r.best, r.bu, r.bv, __uint_as_float(r.best_tri));
}

// The length-table update of one traced ray (Section 3.1.6), the arithmetic of
// table_accumulate_kernel: a ray that hit adds trunc(clamp(t*|d|/E, 0, 64)*2^24)
// and one count to the cell of its 20-bit compacted Aila code.
__device__ __forceinline__ void accumulate_hit(unsigned long long *table, const QuantFrame &f, float invE,
                                               float4 o, float4 d, float4 h) {
    if (__float_as_uint(h.w) == kMiss || !isfinite(h.x)) return;
    uint32_t qo[3], qd[3];
    float dh[3];
    quantise_ray(f, o, d, qo, qd, dh);
    const uint32_t cell = table_cell(qo, qd);
    float x = __fmul_rn(__fmul_rn(h.x, length3(d.x, d.y, d.z)), invE);
    if (!(x > 0.0f)) x = 0.0f;
    if (x > 64.0f) x = 64.0f;
    atomicAdd(table + 2 * (size_t)cell, (unsigned long long)__float2uint_rz(__fmul_rn(x, 16777216.0f)));
    atomicAdd(table + 2 * (size_t)cell + 1, 1ull);
}

// One traversal step of a lane's ray: test one pending triangle, or (after
// popping the next node group when the current one is used up) visit one
// node.  Returns false once the ray is finished.  A stack that would
// overflow records RR_DEVERR_TRACE_STACK and ends the ray as a miss.
template <bool ANY>
__device__ __forceinline__ bool ray_step(RayState &r, uint2 *stack, const SceneRef &sc, uint32_t *err) {
    if (r.t_hits != 0u) {
        test_one_triangle<ANY>(r, sc, err);
        return true;
    }
    if (r.g_hits == 0u) {
        if (r.sp == 0) return false;
        const uint2 e = stack[--r.sp];
        r.g_base = e.x;
        r.g_hits = e.y & 0xFFu;
        r.g_imask = (e.y >> 8) & 0xFFu;
    }
    if (!ray_visit_node(r, stack, sc, err)) {
        atomicOr(err, RR_DEVERR_TRACE_STACK);
        r.best_tri = kMiss;
        r.g_hits = 0u;
        r.t_hits = 0u;
        r.sp = 0;
    }
    return true;
}

// Lanes refill from the queue once this many of a warp's 32 lanes are idle
// (their rays finished): finished lanes write their hits together and idle
// lanes take consecutive queue positions together.
constexpr uint32_t kRefillLanes = 8;

// Resident blocks asked of the compiler: 36 warps per SM (nine 128-thread
// blocks at 56 registers; the step loop keeps the ray's state and the refill
// bookkeeping without spills).  Larger blocks round down to 32 warps.
template <int BLOCK>
constexpr int trace_min_blocks() {
    return 1152 / BLOCK > 0 ? 1152 / BLOCK : 1;
}

// Dynamic shared memory of the batch kernels: the scene of every segment, then
// the segment offsets.
inline size_t multi_smem(uint32_t n_segs) { return sizeof(SceneRef) * n_segs + sizeof(uint32_t) * (n_segs + 1); }

// MULTI: rays of several scenes in one launch (a batch); each lane finds the
// segment of its ray when it takes the ray and traces that segment's BVH
// (and updates its table).  The segments' scenes sit in shared memory, so a
// lane keeps only its segment number in registers during traversal.
//
// Each lane traces its own ray, one traversal step (a node or a triangle) per
// loop iteration, so a warp spends an iteration on triangle tests only for as
// long as some lane has a triangle left, and lanes whose ray has finished are
// refilled from the queue (kRefillLanes at a time) instead of idling until the
// warp's slowest ray is done.
template <bool ACCUM, bool ANY, bool MULTI, int BLOCK>
__global__ void __launch_bounds__(BLOCK, (trace_min_blocks<BLOCK>())) trace_kernel(TraceArgs a) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    SceneRef *s_sc = reinterpret_cast<SceneRef *>(s_dyn);
    uint32_t *s_off = reinterpret_cast<uint32_t *>(s_sc + (MULTI ? a.n_segs : 0));
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t lanes_below = (1u << lane) - 1u;
    // the table's quantisation frame is the same for the whole launch: it lives
    // in shared memory, not in every thread's registers during traversal
    __shared__ QuantFrame s_frame;
    __shared__ float s_invE;
    uint2 stack[kTraceStack];
    if (ACCUM && !MULTI && threadIdx.x == 0) {
        s_frame = make_frame(a.tlo, a.thi);
        s_invE = __fdiv_rn(1.0f, s_frame.E);
    }
    if (MULTI) {
        for (uint32_t k = threadIdx.x; k <= a.n_segs; k += BLOCK) s_off[k] = a.seg_offsets[k];
        for (uint32_t k = threadIdx.x; k < a.n_segs; k += BLOCK) {
            const BatchScene *bs = a.segs + k;
            s_sc[k].nodes = bs->nodes;
            s_sc[k].tris = bs->tris;
            s_sc[k].planes = bs->planes;
            s_sc[k].n_nodes = bs->n_nodes;
            s_sc[k].n_tris = bs->n_tris;
        }
    }
    if (MULTI || ACCUM) __syncthreads();
    RayState r;
    uint32_t ray = 0, seg = 0;
    bool live = false, finished = false, exhausted = false;
    while (true) {
        const uint32_t idle = __ballot_sync(0xFFFFFFFFu, !live);
        if ((uint32_t)__popc(idle) >= kRefillLanes) {
            if (finished) {  // the hits of the lanes whose rays finished
                const SceneRef &sc = MULTI ? s_sc[seg] : a.scene;
                const float4 h = ray_result(r, sc);
                a.hits[ray] = h;
                if (ACCUM) {
                    if (MULTI) {
                        const BatchScene *bs = a.segs + seg;
                        if (bs->table) accumulate_hit(bs->table, bs->frame, bs->invE, r.o, r.d, h);
                    } else if (a.table) {
                        accumulate_hit(a.table, s_frame, s_invE, r.o, r.d, h);
                    }
                }
                finished = false;
            }
            if (exhausted) {
                if (idle == 0xFFFFFFFFu) break;
            } else {
                // idle lanes take consecutive queue positions, in lane order
                const uint32_t want = __popc(idle);
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(a.queue, want);
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (base + want >= a.n) exhausted = true;
                if (!live) {
                    const uint32_t pos = base + __popc(idle & lanes_below);
                    if (pos < a.n) {
                        const uint32_t i = a.order ? __ldg(a.order + pos) : pos;
                        if (i >= a.n) {  // not a permutation of [0, n): record and skip
                            atomicOr(a.err, RR_DEVERR_BAD_INDEX);
                        } else {
                            ray = i;
                            if (MULTI) {
                                // the last segment starting at or before i (empty
                                // segments share their start with the next one, which wins)
                                uint32_t lo = 0, hi = a.n_segs;
                                while (hi - lo > 1) {
                                    const uint32_t mid = (lo + hi) >> 1;
                                    if (s_off[mid] <= i)
                                        lo = mid;
                                    else
                                        hi = mid;
                                }
                                seg = lo;
                            }
                            ray_begin(r, MULTI ? s_sc[seg] : a.scene, __ldg(a.o_tmin + i), __ldg(a.d_tmax + i));
                            live = true;
                        }
                    }
                }
                if (exhausted && __ballot_sync(0xFFFFFFFFu, live) == 0u) break;
            }
        }
        if (live && !ray_step<ANY>(r, stack, MULTI ? s_sc[seg] : a.scene, a.err)) {
            live = false;
            finished = true;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const uint32_t prev = atomicAdd(a.queue + 1, 1u);
        if (prev == gridDim.x - 1) {  // every block has stopped fetching: reset for the next launch
            a.queue[0] = 0u;
            a.queue[1] = 0u;
        }
    }
}

}  // namespace rr

using namespace rr;

namespace {

// Uploads a host BVH into a new handle (synchronous).
rr_status upload_bvh(const HostBVH &h, uint32_t n_tris, double seconds, const char *what, rr_bvh **out) {
    rr_bvh *b = new rr_bvh();
    cudaGetDevice(&b->device);
    b->nodes = nullptr;
    b->tris = nullptr;
    b->planes = nullptr;
    b->n_nodes = (uint32_t)h.nodes.size();
    b->n_tris = n_tris;
    b->root_is_leaf = 0;
    b->root_leaf_ref = 0;
    cudaError_t e = cudaSuccess;
    if (b->n_nodes) {
        e = lib_malloc(reinterpret_cast<void **>(&b->nodes), sizeof(RRNode8) * h.nodes.size());
        if (e == cudaSuccess) e = lib_malloc(reinterpret_cast<void **>(&b->tris), sizeof(RRTri) * h.tris.size());
        if (e == cudaSuccess) e = lib_malloc(reinterpret_cast<void **>(&b->planes), sizeof(float4) * h.planes.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->planes, h.planes.data(), sizeof(float4) * h.planes.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->nodes, h.nodes.data(), sizeof(RRNode8) * h.nodes.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->tris, h.tris.data(), sizeof(RRTri) * h.tris.size(), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(b->nodes);
        cudaFree(b->tris);
        cudaFree(b->planes);
        delete b;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? RR_ERR_OOM : RR_ERR_CUDA, std::string(what) + ": upload failed");
    }
    rr_bvh_info &i = b->info;
    i.n_tris = n_tris;
    i.n_nodes = b->n_nodes;
    i.n_leaves = h.n_leaves;
    i.depth = h.depth;
    i.node_bytes = sizeof(RRNode8) * (uint64_t)h.nodes.size();
    i.tri_bytes = sizeof(RRTri) * (uint64_t)h.tris.size() + sizeof(float4) * (uint64_t)h.planes.size();
    for (int c = 0; c < 3; ++c) {
        i.aabb_lo[c] = h.lo[c];
        i.aabb_hi[c] = h.hi[c];
    }
    i.build_seconds = seconds;
    *out = b;
    return RR_OK;
}

}  // namespace

extern "C" rr_status rr_build_bvh(const float *tris_host, uint32_t n_tris, rr_bvh **out) {
    if (!out) return fail(RR_ERR_INVALID_ARG, "rr_build_bvh: out is NULL");
    *out = nullptr;
    if (n_tris > 0 && !tris_host) return fail(RR_ERR_INVALID_ARG, "rr_build_bvh: tris is NULL");
    if (n_tris >= (1u << 28)) return fail(RR_ERR_UNSUPPORTED, "rr_build_bvh: at most 2^28 - 1 triangles");
    rr_status st;
    if (!device_state(&st)) return st;
    const auto t0 = std::chrono::steady_clock::now();
    HostBVH h;
    std::string err;
    st = build_wide_bvh(tris_host, n_tris, &h, &err);
    if (st != RR_OK) return fail(st, err);
    if (h.stack_need > kTraceStack)
        return fail(RR_ERR_UNSUPPORTED, "rr_build_bvh: tree needs a deeper traversal stack than the kernel has");
    return upload_bvh(h, n_tris, std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(),
                      "rr_build_bvh", out);
}

extern "C" rr_status rr_bvh_serialize(const rr_bvh *b, void *buf, size_t *bytes) {
    if (!b || !bytes) return fail(RR_ERR_INVALID_ARG, "rr_bvh_serialize: NULL argument");
    const size_t need = serialized_bvh_bytes(b->n_nodes, b->n_tris);
    if (!buf) {
        *bytes = need;
        return RR_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return fail(RR_ERR_INVALID_ARG, "rr_bvh_serialize: buffer too small");
    }
    HostBVH h;
    h.nodes.resize(b->n_nodes);
    h.tris.resize(b->n_nodes ? b->n_tris : 0);
    h.planes.resize(2 * h.tris.size());
    cudaError_t e = cudaSuccess;
    if (b->n_nodes) {
        e = cudaMemcpy(h.nodes.data(), b->nodes, sizeof(RRNode8) * h.nodes.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(h.tris.data(), b->tris, sizeof(RRTri) * h.tris.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            e = cudaMemcpy(h.planes.data(), b->planes, sizeof(float4) * h.planes.size(), cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) return fail_cuda(e, "rr_bvh_serialize: download");
    for (int c = 0; c < 3; ++c) {
        h.lo[c] = b->info.aabb_lo[c];
        h.hi[c] = b->info.aabb_hi[c];
    }
    h.depth = b->info.depth;
    h.n_leaves = b->info.n_leaves;
    serialize_bvh(h, buf);
    *bytes = need;
    return RR_OK;
}

extern "C" rr_status rr_bvh_deserialize(const void *buf, size_t bytes, rr_bvh **out) {
    if (!out) return fail(RR_ERR_INVALID_ARG, "rr_bvh_deserialize: out is NULL");
    *out = nullptr;
    rr_status st;
    if (!device_state(&st)) return st;
    HostBVH h;
    std::string err;
    st = deserialize_bvh(buf, bytes, &h, &err);
    if (st != RR_OK) return fail(st, err);
    return upload_bvh(h, (uint32_t)h.tris.size(), 0.0, "rr_bvh_deserialize", out);
}

extern "C" rr_status rr_bvh_destroy(rr_bvh *b) {
    if (!b) return RR_OK;
    cudaFree(b->nodes);
    cudaFree(b->tris);
    cudaFree(b->planes);
    delete b;
    return RR_OK;
}

extern "C" rr_status rr_bvh_get_info(const rr_bvh *b, rr_bvh_info *info) {
    if (!b || !info) return fail(RR_ERR_INVALID_ARG, "rr_bvh_get_info: NULL argument");
    *info = b->info;
    return RR_OK;
}

extern "C" rr_status rr_bvh_aabb(const rr_bvh *b, float lo[3], float hi[3]) {
    if (!b || !lo || !hi) return fail(RR_ERR_INVALID_ARG, "rr_bvh_aabb: NULL argument");
    for (int c = 0; c < 3; ++c) {
        lo[c] = b->info.aabb_lo[c];
        hi[c] = b->info.aabb_hi[c];
    }
    return RR_OK;
}

namespace {

template <bool ACC, bool ANY, bool MULTI, int BLOCK>
int trace_blocks_per_sm(size_t smem) {
    static int bps = 0;
    static size_t bps_smem = 0;
    if (bps == 0 || bps_smem != smem) {  // the batch kernels' shared memory varies with the segments
        int v = 0;
        const cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, trace_kernel<ACC, ANY, MULTI, BLOCK>, BLOCK, smem);
        bps = (e != cudaSuccess || v < 1) ? 1 : v;
        bps_smem = smem;
    }
    return bps;
}

template <bool ACC, bool ANY, bool MULTI, int BLOCK>
void trace_enqueue(const TraceArgs &a, int sm_count, cudaStream_t s) {
    const size_t smem = MULTI ? multi_smem(a.n_segs) : 0;
    const uint32_t want = (a.n + 31u) / 32u;  // warps that can get work
    uint32_t grid = (uint32_t)sm_count * (uint32_t)trace_blocks_per_sm<ACC, ANY, MULTI, BLOCK>(smem);
    grid = std::max(1u, std::min(grid, (want + BLOCK / 32 - 1) / (BLOCK / 32)));
    trace_kernel<ACC, ANY, MULTI, BLOCK><<<grid, BLOCK, smem, s>>>(a);
}

rr_status launch_trace(const rr_bvh *b, const float *o_tmin, const float *d_tmax, const uint32_t *order, uint32_t n,
                       float *hits_out, uint32_t flags, rr_length_table *table, void *stream, const char *what) {
    if (!b) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": NULL bvh");
    if (flags & ~(uint32_t)RR_TRACE_ANY_HIT) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": unknown flags");
    const bool any = (flags & RR_TRACE_ANY_HIT) != 0;
    if (any && table)
        return fail(RR_ERR_INVALID_ARG, std::string(what) + ": any-hit distances are not ray lengths for the table");
    if (n == 0) return RR_OK;
    if (!o_tmin || !d_tmax || !hits_out) return fail(RR_ERR_INVALID_ARG, std::string(what) + ": NULL buffer");
    if (!aligned16(o_tmin) || !aligned16(d_tmax) || !aligned16(hits_out) || !aligned(order, 4))
        return fail(RR_ERR_INVALID_ARG, std::string(what) + ": misaligned buffer");
    if (overlaps(hits_out, 16ull * n, o_tmin, 16ull * n) || overlaps(hits_out, 16ull * n, d_tmax, 16ull * n) ||
        (order && overlaps(hits_out, 16ull * n, order, 4ull * n)))
        return fail(RR_ERR_INVALID_ARG, std::string(what) + ": hits overlap an input");
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    cudaStream_t s = as_stream(stream);
    TraceArgs a{};
    a.scene.nodes = reinterpret_cast<const float4 *>(b->nodes);
    a.scene.tris = reinterpret_cast<const float4 *>(b->tris);
    a.scene.planes = b->planes;
    a.scene.n_nodes = b->n_nodes;
    a.scene.n_tris = b->n_tris;
    a.o_tmin = reinterpret_cast<const float4 *>(o_tmin);
    a.d_tmax = reinterpret_cast<const float4 *>(d_tmax);
    a.hits = reinterpret_cast<float4 *>(hits_out);
    a.order = order;
    a.n = n;
    a.err = error_word(ds, s);
    a.table = table ? table->cells : nullptr;
    for (int c = 0; c < 3; ++c) {
        a.tlo[c] = table ? table->box.lo[c] : 0.0f;
        a.thi[c] = table ? table->box.hi[c] : 0.0f;
    }
    // The length-table update: a separate pass over the traced rays when the
    // hits land in device memory (it runs at full lane use, with lanes that
    // share a cell combined before the atomics, and reads rays and hits from
    // L2), fused into the trace when they go straight to host memory.
    cudaPointerAttributes pa{};
    bool hits_on_device = false;
    if (table) {
        if (cudaPointerGetAttributes(&pa, hits_out) == cudaSuccess)
            hits_on_device = pa.type == cudaMemoryTypeDevice;
        else
            cudaGetLastError();
    }
    const bool fuse = table && !hits_on_device;
    const rr_status st2 = with_trace_queue(ds, s, [&](uint32_t *queue) {
        a.queue = queue;
        if (fuse)
            trace_enqueue<true, false, false, kTraceBlock>(a, ds->sm_count, s);
        else if (any)
            trace_enqueue<false, true, false, kTraceBlock>(a, ds->sm_count, s);
        else
            trace_enqueue<false, false, false, kTraceBlock>(a, ds->sm_count, s);
        note_launches(1);
        return check_launch(what);
    });
    if (st2 != RR_OK || !table || fuse) return st2;
    return rr_length_table_accumulate(table, o_tmin, d_tmax, hits_out, n, stream);
}

}  // namespace

namespace rr {

rr_status launch_trace_batch(const BatchScene *segs, const uint32_t *seg_offsets, uint32_t n_segs, const float *o_tmin,
                             const float *d_tmax, const uint32_t *order, uint32_t n, float *hits_out,
                             bool accumulate, uint32_t block, uint32_t *queue, uint32_t *err, cudaStream_t s) {
    rr_status st;
    DeviceState *ds = device_state(&st);
    if (!ds) return st;
    TraceArgs a{};
    a.o_tmin = reinterpret_cast<const float4 *>(o_tmin);
    a.d_tmax = reinterpret_cast<const float4 *>(d_tmax);
    a.hits = reinterpret_cast<float4 *>(hits_out);
    a.order = order;
    a.n = n;
    a.queue = queue;
    a.err = err;
    a.segs = segs;
    a.seg_offsets = seg_offsets;
    a.n_segs = n_segs;
    const int sms = ds->sm_count;
    if (accumulate) {
        if (block == 128) trace_enqueue<true, false, true, 128>(a, sms, s);
        else if (block == 512) trace_enqueue<true, false, true, 512>(a, sms, s);
        else trace_enqueue<true, false, true, 256>(a, sms, s);
    } else {
        if (block == 128) trace_enqueue<false, false, true, 128>(a, sms, s);
        else if (block == 512) trace_enqueue<false, false, true, 512>(a, sms, s);
        else trace_enqueue<false, false, true, 256>(a, sms, s);
    }
    note_launches(1);
    return check_launch("rr_batch trace");
}

}  // namespace rr

extern "C" rr_status rr_trace(const rr_bvh *b, const float *o_tmin, const float *d_tmax, uint32_t n, float *hits_out,
                              void *stream) {
    return launch_trace(b, o_tmin, d_tmax, nullptr, n, hits_out, 0u, nullptr, stream, "rr_trace");
}

extern "C" rr_status rr_trace_accumulate(const rr_bvh *b, const float *o_tmin, const float *d_tmax, uint32_t n,
                                         float *hits_out, rr_length_table *table, void *stream) {
    if (!table) return fail(RR_ERR_INVALID_ARG, "rr_trace_accumulate: NULL table");
    return launch_trace(b, o_tmin, d_tmax, nullptr, n, hits_out, 0u, table, stream, "rr_trace_accumulate");
}

extern "C" rr_status rr_trace_ex(const rr_bvh *b, const float *o_tmin, const float *d_tmax, const uint32_t *order,
                                 uint32_t n, float *hits_out, uint32_t flags, rr_length_table *table, void *stream) {
    return launch_trace(b, o_tmin, d_tmax, order, n, hits_out, flags, table, stream, "rr_trace_ex");
}
