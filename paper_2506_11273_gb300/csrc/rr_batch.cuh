// Internal interface between the library's units: the batch runtime, the
// serving loop and the fused key + sort call, and the kernels they enqueue.
#pragma once

#include "rr_common.cuh"
#include "rr_keymath.cuh"

namespace rr {

constexpr uint32_t kMaxBatchSegments = 1024;

// Device descriptor of one wavefront (segment) of a batch: its scene's BVH,
// the quantisation frame of its box, and its length table (or null).
struct BatchScene {
    const float4 *nodes;
    const float4 *tris;
    const float4 *planes;
    uint32_t n_nodes;
    uint32_t n_tris;
    unsigned long long *table;  // cells {sum, count}; null: no adaptive estimate, no update
    QuantFrame frame;           // make_frame of the wavefront's box (computed on the device)
    float invE;                 // 1 / frame.E
};

// Fills frame and invE of segs[k] from boxes[k] (6 floats lo, hi) for k < n.
cudaError_t launch_batch_frames(BatchScene *segs, const float *boxes, uint32_t n, cudaStream_t s);

// Keys of every ray of a batch: segment s in the bits above key_bits, the
// wavefront's own key (layout, estimate) below.  keys: u32 when
// key_bits + seg_bits <= 32, else u64.
rr_status launch_keys_batch(const BatchScene *segs, const uint32_t *seg_offsets, uint32_t n_segs,
                            rr_key_layout layout, rr_t_source tsrc, float ratio, uint32_t key_bits,
                            uint32_t seg_bits, const float *o_tmin, const float *d_tmax, uint32_t n, void *keys,
                            cudaStream_t s);

// Closest-hit trace of a batch through `order`, hits in input order; the
// length tables of the segments are updated when `accumulate`.  queue: two
// device words at zero, owned by the caller.  err: the error word the kernel
// reports to.
rr_status launch_trace_batch(const BatchScene *segs, const uint32_t *seg_offsets, uint32_t n_segs, const float *o_tmin,
                             const float *d_tmax, const uint32_t *order, uint32_t n, float *hits_out,
                             bool accumulate, uint32_t block, uint32_t *queue, uint32_t *err, cudaStream_t s);

// rr_sort with arguments already checked and device errors reported to `err`.
rr_status sort_enqueue(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                       uint32_t radix_bits, void *workspace, uint32_t *err, int sm_count, cudaStream_t s);

// The argument checks of rr_sort, with `what` naming the caller in messages.
rr_status sort_check(const char *what, const void *keys_in, const void *keys_out, const uint32_t *perm_out,
                     uint32_t n, uint32_t bits, uint32_t radix_bits, const void *workspace,
                     size_t workspace_bytes);

// Where a sort's counting stage puts its results inside the workspace: the
// digit counts [pass][2^radix_bits] (zeroed by the caller, then added to),
// the tile counters [pass] and the look-back words (zero_count uint4 to
// clear).  Lets a kernel that produces the keys count their digits itself.
struct SortCountTarget {
    uint32_t *hist;
    uint32_t *counters;
    uint4 *zero_words;
    size_t zero_count;
    uint32_t passes;
    uint32_t radix_bits;
};
SortCountTarget sort_count_target(uint32_t n, uint32_t bits, uint32_t radix_bits, void *workspace);

// The digit passes of rr_sort once the counting stage has filled the
// workspace (arguments already checked).
rr_status sort_enqueue_passes(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                              uint32_t radix_bits, void *workspace, uint32_t *err, int sm_count, cudaStream_t s);

}  // namespace rr
