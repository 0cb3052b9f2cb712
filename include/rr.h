/*
 * rr.h - C ABI of the GB300 ray-reordering library (librr.so).
 *
 * The library implements, per bounce of a wavefront ray tracer, the pipeline
 * studied by Meister, Boksansky, Guthe and Bittner, "On Ray Reordering
 * Techniques for Faster GPU Ray Tracing" (I3D 2020):
 *
 *   rr_compute_keys  per-ray sorting key (Section 3.1, Figure 2)
 *   rr_sort          stable LSD radix sort of (key, ray index) pairs (Section 3.2)
 *   rr_permute       the extra pass that moves ray data into sorted order (Section 3.2)
 *   rr_trace         closest-hit traversal of a BVH; it does not depend on the order
 *                    of the rays (Section 1: reordering is agnostic to the trace kernel)
 *   rr_length_table_accumulate
 *                    the adaptive ray-length cache updated after each trace (Section 3.1.6)
 *
 * and around it:
 *
 *   rr_trace_ex          indirect ray access through a permutation (Section 4.4.1)
 *                        and any-hit traversal for shadow rays (Section 4)
 *   rr_key_sort          keys and their sort in one call, the sort's digit counting
 *                        fused into the key kernel
 *   rr_sort_segments     local (block-wise) sort (Section 3.2)
 *   rr_coherence_capsule the capsule coherence measure (Section 4.3)
 *   rr_bvh_serialize, rr_bvh_deserialize
 *                        store a built BVH and reload it (checked before upload)
 *   rr_pipeline_*        one bounce behind one handle
 *   rr_batch_*           many wavefronts over resident scenes as one CUDA graph, with
 *                        an autotuner and its JSON cache
 *   rr_server_*          a serving loop with continuous batching under a memory budget
 *
 * Conventions shared by every call:
 *  - Device buffers are owned by the caller.  The library owns only the opaque
 *    handles (rr_bvh, rr_length_table, rr_pipeline, rr_batch, rr_server) and the
 *    device memory behind them.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream) and the call returns without synchronising, unless stated otherwise.
 *  - Arguments are checked on the host before anything is enqueued.  A bad
 *    argument returns RR_ERR_INVALID_ARG and enqueues nothing.  n == 0 is a
 *    no-op that returns RR_OK.
 *  - Failures inside kernels (a radix-sort look-back or a bulk copy that waited
 *    too long, a traversal stack overflow, an index out of range) never trap:
 *    the kernel records a flag in the error word of the stream it runs on and
 *    finishes.  rr_stream_error() reads and clears one stream's word without
 *    synchronising; rr_device_error() synchronises the device and reads and
 *    clears every word.
 *  - Ray layout (structure of arrays, 16-byte aligned):
 *      o_tmin  float4 per ray: origin.x, origin.y, origin.z, tmin
 *      d_tmax  float4 per ray: direction.x, .y, .z, tmax
 *      payload uint32 per ray: caller data moved with the ray (optional)
 *  - Hit layout: float4 per ray: t, u, v, triangle id (the id's uint32 bits).
 *    A miss is t = +inf, u = v = 0, id = 0xFFFFFFFF.  Hits are written in the
 *    order of the rays that were traced.
 *  - Keys are uint32 when bits <= 32 and uint64 when 32 < bits <= 64.
 *  - A handle is used by one host thread at a time; rr_server's calls may come
 *    from any thread.
 */
#ifndef RR_H
#define RR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RR_OK = 0,
    RR_ERR_INVALID_ARG = 1, /* a pointer, size or option failed the host-side checks */
    RR_ERR_CUDA = 2,        /* a CUDA runtime call failed (see rr_last_error_message) */
    RR_ERR_OOM = 3,         /* a library-owned allocation failed */
    RR_ERR_TIMEOUT = 4,     /* device: a bounded wait gave up (radix-sort look-back) */
    RR_ERR_STACK = 5,       /* device: a traversal stack would have overflowed */
    RR_ERR_UNSUPPORTED = 6, /* a valid request this build does not handle */
    RR_ERR_TOO_LARGE = 7,   /* n exceeds the fixed maximum of rr_sort_noalloc */
    RR_ERR_DEVICE = 8       /* a kernel of the work recorded a device error flag (served requests) */
} rr_status;

/* Device error flags accumulated in the per-device error word. */
#define RR_DEVERR_LOOKBACK_TIMEOUT 0x1u
#define RR_DEVERR_TRACE_STACK 0x2u
#define RR_DEVERR_BAD_INDEX 0x4u /* an index buffer entry was >= n; that entry was skipped */
#define RR_DEVERR_COPY_TIMEOUT 0x8u /* a bulk copy into shared memory did not complete in time */

/* Sorting-key layouts (Section 3.1, Figure 2). */
typedef enum {
    RR_KEY_AILA = 0,         /* origin and direction interleaved; each quantised direction
                                component has three leading zero bits (Section 3.1.4) */
    RR_KEY_AILA_COMPACT = 1, /* the same bits with the leading zeros removed (Section 3.1.4) */
    RR_KEY_TWO_POINT = 2,    /* origin and estimated termination point interleaved,
                                origin first in every level (Section 3.1.5) */
    RR_KEY_ORIGIN = 3,       /* 3D Morton code of the origin only (Section 3.1.1) */
    RR_KEY_REIS = 4,         /* origin bits, then direction bits: 22 + 10 at 32 bits, the same
                                ratio at other lengths (Section 3.1.2) */
    RR_KEY_COSTA = 5,        /* direction bits, then origin bits: 8 + 24 at 32 bits (Section 3.1.3) */
    RR_KEY_OCTAHEDRON = 6    /* origin interleaved with the octahedral 2D direction (Meyer et
                                al. 2010), compacted as Aila (Section 3.1.4, Figure 2) */
} rr_key_layout;

/* Termination estimate of the Two Point key (Section 3.1.6). */
typedef enum {
    RR_T_FIXED = 0,    /* ratio * largest extent of the scene box (paper: ratio 0.25) */
    RR_T_ADAPTIVE = 1, /* mean ray length of the ray's cell in a rr_length_table */
    RR_T_GIVEN = 2     /* caller-supplied lengths, e.g. real hits ("Two Point Real") */
} rr_t_source;

typedef struct rr_bvh rr_bvh;
typedef struct rr_length_table rr_length_table;
typedef struct rr_pipeline rr_pipeline;

typedef struct {
    uint32_t layout;   /* rr_key_layout */
    uint32_t bits;     /* key length b, 1..64: the first b bits of the interleaved string */
    uint32_t t_source; /* rr_t_source; read only for RR_KEY_TWO_POINT */
    float ratio;       /* RR_T_FIXED: estimate = ratio * E */
    float aabb_lo[3];  /* scene box: origins, directions and termination points are */
    float aabb_hi[3];  /* quantised per axis inside it (finite, lo <= hi) */
    const float *t_given;          /* RR_T_GIVEN: device, n world-space lengths */
    const rr_length_table *table;  /* RR_T_ADAPTIVE: a table created for the same box */
} rr_key_params;

typedef struct {
    uint32_t n_tris;
    uint32_t n_nodes;  /* 8-wide nodes */
    uint32_t n_leaves; /* leaf slots (1..4 triangles each) */
    uint32_t depth;    /* node levels from the root to the deepest node */
    uint64_t node_bytes;
    uint64_t tri_bytes;
    float aabb_lo[3];
    float aabb_hi[3];
    double build_seconds;
} rr_bvh_info;

/* ---------------------------------------------------------------- keys */

/*
 * rr_compute_keys - one sorting key per ray (Section 3.1; layouts in Figure 2).
 *
 * Each coordinate is mapped per axis into [0,1] by the scene box (params->aabb),
 * clamped, and quantised to 32 bits by truncation.  Directions are normalised
 * and mapped from [-1,1] to [0,1].  The Aila layouts interleave origin and
 * direction (the direction shifted right by 3: its three leading zero bits);
 * the compact layout drops the nine zero bits.  The origin, Reis and Costa
 * layouts take prefixes of the 3D Morton strings of the origin and of the
 * direction; the octahedron layout interleaves the origin with the two
 * octahedral coordinates of the direction (each shifted right by 4, the
 * zero slots dropped).  The Two Point layout
 * interleaves the origin with p = o + t_est * normalize(d), where t_est comes
 * from params->t_source; a non-finite t_est is replaced by 4 * E.  The key is
 * the first `bits` bits of the 192-bit interleaved string, x before y before z.
 * All float arithmetic is correctly rounded binary32, so keys are exact.
 *
 * o_tmin, d_tmax: device, n float4 each.  keys_out: device, n uint32 (bits <= 32)
 * or n uint64.  For RR_T_ADAPTIVE the table must have been created for the same
 * box as params->aabb.
 */
rr_status rr_compute_keys(const float *o_tmin, const float *d_tmax, uint32_t n,
                          const rr_key_params *params, void *keys_out, void *stream);

/* ---------------------------------------------------------------- sort */

/*
 * rr_sort_workspace_size - device workspace bytes rr_sort needs for n keys of
 * `bits` bits sorted with `radix_bits`-bit digits (4 or 8).
 */
rr_status rr_sort_workspace_size(uint32_t n, uint32_t bits, uint32_t radix_bits, size_t *bytes);

/*
 * rr_sort - stable least-significant-digit radix sort of (key, index) pairs
 * (Section 3.2: the pairs are sorted first and the ray data moved afterwards).
 *
 * perm_out[i] = index of the i-th smallest key; equal keys keep their input
 * order.  keys_in (device, uint32 for bits <= 32 else uint64) is not modified;
 * only bits [0, bits) are sorted and the higher bits must be zero.  keys_out
 * (device, same type, may be NULL) receives the sorted keys.  keys_in, keys_out
 * and perm_out must not overlap.  workspace: device, at least
 * rr_sort_workspace_size() bytes, 256-byte aligned, owned by the caller and
 * free again once the work on `stream` has completed.  n < 2^30.
 * One histogram pass plus ceil(bits / radix_bits) onesweep passes are enqueued;
 * the passes use programmatic dependent launch, and the last one lets the next
 * kernel of `stream` start early: a caller's kernel launched there with
 * cudaLaunchAttributeProgrammaticStreamSerialization must call
 * cudaGridDependencySynchronize() before it reads the sort's outputs (kernels
 * launched without that attribute wait for the sort as usual).
 */
rr_status rr_sort(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n,
                  uint32_t bits, uint32_t radix_bits, void *workspace, size_t workspace_bytes,
                  void *stream);

/*
 * rr_key_sort - the keys of Section 3.1 and their stable radix sort of
 * Section 3.2 in one call: exactly rr_compute_keys(o_tmin, d_tmax, n, params,
 * keys_out) followed by rr_sort(keys_out, NULL, perm_out, n, params->bits,
 * radix_bits, workspace), with the sort's digit counting done by the key
 * kernel as it produces the keys (the sort's separate counting pass, which
 * reads every key once more, is not launched).
 *
 * keys_out: device, n uint32 (bits <= 32) or n uint64; receives the keys in
 * input order.  perm_out: device, n uint32; receives the sort permutation.
 * workspace: as for rr_sort with bits = params->bits.  Every check of
 * rr_compute_keys and rr_sort applies; the rays must not overlap keys_out,
 * perm_out or the workspace.  Device errors go to the error word of `stream`.
 */
rr_status rr_key_sort(const float *o_tmin, const float *d_tmax, uint32_t n, const rr_key_params *params,
                      void *keys_out, uint32_t *perm_out, uint32_t radix_bits, void *workspace,
                      size_t workspace_bytes, void *stream);

/*
 * rr_sort_segments - local (block-wise) sort, Section 3.2: the keys are cut
 * into consecutive segments of `segment` keys (256, 512, 1024, 2048 or 4096;
 * the last segment may be shorter) and each segment is sorted stably by its
 * low `bits` bits on its own, in on-chip memory.  perm_out[i] (device, n
 * uint32) is a global index: segment s holds a permutation of its own range
 * [s * segment, min(n, (s + 1) * segment)).  keys_out (device or NULL)
 * receives the keys in that order.  Same key types and alignment rules as
 * rr_sort; needs no workspace; one kernel.  n < 2^30.
 */
rr_status rr_sort_segments(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n, uint32_t bits,
                           uint32_t segment, void *stream);

/*
 * rr_sort_noalloc - rr_sort for callers that cannot allocate device memory.
 * The paper has no counterpart: it exists for integration, not for the method.
 *
 * Some callers cannot give rr_sort a workspace: a renderer or game engine whose
 * own allocator owns the device-memory budget, a plug-in running inside such a
 * host, or a real-time frame loop that forbids cudaMalloc/cudaFree once it has
 * started.  This entry point allocates nothing.  Its scratch is one file-scope
 * device array of RR_SORT_NOALLOC_SCRATCH_BYTES (26 MiB) inside librr.so, and
 * every GPU that loads the library holds that array until the process exits.
 *
 * Arguments, results and launches are those of rr_sort without the workspace
 * (including its programmatic dependent launch): perm_out receives the stable
 * order, keys_out (may be NULL) the sorted keys.  n may be
 * at most RR_SORT_NOALLOC_MAX_N (2^20 keys); a larger n returns
 * RR_ERR_TOO_LARGE and enqueues nothing.  Other bad arguments return
 * RR_ERR_INVALID_ARG.  Errors are reported by the returned status only; this
 * call records no message for rr_last_error_message().
 *
 * The first call on a device does a one-time set-up with that device current:
 * it looks up the array's device address (cudaGetSymbolAddress) and the SM
 * count.  Make that first call before any stream capture.
 *
 * All calls on a device share the one array, and the array keeps the last
 * call's contents; each call clears what must start at zero before it uses it.
 * Calls whose work can overlap on the GPU (on different streams, or from host
 * threads without ordering between them) race on the array: serialise them.
 * The error word of these calls lives in the array; a look-back wait that runs
 * out sets RR_DEVERR_LOOKBACK_TIMEOUT there, where it stays until
 * rr_device_error() reads and clears it (rr_stream_error() does not see it).
 */
#define RR_SORT_NOALLOC_MAX_N (1u << 20)
#define RR_SORT_NOALLOC_SCRATCH_BYTES (26u << 20)
rr_status rr_sort_noalloc(const void *keys_in, void *keys_out, uint32_t *perm_out, uint32_t n,
                          uint32_t bits, uint32_t radix_bits, void *stream);

/* ---------------------------------------------------------------- reorder */

/*
 * rr_permute - the reorder pass of Section 3.2: out[i] = in[perm[i]] for
 * o_tmin, d_tmax and (when both pointers are non-NULL) payload.  Bitwise copy.
 * perm: device, n indices < n.  Inputs and outputs must not overlap.
 */
rr_status rr_permute(const float *o_tmin_in, const float *d_tmax_in, const uint32_t *payload_in,
                     const uint32_t *perm, uint32_t n, float *o_tmin_out, float *d_tmax_out,
                     uint32_t *payload_out, void *stream);

/* ---------------------------------------------------------------- BVH and trace */

/*
 * rr_build_bvh - builds, on the host, a BVH with 8-wide compressed nodes over
 * a triangle soup (tris_host: 9 floats per triangle, v0 v1 v2) and uploads it
 * to the current device.  Synchronous.  The paper's trace is RTX hardware; this
 * BVH serves the software trace kernel.  The handle owns its device memory.
 */
rr_status rr_build_bvh(const float *tris_host, uint32_t n_tris, rr_bvh **out);
rr_status rr_bvh_destroy(rr_bvh *bvh);
rr_status rr_bvh_get_info(const rr_bvh *bvh, rr_bvh_info *info);
/* The scene box: min and max over all vertices (the box the keys quantise in, Section 3). */
rr_status rr_bvh_aabb(const rr_bvh *bvh, float lo[3], float hi[3]);

/*
 * rr_bvh_serialize - writes a BVH into host memory, so that a scene's build
 * (seconds for millions of triangles) can be stored and reloaded.  The format:
 * a 64-byte header (magic "RRBVH8", format version 1, node size, node and
 * triangle counts, depth, leaf count, scene box) followed by the node,
 * triangle and plane arrays as they sit in device memory (little-endian).
 * buf == NULL: *bytes receives the size needed and nothing is written.
 * Otherwise *bytes is the capacity of buf (host); a smaller capacity returns
 * RR_ERR_INVALID_ARG with the size needed in *bytes.  Synchronous.
 */
rr_status rr_bvh_serialize(const rr_bvh *bvh, void *buf, size_t *bytes);

/*
 * rr_bvh_deserialize - a new handle from rr_bvh_serialize's bytes (host),
 * uploaded to the current device.  The buffer is checked before anything is
 * uploaded: size against the header, children stored after their parent and
 * inside the node array, triangles inside the triangle array, leaf bits, depth
 * within the trace kernel's stack, triangle ids below the count; a buffer that
 * fails a check returns RR_ERR_INVALID_ARG.  Synchronous; the caller keeps
 * ownership of buf.
 */
rr_status rr_bvh_deserialize(const void *buf, size_t bytes, rr_bvh **out);

/*
 * rr_trace - closest hit of every ray: the smallest t with tmin < t < tmax over
 * all triangles (two-sided), with its barycentrics and triangle id (index in the
 * soup given to rr_build_bvh).  o_tmin, d_tmax: device, n float4.  hits_out:
 * device, n float4.  The kernel is persistent: warps take batches of 32
 * consecutive rays from a queue, so the order of the rays decides which rays
 * share a warp (the effect reordering is meant to improve, Section 4.2).
 */
rr_status rr_trace(const rr_bvh *bvh, const float *o_tmin, const float *d_tmax, uint32_t n,
                   float *hits_out, void *stream);

/*
 * rr_trace_accumulate - rr_trace and, in the same kernel, the length-table
 * update of rr_length_table_accumulate for the traced rays (Section 3.1.6: the
 * table is updated after each trace pass).  Same hits and same table contents
 * as rr_trace followed by rr_length_table_accumulate on the same rays; the rays
 * and hits are not read a second time.  table: a table created for the box the
 * caller quantises with (the usual rr_length_table rules apply).
 */
rr_status rr_trace_accumulate(const rr_bvh *bvh, const float *o_tmin, const float *d_tmax,
                              uint32_t n, float *hits_out, rr_length_table *table, void *stream);

/* Flags of rr_trace_ex. */
#define RR_TRACE_ANY_HIT 0x1u /* shadow rays: stop at the first hit inside (tmin, tmax) */

/*
 * rr_trace_ex - rr_trace with two options of the reordering study.
 *
 * order (device, n uint32, or NULL): indirect access.  Work position k traces
 * ray order[k] and writes its hit to hits_out[order[k]], so a permutation from
 * rr_sort sets which rays share a warp without the rays being gathered first,
 * and the hits come back in the order of the input rays (Section 4.4.1, the
 * indirect ray access of the CUDA trace kernel).  order must be a permutation
 * of [0, n): an entry >= n is skipped and sets RR_DEVERR_BAD_INDEX; a repeated
 * entry traces that ray twice.  NULL: position k traces ray k (rr_trace).
 *
 * flags: RR_TRACE_ANY_HIT ends each ray at the first triangle it meets inside
 * (tmin, tmax), as an any-hit kernel for shadow rays does (Section 4, shadow
 * rays); the hit record describes that triangle (its t, barycentrics and id),
 * and a miss is reported as in rr_trace.  Which triangle is found first
 * depends on the traversal order; whether one is found does not.
 *
 * table: NULL, or a length table to update as rr_trace_accumulate does (not
 * with RR_TRACE_ANY_HIT: RR_ERR_INVALID_ARG).
 */
rr_status rr_trace_ex(const rr_bvh *bvh, const float *o_tmin, const float *d_tmax, const uint32_t *order,
                      uint32_t n, float *hits_out, uint32_t flags, rr_length_table *table, void *stream);

/* ---------------------------------------------------------------- ray-length table */

/*
 * Adaptive termination estimate (Section 3.1.6): a table of 2^20 cells indexed
 * by the 20-bit compacted Aila code of (origin, direction).  Each cell holds
 * the sum of ray lengths (uint64, fixed point in units of E / 2^24) and the
 * number of rays (uint32).  Every cell starts with one dummy ray of length
 * 0.25 * E, E = largest extent of the box.  Lengths are t * |d| of rays that
 * hit, clamped to [0, 64 * E].  Integer accumulation makes the table
 * independent of the order of the rays.
 */
rr_status rr_length_table_create(const float aabb_lo[3], const float aabb_hi[3],
                                 rr_length_table **out, void *stream);
rr_status rr_length_table_reset(rr_length_table *table, void *stream);
rr_status rr_length_table_accumulate(rr_length_table *table, const float *o_tmin,
                                     const float *d_tmax, const float *hits, uint32_t n,
                                     void *stream);
/* Copies the cells to host arrays of 2^20 entries each (synchronous). */
rr_status rr_length_table_read(const rr_length_table *table, uint64_t *sum_host,
                               uint32_t *cnt_host);
/* Overwrites the cells from host arrays of 2^20 entries each (synchronous). */
rr_status rr_length_table_write(rr_length_table *table, const uint64_t *sum_host,
                                const uint32_t *cnt_host);
rr_status rr_length_table_destroy(rr_length_table *table);

/* ---------------------------------------------------------------- one bounce */

/*
 * rr_pipeline - one bounce of the reordered path: keys -> sort -> permute ->
 * trace (-> length-table update when the key uses RR_T_ADAPTIVE).  The handle
 * owns the workspace and the sorted ray buffers for up to max_n rays.
 * key params are copied; their pointers (t_given, table) must stay valid.
 */
rr_status rr_pipeline_create(const rr_bvh *bvh, uint32_t max_n, const rr_key_params *params,
                             uint32_t radix_bits, rr_pipeline **out);
rr_status rr_pipeline_destroy(rr_pipeline *p);

/*
 * rr_pipeline_run - device buffers.  Writes hits_out (device, n float4) and,
 * when payload_in/payload_out are non-NULL, the payloads, both in sorted order.
 */
rr_status rr_pipeline_run(rr_pipeline *p, const float *o_tmin, const float *d_tmax,
                          const uint32_t *payload_in, uint32_t n, float *hits_out,
                          uint32_t *payload_out, void *stream);

/*
 * rr_pipeline_submit_host - one bounce on host buffers, enqueued without
 * waiting.  Submissions alternate between two device staging slots, so the
 * upload of one submission overlaps the kernels of the one before: rays and
 * payloads go up on the handle's upload stream, the bounce runs on `stream`
 * with its hits staged in the slot, and the sorted payloads and the hits come
 * back on the handle's side stream while the next submission computes.
 *
 * *ticket receives a number for rr_pipeline_wait (0 for n == 0).  Until that
 * wait returns, the host buffers of the submission must stay allocated, its
 * inputs unchanged and its outputs unread.  All submissions to one handle use
 * the same `stream` (they share the handle's key, sort and sorted-ray
 * buffers); with the adaptive estimate, each bounce sees the table updated by
 * the submissions before it, as if they had run one after the other.
 * Page-locked buffers give full link speed; pageable ones work, slower.
 */
rr_status rr_pipeline_submit_host(rr_pipeline *p, const float *o_tmin_host, const float *d_tmax_host,
                                  const uint32_t *payload_host, uint32_t n, float *hits_host,
                                  uint32_t *payload_out_host, void *stream, uint64_t *ticket);

/* Blocks until submission `ticket` (and every submission before it on the
 * handle) has written its hits and payloads to the host.  0 returns at once. */
rr_status rr_pipeline_wait(rr_pipeline *p, uint64_t ticket);

/*
 * rr_pipeline_run_host - rr_pipeline_submit_host followed by rr_pipeline_wait.
 */
rr_status rr_pipeline_run_host(rr_pipeline *p, const float *o_tmin_host, const float *d_tmax_host,
                               const uint32_t *payload_host, uint32_t n, float *hits_host,
                               uint32_t *payload_out_host, void *stream);

/* ---------------------------------------------------------------- coherence measure */

/*
 * rr_coherence_capsule - the capsule coherence measure of Section 4.3.  For
 * each run of `subset` consecutive rays (1..64; the paper uses 64) the capsule
 * is fitted as follows: its axis joins the centroid of the origins and the
 * centroid of the termination points o + normalize(d) * t (t from hits; a miss
 * ends at 4 * E); its radii are the mean distances of the origins and of the
 * termination points from that axis; its area is two hemispheres plus the
 * lateral area of the cone frustum between them.  areas_out (device) receives
 * one float per run: n / subset runs (a shorter tail is ignored), or one run
 * when n < subset.  The mean of the areas is the paper's coherence value; lower
 * means more coherent.  fp32 arithmetic.
 */
rr_status rr_coherence_capsule(const float *o_tmin, const float *d_tmax, const float *hits, uint32_t n,
                               uint32_t subset, float E, float *areas_out, void *stream);

/* ---------------------------------------------------------------- batched execution */

/*
 * A batch is many wavefronts, each traced against one of several resident
 * scenes, handled by one chain of launches: keys of every ray (each in its own
 * wavefront's box and table), one stable radix sort whose keys carry the
 * wavefront number above the key's bits (so every wavefront is sorted on its
 * own and stays in its range: the local sort of Section 3.2 with
 * wavefront-sized segments), and one trace of all rays through the
 * permutation (indirect access, Section 4.4.1), hits in input order.  The chain
 * is captured once per configuration and buffer set into a CUDA graph and
 * replayed (rr_batch_run); rr_batch_run_loop issues the same work wavefront
 * by wavefront through the single-wavefront calls, with the same results.
 *
 * The rays of all wavefronts lie in one pair of buffers (o_tmin, d_tmax,
 * float4 each); wavefront k holds rays [offset, offset + count), contiguous
 * and in order.
 */
typedef struct {
    const rr_bvh *bvh;        /* the scene this wavefront is traced against */
    rr_length_table *table;   /* Two Point ADAPTIVE: the scene's table (read by the key,
                                 updated by the trace); otherwise ignored */
    float aabb_lo[3];         /* the quantisation box of the wavefront's keys */
    float aabb_hi[3];
    uint32_t offset;          /* first ray of the wavefront in the batch buffers */
    uint32_t count;           /* rays of the wavefront (0 allowed) */
} rr_wavefront;

typedef struct {
    uint32_t key_bits;     /* bits of each wavefront's own key; key_bits + wavefront bits <= 64.
                              0: no reordering (rays traced in input order, no keys, no sort,
                              perm_out not written) */
    uint32_t radix_bits;   /* 4 or 8 */
    uint32_t trace_block;  /* threads per trace block: 128, 256 or 512 */
    int32_t layout;        /* key layout of this run (an rr_key_layout), or -1 for the batch's own
                              layout and estimate; another layout only orders the rays (Two Point
                              then takes the FIXED estimate) and the tables are still updated */
} rr_batch_config;

typedef struct rr_batch rr_batch;

/*
 * rr_batch_create - validates 1..1024 wavefronts (the array is copied; BVHs and
 * tables must outlive the batch) and allocates the batch's device memory
 * (keys, permutation, sort workspace, descriptors).  layout/t_source/ratio as
 * in rr_key_params; RR_T_GIVEN is not batched (RR_ERR_UNSUPPORTED).
 * Synchronising.
 */
rr_status rr_batch_create(const rr_wavefront *fronts, uint32_t n_fronts, rr_key_layout layout,
                          rr_t_source t_source, float ratio, rr_batch **out);
rr_status rr_batch_destroy(rr_batch *batch);

/* Rays in the batch, wavefront-number bits, graphs captured so far (each may be NULL). */
rr_status rr_batch_info(const rr_batch *batch, uint32_t *n_rays, uint32_t *seg_bits, uint32_t *n_graphs);

/*
 * rr_batch_run - the whole batch as one CUDA graph launch on `stream`.  The
 * graph for (cfg, o_tmin, d_tmax, hits_out, perm_out) is captured on first use
 * and kept with the batch (at most 32 graphs; the oldest is dropped).  hits_out (device, float4 per ray) in input order;
 * perm_out (device, uint32 per ray, or NULL): the batch permutation, whose
 * range of wavefront k is the stable sort of that wavefront's keys (global
 * indices).  Runs of one batch must not overlap in time (they share the
 * batch's scratch); use one stream per batch.
 */
rr_status rr_batch_run(rr_batch *batch, const float *o_tmin, const float *d_tmax, float *hits_out,
                       uint32_t *perm_out, const rr_batch_config *cfg, void *stream);

/*
 * rr_batch_run_loop - the same work without a graph, launched wavefront by
 * wavefront through rr_compute_keys, rr_sort and rr_trace_ex (all keys first,
 * so the tables are read as rr_batch_run reads them).  Same hits and tables as
 * rr_batch_run; perm_out holds indices local to each wavefront (the batch
 * permutation minus the wavefront's offset).
 */
rr_status rr_batch_run_loop(rr_batch *batch, const float *o_tmin, const float *d_tmax, float *hits_out,
                            uint32_t *perm_out, const rr_batch_config *cfg, void *stream);

/*
 * rr_batch_tune - autotuner: times rr_batch_run on these buffers for the key
 * layouts {the batch's own, Costa, Aila Compact} x key bits {12, 16, 20, 24, 32,
 * 48, 64} (capped by the wavefront bits) x radix width {4, 8}, and for no
 * reordering (key bits 0), at 256-thread trace blocks, then trace blocks of 128
 * and 512 for the winner,
 * and returns the fastest configuration (mean of 3 timed runs after one
 * warm-up) and its time.  Length tables are saved before and restored after,
 * so tuning leaves them as it found them.  Synchronising.
 */
rr_status rr_batch_tune(rr_batch *batch, const float *o_tmin, const float *d_tmax, float *hits_out,
                        rr_batch_config *best, float *best_ms, void *stream);

/*
 * rr_batch_tune_cached - rr_batch_tune with its choice kept in a JSON file at
 * cache_path (host path, created when missing), so that a later process tunes
 * a batch of the same kind without timing anything.  The entry's key is the
 * GPU (name, SM count, compute capability), the batch's ray count and
 * wavefront count each rounded down to a power of two, the wavefront bits, and
 * the batch's key layout and estimate.  On a hit *best (and *best_ms, the time
 * recorded with it) come from the file and *from_cache = 1; on a miss, or an
 * entry this batch cannot run, the batch is tuned, the entry written (the file
 * is replaced by rename, its other entries kept) and *from_cache = 0.  The file
 * format: {"format": "rr-batch-tune-cache", "version": 1, "entries":
 * {"<key>": {"key_bits", "radix_bits", "trace_block", "layout", "ms"}}}; a
 * malformed file counts as empty and is rewritten.  A file that cannot be
 * written returns RR_ERR_INVALID_ARG after *best has been filled.
 * best_ms and from_cache may be NULL.
 */
rr_status rr_batch_tune_cached(rr_batch *batch, const float *o_tmin, const float *d_tmax, float *hits_out,
                               const char *cache_path, rr_batch_config *best, float *best_ms,
                               uint32_t *from_cache, void *stream);

/* ---------------------------------------------------------------- serving */

/*
 * A server answers ray-batch requests (host buffers in, closest hits out)
 * against resident scenes.  A worker thread owned by the server admits the
 * requests that have arrived, in arrival order, as far as a free stream slot
 * and the device-memory budget allow, and runs each admitted group as one
 * multi-scene batch (the rr_batch chain: keys in each request's own box, one
 * stable sort with the request number above the key bits, one trace through
 * the permutation) between its copy-in and copy-out, on the slot's stream.
 * Groups on different slots overlap on the device, and requests that arrive
 * meanwhile join the next group (continuous batching).  A request's hits do
 * not depend on which other requests share its group: each ray's closest hit
 * is computed by the same arithmetic whatever the order.
 */
typedef struct {
    uint64_t budget_bytes;     /* device memory the admitted requests may hold at once */
    uint32_t slots;            /* concurrent groups (streams), 1..64 */
    uint32_t max_batch_rays;   /* rays per group, and the largest request accepted */
    uint32_t layout;           /* rr_key_layout of every request */
    uint32_t t_source;         /* rr_t_source (Two Point; GIVEN is not served) */
    float ratio;               /* FIXED estimate ratio */
    uint32_t key_bits;         /* bits of each request's own key (capped at 64 - request bits) */
    uint32_t radix_bits;       /* 4 or 8 */
    uint32_t trace_block;      /* 128, 256 or 512; 128 lets the host-link copy kernel of RR_UPLOAD_KERNEL
                                  run beside a full trace (one warp per SM fits in its registers) */
    uint64_t reserve_bytes;    /* device memory taken from the pool and returned at creation, so
                                  that the first groups do not wait for the pool to grow (0: none;
                                  at most budget_bytes) */
    uint32_t upload;           /* how page-locked request rays go up: RR_UPLOAD_ADAPTIVE (0),
                                  RR_UPLOAD_ENGINES (1) or RR_UPLOAD_KERNEL (2) */
} rr_server_config;

/* Upload policies of rr_server_config.upload (see rr_server_submit). */
#define RR_UPLOAD_ADAPTIVE 0u /* copy engines; the copy kernel for 10 s after a slow engine upload */
#define RR_UPLOAD_ENGINES 1u  /* always the copy engines */
#define RR_UPLOAD_KERNEL 2u   /* always the library's copy kernel (page-locked, 16-byte aligned rays) */

typedef struct {
    uint64_t submit_ns;        /* steady-clock times: submission, */
    uint64_t start_ns;         /* admission (group enqueued), */
    uint64_t done_ns;          /* copy-out finished (host function ran) */
    uint32_t batch_requests;   /* requests in the group that carried this one */
    uint32_t device_flags;     /* RR_DEVERR_* flags the group's kernels recorded (0: none); when
                                  non-zero rr_server_wait returns RR_ERR_DEVICE for each request of
                                  that group, and requests of other groups are unaffected */
    uint64_t enqueued_ns;      /* steady-clock time the group's work was fully enqueued */
    float copy_in_ms;          /* device time of the group's stages (CUDA events on its stream): */
    float kernels_ms;          /*   rays up, keys + sort + trace, hits down */
    float copy_out_ms;
    float device_ms;           /* from the group's first copy to its last, waits on the device included */
    uint32_t kernel_copies;    /* 1: the group's page-locked rays were uploaded by the copy kernel */
} rr_request_times;

typedef struct {
    uint64_t batches;             /* groups run so far */
    uint64_t max_batch_requests;  /* largest group */
    uint64_t peak_reserved_bytes; /* most device memory admitted at once */
    uint64_t reserved_bytes;      /* device memory admitted now */
    uint64_t waiting;             /* requests not yet admitted */
    uint64_t engine_slowdowns;    /* slow copy-engine uploads seen (each moves uploads to the copy kernel for 10 s) */
    uint64_t kernel_copy_groups;  /* groups whose page-locked rays were uploaded by the copy kernel */
} rr_server_stats_t;

typedef struct rr_server rr_server;

/*
 * Starts the worker thread; the current device is the server's.  Device memory
 * of admitted groups comes from the device's default stream-ordered memory
 * pool, whose release threshold the server raises to budget_bytes so that
 * freed memory stays cached for the next groups.
 */
rr_status rr_server_create(const rr_server_config *cfg, rr_server **out);

/*
 * Makes a scene resident: its BVH (which must outlive the server), the box its
 * keys are quantised in, and for Two Point ADAPTIVE its length table (read by
 * the keys and updated by the trace of every request on the scene).
 */
rr_status rr_server_add_scene(rr_server *srv, const rr_bvh *bvh, rr_length_table *table,
                              const float aabb_lo[3], const float aabb_hi[3], uint32_t *scene_id);

/*
 * Queues a request of n rays (host float4 o_tmin and d_tmax; hits_host
 * receives n float4 hits in input order).  The buffers must stay valid and
 * untouched until rr_server_wait returns for the ticket.  Page-locked buffers
 * (cudaHostAlloc / cudaHostRegister) let the copies run asynchronously; rays
 * go up through the copy engines unless an upload of the last 10 s ran below
 * 40 GB/s, in which case page-locked, 16-byte aligned rays are uploaded by the
 * library's copy kernel (SM loads over the host link).  On
 * GB300 the copy engines were measured to slow down to 11-20 GB/s for ~70 ms
 * every ~0.5 s after an earlier process had used the GPU, while kernel copies
 * kept ~207 GB/s.  Returns at once.  A request whose memory alone exceeds the
 * budget is refused (RR_ERR_INVALID_ARG).
 */
rr_status rr_server_submit(rr_server *srv, uint32_t scene_id, const float *o_tmin_host,
                           const float *d_tmax_host, uint32_t n, float *hits_host, uint64_t *ticket);

/*
 * Blocks until the request is finished (its hits are in hits_host) or
 * timeout_s passes (RR_ERR_TIMEOUT, the ticket stays valid).  On return the
 * ticket is released; times (may be NULL) receives its timestamps.
 */
rr_status rr_server_wait(rr_server *srv, uint64_t ticket, double timeout_s, rr_request_times *times);

rr_status rr_server_stats(rr_server *srv, rr_server_stats_t *out);

/* Finishes every queued request, stops the worker and frees the server. */
rr_status rr_server_destroy(rr_server *srv);

/* ---------------------------------------------------------------- diagnostics */

/*
 * rr_selftest_lookback_timeout - failure-detection self-test (no paper
 * counterpart): runs one radix-sort pass over two tiles of which only the
 * second is launched, so its look-back waits on a word nothing publishes until
 * the bounded wait gives up (about 2^20 polls).  Afterwards rr_device_error
 * reports RR_DEVERR_LOOKBACK_TIMEOUT and the device stays usable.  Allocates
 * and frees its own buffers; synchronising.
 */
rr_status rr_selftest_lookback_timeout(void *stream);

/*
 * rr_stream_error - reads and clears the error word of `stream`: the RR_DEVERR_*
 * flags recorded by the library's kernels that ran on that stream (graphs of
 * rr_batch_run report to the stream they are launched on).  Asynchronous: one
 * kernel is enqueued on `stream` that writes the flags to *flags_out and
 * clears the word, so the flags cover every library call enqueued on the
 * stream before this one; read *flags_out after the stream has reached that
 * point (e.g. cudaStreamSynchronize).  flags_out: 4 bytes of device memory or
 * of page-locked host memory (cudaHostAlloc / cudaHostRegister); pageable
 * memory returns RR_ERR_INVALID_ARG.  Each device keeps 1023 stream words;
 * further streams share one extra word (their flags are then reported for
 * all of them together).
 */
rr_status rr_stream_error(void *stream, uint32_t *flags_out);

/*
 * rr_fault_inject - host-side fault injection for testing callers' error paths
 * (no paper counterpart).  spec "alloc@N", "launch@N" or "timeout@N" (N >= 1)
 * makes the N-th event of that kind from now on fail, once:
 *   alloc    a device allocation owned by the library (handles, the serving
 *            loop's group memory) fails as cudaMalloc would: RR_ERR_OOM or
 *            RR_ERR_CUDA from the call, or the request's status for a served
 *            group; nothing of that allocation's work is enqueued;
 *   launch   a launch check reports RR_ERR_CUDA (the kernels of that call may
 *            have been enqueued; its outputs are undefined);
 *   timeout  rr_server_wait or rr_pipeline_wait returns RR_ERR_TIMEOUT at once
 *            without waiting; the ticket stays valid and can be waited on again.
 * NULL or "" clears.  The environment variable RR_FAULT sets a spec at load
 * time.  No GPU fault is ever made; handles stay usable after an injected
 * failure.  A malformed spec returns RR_ERR_INVALID_ARG.
 */
rr_status rr_fault_inject(const char *spec);

/* Synchronises the device, then reads and clears every stream's error word and
 * the error word of rr_sort_noalloc, returning the union of their flags. */
rr_status rr_device_error(uint32_t *flags_out);
const char *rr_status_string(rr_status s);
/* Message of the last failing call on this thread ("" if none). */
const char *rr_last_error_message(void);
/* Number of kernels the library has launched in this process (all devices). */
uint64_t rr_kernel_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* RR_H */
