// Internal definitions shared by the translation units of librr.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <mutex>
#include <string>
#include <unordered_map>

#include "../../include/rr.h"

namespace rr {

constexpr uint32_t kMiss = 0xFFFFFFFFu;
constexpr uint32_t kTableCells = 1u << 20;

// ------------------------------------------------------------------ host helpers

// Records `msg` as this thread's last error message and returns `s`.
rr_status fail(rr_status s, const std::string &msg);
rr_status fail_cuda(cudaError_t e, const char *what);

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Per-device state: error words, trace work-queue counters, cached properties.
//
// Error words: kernels OR RR_DEVERR_* flags into the word of the stream they
// run on (word 0 is shared by the streams beyond the first kErrorWords - 1),
// so rr_stream_error can tell one stream's failures from another's.
//
// Trace work queues: a persistent trace launch needs a pair of counter words
// that no concurrent launch shares (the last block resets them).  Launches
// take pairs round-robin from kQueueSlots; each pair's last launch records an
// event, and the next launch that takes the pair waits for it on its own
// stream, so two launches can never share a pair at the same time.  Launches
// under stream capture take pairs from a separate ring of kCaptureQueueSlots
// without events (a captured trace must not run concurrently with itself).
constexpr uint32_t kErrorWords = 1024;
constexpr uint32_t kQueueSlots = 2048;
constexpr uint32_t kCaptureQueueSlots = 1024;

struct DeviceState {
    uint32_t *err = nullptr;       // kErrorWords device words of RR_DEVERR_* flags
    uint32_t *counters = nullptr;  // 2 * (kQueueSlots + kCaptureQueueSlots) queue words (zero at rest)
    int sm_count = 0;
    int max_smem_optin = 0;
    std::mutex mu;
    std::unordered_map<unsigned long long, uint32_t> stream_words;  // stream id -> error word
    uint32_t next_word = 1;
    cudaEvent_t queue_done[kQueueSlots] = {};
    uint64_t next_queue = 0, next_capture_queue = 0;
};

// Returns the state of the current device (initialised on first use) or null.
DeviceState *device_state(rr_status *st);

// The error word of stream `s` on this device (never null).
uint32_t *error_word(DeviceState *d, cudaStream_t s);

// Runs `launch(queue)` with a trace work-queue pair no concurrent launch
// holds, and records the pair's completion event after it (see above).
rr_status with_trace_queue(DeviceState *d, cudaStream_t s, const std::function<rr_status(uint32_t *)> &launch);

// Reads and clears the error word of rr_sort_noalloc (defined with it).
uint32_t take_noalloc_error();

// Enqueues on `s`: *out = the flags of `word`, and `word` cleared.  out:
// device-accessible (device or page-locked host memory).
rr_status enqueue_take_error(uint32_t *word, uint32_t *out, cudaStream_t s);

// Device address of the page-locked host range [host, host + bytes), or null
// when either end is not page-locked, mapped host memory.
void *mapped_host_range(const void *host, size_t bytes);

// Copies `bytes` (a multiple of 16) between two device-accessible addresses
// (device memory or page-locked host memory) with a kernel: SM loads and
// stores over the host link instead of the copy engines, which the driver
// may be using for its own work.  Enqueued on `s`.
rr_status enqueue_kernel_copy(void *dst, const void *src, size_t bytes, int sm_count, cudaStream_t s);

// Host-side fault injection (rr_fault_inject, or RR_FAULT in the environment):
// returns true exactly once, at the N-th call of that kind after the spec was
// set.  Kinds: library device allocations, launch checks, bounded host waits.
enum class Fault { Alloc = 1, Launch = 2, Timeout = 3 };
bool fault_fires(Fault kind);

// Library-owned device allocations (an injected Alloc fault fails them).
cudaError_t lib_malloc(void **p, size_t bytes);
cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Counts kernel launches made by the library.
void note_launches(uint32_t k);

// A kernel launch check: returns RR_OK or RR_ERR_CUDA with the message recorded.
rr_status check_launch(const char *what);

// Index checks of the bounds-checked build (compiled with RR_CHECKED, library
// librr_checked.so): an index outside its buffer records RR_DEVERR_BAD_INDEX
// in the error word and the access is skipped.  Compiled out otherwise.
#ifdef RR_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

#ifdef __CUDACC__
__device__ __forceinline__ bool index_ok(uint32_t i, uint32_t n, uint32_t *err) {
    if (!kChecked || i < n) return true;
    atomicOr(err, RR_DEVERR_BAD_INDEX);
    return false;
}
#endif

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
inline bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
inline bool overlaps(const void *a, size_t na, const void *b, size_t nb) {
    uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// ------------------------------------------------------------------ library-owned objects

struct Box {
    float lo[3];
    float hi[3];
};

}  // namespace rr

struct rr_length_table {
    int device;
    rr::Box box;
    float E;                 // largest extent of box
    unsigned long long *cells;  // 2^20 x {sum (u64), count (u64 slot, low 32 bits used)}
};

// Compressed 8-wide BVH node (80 bytes, five 16-byte loads).
//   A child box is p + q * 2^(e - 127) per axis: q in [qlo, qhi] (8 bits each),
//   widened by one step on every side of the child it bounds.
//   imask: bit s set when slot s holds an inner child.  Inner children are
//   stored consecutively in slot order: the child in slot s is node
//   child_base + popc(imask & ((1 << s) - 1)).
//   tribits: four bits per slot; leaf slot s holds `count` (1..4) triangles,
//   marked by the low `count` bits of nibble s.  Leaf triangles are stored
//   consecutively in slot order: the triangle of bit b is number
//   tri_base + popc(tribits & ((1 << b) - 1)) of the BVH-ordered array.
//   valid: bit s set when slot s is used (inner child or leaf).
struct alignas(16) RRNode8 {
    float px, py, pz;
    uint8_t ex, ey, ez, imask;
    uint32_t child_base;
    uint32_t tri_base;
    uint32_t tribits;
    uint32_t valid;
    uint8_t qlo_x[8];
    uint8_t qlo_y[8];
    uint8_t qlo_z[8];
    uint8_t qhi_x[8];
    uint8_t qhi_y[8];
    uint8_t qhi_z[8];
};
static_assert(sizeof(RRNode8) == 80, "node layout");

// Triangle in BVH order: v0, e1 = v1 - v0, e2 = v2 - v0; w of the first float4
// holds the original triangle id.
struct alignas(16) RRTri {
    float4 v0_id;
    float4 e1;
    float4 e2;
};

struct rr_bvh {
    int device;
    RRNode8 *nodes;   // device
    RRTri *tris;      // device
    float4 *planes;   // device, two per triangle (normal as hi + lo floats)
    uint32_t n_nodes;
    uint32_t n_tris;
    uint32_t root_is_leaf;  // scenes of 1..4 triangles: no inner node, the root is one leaf
    uint32_t root_leaf_ref;
    rr_bvh_info info;
};
