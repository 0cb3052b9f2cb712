// Library-wide plumbing: status strings, per-thread error messages, the
// per-device error word and launch accounting.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "rr_common.cuh"

namespace rr {

static thread_local std::string t_last_error;
static std::atomic<uint64_t> g_launches{0};
constexpr int kMaxDevices = 64;
static DeviceState g_dev[kMaxDevices];
static bool g_dev_ready[kMaxDevices];
static std::mutex g_dev_mutex;

rr_status fail(rr_status s, const std::string &msg) {
    t_last_error = msg;
    return s;
}

rr_status fail_cuda(cudaError_t e, const char *what) {
    t_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RR_ERR_CUDA;
}

void note_launches(uint32_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

rr_status check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail_cuda(e, what);
    if (fault_fires(Fault::Launch)) return fail(RR_ERR_CUDA, std::string(what) + ": injected launch failure");
    return RR_OK;
}

// ------------------------------------------------------------------ fault injection

static std::atomic<int> g_fault_kind{0};
static std::atomic<long long> g_fault_left{0};
static std::once_flag g_fault_env;

// Parses "alloc@N", "launch@N" or "timeout@N" (N >= 1); "" clears.
static bool parse_fault(const char *spec, int *kind, long long *n) {
    *kind = 0;
    *n = 0;
    if (!spec || !*spec) return true;
    const std::string s(spec);
    const size_t at = s.find('@');
    if (at == std::string::npos) return false;
    const std::string k = s.substr(0, at), num = s.substr(at + 1);
    if (num.empty() || num.size() > 12 || num.find_first_not_of("0123456789") != std::string::npos) return false;
    const long long v = std::stoll(num);
    if (v < 1) return false;
    if (k == "alloc") *kind = (int)Fault::Alloc;
    else if (k == "launch") *kind = (int)Fault::Launch;
    else if (k == "timeout") *kind = (int)Fault::Timeout;
    else return false;
    *n = v;
    return true;
}

static void fault_from_env() {
    std::call_once(g_fault_env, [] {
        int kind;
        long long n;
        if (parse_fault(std::getenv("RR_FAULT"), &kind, &n) && kind) {
            g_fault_left.store(n);
            g_fault_kind.store(kind);
        }
    });
}

bool fault_fires(Fault kind) {
    fault_from_env();
    if (g_fault_kind.load(std::memory_order_relaxed) != (int)kind) return false;
    if (g_fault_left.fetch_sub(1) != 1) return false;
    g_fault_kind.store(0);
    return true;
}

cudaError_t lib_malloc(void **p, size_t bytes) {
    if (fault_fires(Fault::Alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t lib_malloc_async(void **p, size_t bytes, cudaStream_t s) {
    if (fault_fires(Fault::Alloc)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, s);
}

DeviceState *device_state(rr_status *st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *st = fail_cuda(e, "cudaGetDevice");
        return nullptr;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *st = fail(RR_ERR_UNSUPPORTED, "device index out of range");
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    DeviceState &d = g_dev[dev];
    if (!g_dev_ready[dev]) {
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, dev);
        if (e != cudaSuccess) {
            *st = fail_cuda(e, "cudaGetDeviceProperties");
            return nullptr;
        }
        d.sm_count = prop.multiProcessorCount;
        d.max_smem_optin = (int)prop.sharedMemPerBlockOptin;
        // the error words and the trace queue counters live in one allocation
        const size_t words = kErrorWords + 2 * (size_t)(kQueueSlots + kCaptureQueueSlots);
        uint32_t *mem = nullptr;
        e = lib_malloc(reinterpret_cast<void **>(&mem), sizeof(uint32_t) * words);
        if (e != cudaSuccess) {
            *st = fail_cuda(e, "device state allocation");
            return nullptr;
        }
        e = cudaMemset(mem, 0, sizeof(uint32_t) * words);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(mem);
            *st = fail_cuda(e, "device state memset");
            return nullptr;
        }
        d.err = mem;
        d.counters = mem + kErrorWords;
        g_dev_ready[dev] = true;
    }
    *st = RR_OK;
    return &d;
}

uint32_t *error_word(DeviceState *d, cudaStream_t s) {
    unsigned long long id = 0;
    if (cudaStreamGetId(s, &id) != cudaSuccess) {
        cudaGetLastError();
        return d->err;
    }
    std::lock_guard<std::mutex> lock(d->mu);
    auto it = d->stream_words.find(id);
    if (it != d->stream_words.end()) return d->err + it->second;
    if (d->next_word >= kErrorWords) return d->err;  // every word taken: the shared word
    const uint32_t w = d->next_word++;
    d->stream_words.emplace(id, w);
    return d->err + w;
}

rr_status with_trace_queue(DeviceState *d, cudaStream_t s, const std::function<rr_status(uint32_t *)> &launch) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(s, &cs);
    if (e != cudaSuccess) return fail_cuda(e, "trace queue: capture status");
    std::lock_guard<std::mutex> lock(d->mu);
    if (cs != cudaStreamCaptureStatusNone) {
        const uint64_t k = d->next_capture_queue++ % kCaptureQueueSlots;
        return launch(d->counters + 2 * (kQueueSlots + k));
    }
    const uint64_t k = d->next_queue++ % kQueueSlots;
    cudaEvent_t &ev = d->queue_done[k];
    if (!ev) {
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            ev = nullptr;
            return fail_cuda(e, "trace queue: event");
        }
    } else {
        // the pair's previous launch (on any stream) must be finished first
        e = cudaStreamWaitEvent(s, ev, 0);
        if (e != cudaSuccess) return fail_cuda(e, "trace queue: wait");
    }
    const rr_status st = launch(d->counters + 2 * k);
    if (st != RR_OK) return st;
    e = cudaEventRecord(ev, s);
    return e == cudaSuccess ? RR_OK : fail_cuda(e, "trace queue: record");
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_device_error(uint32_t *flags_out) {
    if (!flags_out) return fail(RR_ERR_INVALID_ARG, "rr_device_error: NULL output");
    rr_status st;
    DeviceState *d = device_state(&st);
    if (!d) return st;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "rr_device_error: synchronise");
    uint32_t words[kErrorWords];
    e = cudaMemcpy(words, d->err, sizeof(words), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(e, "rr_device_error: read");
    e = cudaMemset(d->err, 0, sizeof(words));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return fail_cuda(e, "rr_device_error: clear");
    uint32_t v = take_noalloc_error();
    for (uint32_t w : words) v |= w;
    *flags_out = v;
    return RR_OK;
}

namespace rr {
namespace {
__global__ void take_error_kernel(uint32_t *word, uint32_t *out) { *out = atomicExch(word, 0u); }
}  // namespace

rr_status enqueue_take_error(uint32_t *word, uint32_t *out, cudaStream_t s) {
    take_error_kernel<<<1, 1, 0, s>>>(word, out);
    note_launches(1);
    return check_launch("device error word");
}

void *mapped_host_range(const void *host, size_t bytes) {
    if (!host || bytes == 0) return nullptr;
    cudaPointerAttributes a{}, b{};
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess ||
        cudaPointerGetAttributes(&b, static_cast<const char *>(host) + bytes - 1) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer || !b.devicePointer)
        return nullptr;
    if (static_cast<char *>(b.devicePointer) - static_cast<char *>(a.devicePointer) != (ptrdiff_t)(bytes - 1))
        return nullptr;
    return a.devicePointer;
}

namespace {
// One warp per block, four 16-byte words per thread per round, strided over
// the grid.  A one-warp block at no more than 32 registers fits beside a
// persistent trace kernel that fills an SM (nine 128-thread blocks at 56
// registers leave 1,024 registers), so a copy for the next group runs while
// the current group's trace does instead of waiting for it to drain; one such
// warp per SM keeps ~300 KB of host-link reads in flight.
constexpr int kCopyDepth = 4;
constexpr int kCopyWarp = 32;
__global__ void __maxnreg__(32) kernel_copy_kernel(const uint4 *__restrict__ src,
                                                   uint4 *__restrict__ dst, size_t n16) {
    const size_t stride = (size_t)gridDim.x * kCopyWarp;
    size_t i = (size_t)blockIdx.x * kCopyWarp + threadIdx.x;
    for (; i + (kCopyDepth - 1) * stride < n16; i += kCopyDepth * stride) {
        uint4 v[kCopyDepth];
#pragma unroll
        for (int k = 0; k < kCopyDepth; ++k) v[k] = src[i + k * stride];
#pragma unroll
        for (int k = 0; k < kCopyDepth; ++k) dst[i + k * stride] = v[k];
    }
    for (; i < n16; i += stride) dst[i] = src[i];
}
}  // namespace

rr_status enqueue_kernel_copy(void *dst, const void *src, size_t bytes, int sm_count, cudaStream_t s) {
    if (bytes == 0) return RR_OK;
    const size_t n16 = bytes / 16;
    const size_t want = (n16 + kCopyWarp * kCopyDepth - 1) / (kCopyWarp * kCopyDepth);  // blocks with a full round
    const uint32_t blocks = (uint32_t)std::max<size_t>(1, std::min<size_t>(want, (size_t)sm_count));
    kernel_copy_kernel<<<blocks, kCopyWarp, 0, s>>>(static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), n16);
    note_launches(1);
    return check_launch("host-link copy");
}
}  // namespace rr

extern "C" rr_status rr_stream_error(void *stream, uint32_t *flags_out) {
    if (!flags_out || !aligned(flags_out, 4)) return fail(RR_ERR_INVALID_ARG, "rr_stream_error: NULL or misaligned output");
    rr_status st;
    DeviceState *d = device_state(&st);
    if (!d) return st;
    // the flags are written by a kernel: device memory or page-locked host memory
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, flags_out) != cudaSuccess) {
        cudaGetLastError();
        return fail(RR_ERR_INVALID_ARG, "rr_stream_error: output is not device-accessible memory");
    }
    uint32_t *out = nullptr;
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        out = flags_out;
    else if (a.type == cudaMemoryTypeHost)
        out = static_cast<uint32_t *>(a.devicePointer);
    if (!out)
        return fail(RR_ERR_INVALID_ARG,
                    "rr_stream_error: output must be device memory or page-locked host memory");
    cudaStream_t s = as_stream(stream);
    return enqueue_take_error(error_word(d, s), out, s);
}

extern "C" const char *rr_status_string(rr_status s) {
    switch (s) {
        case RR_OK: return "ok";
        case RR_ERR_INVALID_ARG: return "invalid argument";
        case RR_ERR_CUDA: return "CUDA error";
        case RR_ERR_OOM: return "out of memory";
        case RR_ERR_TIMEOUT: return "device wait timed out";
        case RR_ERR_STACK: return "traversal stack overflow";
        case RR_ERR_UNSUPPORTED: return "unsupported";
        case RR_ERR_TOO_LARGE: return "size exceeds the fixed maximum of the no-allocation entry point";
        case RR_ERR_DEVICE: return "a kernel recorded a device error flag";
    }
    return "unknown status";
}

extern "C" const char *rr_last_error_message(void) { return t_last_error.c_str(); }

extern "C" rr_status rr_fault_inject(const char *spec) {
    int kind;
    long long n;
    fault_from_env();  // the environment's spec, if any, is replaced below
    if (!parse_fault(spec, &kind, &n)) return fail(RR_ERR_INVALID_ARG, "rr_fault_inject: bad spec");
    g_fault_kind.store(0);
    g_fault_left.store(n);
    g_fault_kind.store(kind);
    return RR_OK;
}

extern "C" uint64_t rr_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
