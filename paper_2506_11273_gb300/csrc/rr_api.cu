// Library-wide plumbing: status strings, per-thread error messages, the
// per-device error word and launch accounting.
#include <cstdio>
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
    return RR_OK;
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
        // the error word and the trace queue counters live in one allocation
        uint32_t *mem = nullptr;
        e = cudaMalloc(&mem, sizeof(uint32_t) * (64 + kCounterPool));
        if (e != cudaSuccess) {
            *st = fail_cuda(e, "device state allocation");
            return nullptr;
        }
        e = cudaMemset(mem, 0, sizeof(uint32_t) * (64 + kCounterPool));
        if (e != cudaSuccess) {
            cudaFree(mem);
            *st = fail_cuda(e, "device state memset");
            return nullptr;
        }
        d.err = mem;
        d.counters = mem + 64;
        g_dev_ready[dev] = true;
    }
    *st = RR_OK;
    return &d;
}

}  // namespace rr

using namespace rr;

extern "C" rr_status rr_device_error(uint32_t *flags_out) {
    if (!flags_out) return fail(RR_ERR_INVALID_ARG, "rr_device_error: NULL output");
    rr_status st;
    DeviceState *d = device_state(&st);
    if (!d) return st;
    uint32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, d->err, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail_cuda(e, "rr_device_error: read");
    e = cudaMemset(d->err, 0, sizeof(uint32_t));
    if (e != cudaSuccess) return fail_cuda(e, "rr_device_error: clear");
    *flags_out = v;
    return RR_OK;
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
    }
    return "unknown status";
}

extern "C" const char *rr_last_error_message(void) { return t_last_error.c_str(); }

extern "C" uint64_t rr_kernel_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
