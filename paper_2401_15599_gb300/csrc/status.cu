// Device status of libtacaw: the sticky per-device flag that bounded device
// waits set when they give up, the host-settable wait limit, device-symbol
// lookup keyed by CUDA context, and host-side fault injection for tests.
//
// Kernels with bounded waits (the staged row pass of the multislice, the
// tensor-core temporal transform) receive the flag's device address and set
// it when a wait gives up; tacaw_status() reads and clears it.  No kernel
// traps or spins without a bound.

#include <cuda.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace tacaw {

namespace {

// Set to 1 by a bounded device wait that gave up; cleared by tacaw_status.
__device__ int g_wait_timeout;

std::atomic<long long> g_wait_limit{-1};   // < 0: each kernel's default

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename F>
F driver_fn(const char* name, int version) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, version, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return reinterpret_cast<F>(p);
    return nullptr;
}

// Unique id of the current CUDA context (never reused within a process), or
// 0 when there is none or the driver cannot say.
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 2000);
    static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

}  // namespace

bool fault_injected(const char* kind) {
    const char* env = getenv("TACAW_FAULT");
    if (env == nullptr || *env == '\0') return false;
    const size_t n = strlen(kind);
    for (const char* p = env; *p;) {
        const char* end = strchr(p, ',');
        const size_t len = end ? (size_t)(end - p) : strlen(p);
        if (len == n && strncmp(p, kind, n) == 0) return true;
        if (!end) break;
        p = end + 1;
    }
    return false;
}

int inject_launch_fault(const char* fn) {
    if (!fault_injected("launch")) return TACAW_OK;
    set_error("%s: injected launch failure (TACAW_FAULT=launch)", fn);
    return TACAW_ECUDA;
}

// Device address of a __device__ variable of this library in the current
// context.  The address belongs to the context, not to the device ordinal, so
// the cache is keyed by the context's unique id: a context created after a
// device reset gets a fresh lookup.  Without a current context (or a driver
// that cannot name it) the address is looked up on every call.
int device_symbol(const void* symbol, void** out, const char* fn) {
    if (fault_injected("symbol")) {
        set_error("%s: injected symbol lookup failure (TACAW_FAULT=symbol)", fn);
        return TACAW_ECUDA;
    }
    static std::mutex mu;
    static std::map<std::pair<unsigned long long, const void*>, void*> cache;
    const unsigned long long id = current_context_id();
    if (id != 0) {
        std::lock_guard<std::mutex> lock(mu);
        auto it = cache.find({id, symbol});
        if (it != cache.end()) {
            *out = it->second;
            return TACAW_OK;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, symbol);
    if (e != cudaSuccess || p == nullptr) {
        set_error("%s: cudaGetSymbolAddress failed: %s", fn, cudaGetErrorString(e));
        return TACAW_ECUDA;
    }
    const unsigned long long id2 = id != 0 ? id : current_context_id();   // the lookup may create it
    if (id2 != 0) {
        std::lock_guard<std::mutex> lock(mu);
        cache[{id2, symbol}] = p;
    }
    *out = p;
    return TACAW_OK;
}

int timeout_flag(int** out, const char* fn) {
    void* p = nullptr;
    const int rc = device_symbol((const void*)&g_wait_timeout, &p, fn);
    *out = static_cast<int*>(p);
    return rc;
}

uint32_t wait_polls(uint32_t dflt) {
    const long long v = g_wait_limit.load(std::memory_order_relaxed);
    if (v < 0) return dflt;
    return v > 0xffffffffLL ? 0xffffffffu : (uint32_t)v;
}

}  // namespace tacaw

using namespace tacaw;

extern "C" int tacaw_set_wait_limit(int64_t polls) {
    clear_error();
    g_wait_limit.store(polls < 0 ? -1 : (long long)polls, std::memory_order_relaxed);
    return TACAW_OK;
}

extern "C" int tacaw_status(void* stream) {
    clear_error();
    const char* fn = "tacaw_status";
    if (fault_injected("timeout")) {
        set_error("%s: injected device wait timeout (TACAW_FAULT=timeout)", fn);
        return TACAW_ETIMEOUT;
    }
    int* flag = nullptr;
    int rc = timeout_flag(&flag, fn);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    int host = 0;
    TACAW_CUDA_CHECK(cudaMemcpyAsync(&host, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    TACAW_CUDA_CHECK(cudaStreamSynchronize(st));
    if (host == 0) return TACAW_OK;
    TACAW_CUDA_CHECK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    TACAW_CUDA_CHECK(cudaStreamSynchronize(st));
    set_error("%s: a bounded device wait gave up; the results of the calls enqueued since the last "
              "tacaw_status are incomplete", fn);
    return TACAW_ETIMEOUT;
}
