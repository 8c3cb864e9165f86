// Shared helpers of libtacaw: status handling, complex arithmetic, launch
// checks.  Host-side state is limited to a thread-local error message.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>

#include "../../include/tacaw.h"

namespace tacaw {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define TACAW_REQUIRE(cond, code, ...)       \
    do {                                     \
        if (!(cond)) {                       \
            ::tacaw::set_error(__VA_ARGS__); \
            return (code);                   \
        }                                    \
    } while (0)

#define TACAW_CUDA_CHECK(expr)                                                         \
    do {                                                                               \
        cudaError_t err__ = (expr);                                                    \
        if (err__ != cudaSuccess) {                                                    \
            ::tacaw::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(err__), \
                               __FILE__, __LINE__);                                    \
            return TACAW_ECUDA;                                                        \
        }                                                                              \
    } while (0)

#define TACAW_LAUNCH_CHECK() TACAW_CUDA_CHECK(cudaGetLastError())

// Device status (status.cu).  fault_injected(kind): `kind` is listed in the
// comma-separated environment variable TACAW_FAULT (host-side fault injection
// for tests: "launch" fails every entry point before its first enqueue,
// "symbol" fails device-symbol lookups, "timeout" makes tacaw_status report a
// timeout); inject_launch_fault returns TACAW_ECUDA with a message when
// "launch" is set.  device_symbol: device address of a __device__ variable in
// the current context.  timeout_flag: address of the sticky flag that bounded
// device waits set when they give up.  wait_polls: the poll limit of bounded
// waits set by tacaw_set_wait_limit, or `dflt`.
bool fault_injected(const char* kind);
int inject_launch_fault(const char* fn);
int device_symbol(const void* symbol, void** out, const char* fn);
int timeout_flag(int** out, const char* fn);
uint32_t wait_polls(uint32_t dflt);

// A kernel's bounded waits: the status flag to set when one gives up, and the
// number of polls before it does.
struct WaitCtl {
    int* flag;
    uint32_t polls;
};

// Workspace carving: aligned sub-buffers of a caller-provided block.
// Planck and Boltzmann constants in meV fs and meV / K (exact SI values).
constexpr double kPlanckMeVfs = 6.62607015e-34 / 1.602176634e-19 * 1e3 * 1e15;
constexpr double kBoltzmannMeVK = 1.380649e-23 / 1.602176634e-19 * 1e3;

struct Carver {
    char* base;
    size_t off = 0;
    explicit Carver(void* b) : base(static_cast<char*>(b)) {}
    template <typename T>
    T* take(size_t count, size_t align = 256) {
        off = (off + align - 1) / align * align;
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) / 256 * 256; }
};

// Raise a kernel's dynamic shared-memory limit once per device (multislice.cu).
cudaError_t ensure_smem(const void* kernel, int bytes);
// Blocks of `kernel` resident on the whole device at once (occupancy times SM count).
cudaError_t resident_blocks(const void* kernel, int threads, int smem, int* out);

// Beam constants (textbook relativistic values, CODATA 2018).
void beam_constants(double kev, double* lambda_A, double* sigma_e);

inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// ---------------------------------------------------------------- complex
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    return make_float2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) {
    return make_float2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) {
    return make_float2(a.x * s, a.y * s);
}

// L2 prefetch hint for [p, p + bytes): p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Bulk asynchronous copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) from global to this block's shared memory, completing on `bar`
// (an mbarrier in shared memory that expects the bytes).
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
                 "l"(src), "r"(bytes), "r"(static_cast<uint32_t>(__cvta_generic_to_shared(bar)))
                 : "memory");
}

// Orders this thread's (and, after a block barrier, the block's) earlier
// ordinary shared-memory accesses before later asynchronous-proxy writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// exp(i x) = cos x + i sin x for the transmission phase sigma_e v.  The phase
// is small in practice, so it uses truncated Taylor series evaluated by
// Horner's rule: for |x| <= 0.25 sin to x^7 and cos to x^8, for |x| <= 0.5 sin
// to x^9 and cos to x^10 (truncation below 2e-11 in both ranges, i.e. far
// under FP32 rounding); larger phases fall back to sincosf.  The result for x
// depends on x alone.
__device__ __forceinline__ void phase_sincos_small(float x, float* s, float* c) {   // |x| <= 0.25
    const float x2 = x * x;
    const float ps = fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 5040.f, 1.f / 120.f), -1.f / 6.f), 1.f);
    *s = x * ps;
    *c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 40320.f, -1.f / 720.f), 1.f / 24.f), -0.5f), 1.f);
}

__device__ __forceinline__ void phase_sincos(float x, float* s, float* c) {
    const float ax = fabsf(x);
    if (ax <= 0.25f) {
        phase_sincos_small(x, s, c);
    } else if (ax <= 0.5f) {
        const float x2 = x * x;
        const float ps = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, 1.f / 362880.f, -1.f / 5040.f), 1.f / 120.f),
                                       -1.f / 6.f), 1.f);
        *s = x * ps;
        *c = fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, fmaf(x2, -1.f / 3628800.f, 1.f / 40320.f), -1.f / 720.f),
                                        1.f / 24.f), -0.5f), 1.f);
    } else {
        sincosf(x, s, c);
    }
}

// v[m] *= exp(i x[m]) for a thread's E values: one test of the largest phase
// selects straight-line code when every phase is small (the same result for
// each value as phase_sincos, which the other branch calls).
template <int E>
__device__ __forceinline__ void transmit(float2 (&v)[E], const float (&x)[E]) {
    float mx = 0.f;
#pragma unroll
    for (int m = 0; m < E; ++m) mx = fmaxf(mx, fabsf(x[m]));
    if (mx <= 0.25f) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            float sn, cs;
            phase_sincos_small(x[m], &sn, &cs);
            v[m] = cmul(v[m], make_float2(cs, sn));
        }
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            float sn, cs;
            phase_sincos(x[m], &sn, &cs);
            v[m] = cmul(v[m], make_float2(cs, sn));
        }
    }
}

}  // namespace tacaw
