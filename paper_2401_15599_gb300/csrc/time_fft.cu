// Temporal transform on the natural energy grid as an FFT over time (the
// HBM-bound alternative to the complex GEMM of the DFT matrix, for Eq. (9)).
//
// On the natural grid E_k = h (k - T/2) / (T dt), so E_k t_n / hbar =
// 2 pi (k - T/2) n / T and
//   Phi(q, E_k) = sum_n A(q, t_n) exp(-2 pi i (k - T/2) n / T) = FFT_T[A](q)[(k - T/2) mod T],
//   I(q, E_k)   = |Phi|^2 / T^2   (times the Kubo factor when asked).
// One block takes W columns q of psi [T][nq] (time-major) and all T samples:
//  1. loads them (thread (c, t) holds times t + TPT m of column c), forms the
//     time mean m_q as an unevaluated sum hi + lo of two floats (pairwise
//     two-sums over each thread's samples with their errors kept, then
//     error-free sums in a fixed-order tree over the block: FP64 arithmetic
//     would run on this GPU's slow FP64 pipe for every sample),
//     I_el = |m_q|^2 in FP64 and A = (psi - m_hi) - m_lo, one rounding away from
//     the exact difference;
//  2. runs the length-T FP32 Stockham FFT (one shared buffer of W x T values);
//  3. writes |Phi|^2 / T^2 in ascending energy through shared memory, so that
//     each row I[q][.] is stored with coalesced writes.
// Each exit wave is read once and each intensity written once.

#include "common.cuh"
#include "fft.cuh"

namespace tacaw {

int launch_kubo(float* kubo, const double* omega, int n_t, int n_w, double dt, double beta,
                cudaStream_t st);
int launch_normalize(float* out, size_t n, double* i_el_user, const double* i_el, int nq,
                     double* partial, double* total, cudaStream_t st);
size_t normalize_ws_doubles();

namespace {

// Knuth's two-sum: s + e == a + b exactly (every operation an explicit
// round-to-nearest, so no contraction changes it).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (h2, l2) for unevaluated sums of two floats
__device__ __forceinline__ void df_add(float& hi, float& lo, float h2, float l2) {
    float s, e;
    two_sum(hi, h2, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, l2));
    two_sum(s, e, hi, lo);
}

// (hi + lo) / n as (qh, ql)
__device__ __forceinline__ void df_div(float hi, float lo, float n, float& qh, float& ql) {
    qh = __fdiv_rn(hi, n);
    const float r = __fmaf_rn(-qh, n, hi);          // exact remainder hi - qh n
    ql = __fdiv_rn(__fadd_rn(r, lo), n);
}

template <int T>
struct TfCfg {
    static constexpr int E = fft::Plan<T>::E;
    static constexpr int TPT = T / E;
    static constexpr int W = (1024 / TPT) < 16 ? (1024 / TPT) : 16;   // columns per block
    static constexpr int THREADS = W * TPT;
    static constexpr int WARPS = THREADS / 32;
    static constexpr size_t SMEM = ((size_t)W * T + fft::TwSize<T>::value) * sizeof(float2);
};

template <int T>
__global__ void tf_twiddle_kernel(float2* tw) {
    fft::fill_twiddles<T>(tw, threadIdx.x + blockIdx.x * blockDim.x, blockDim.x * gridDim.x);
}

template <int T>
__global__ void __launch_bounds__(TfCfg<T>::THREADS)
time_fft_power_kernel(const float2* __restrict__ psi, size_t ld, int nq, const double2* __restrict__ psi_sum,
                      const float2* __restrict__ tw_g, const float* __restrict__ kubo, float scale,
                      float* __restrict__ out, double* __restrict__ i_el) {
    using Cfg = TfCfg<T>;
    constexpr int E = Cfg::E, TPT = Cfg::TPT, W = Cfg::W;
    extern __shared__ float2 smem[];
    __shared__ float4 part[Cfg::WARPS][W];          // (re hi, re lo, im hi, im lo)
    __shared__ float4 mean[W];
    float2* buf = smem;
    float2* tw = smem + W * T;
    for (int i = threadIdx.x; i < fft::TwSize<T>::value; i += blockDim.x) tw[i] = __ldg(tw_g + i);
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int q0 = blockIdx.x * W;
    const int q = q0 + c;
    const bool valid = q < nq;

    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = valid ? __ldcs(psi + (size_t)(t + TPT * m) * ld + q) : make_float2(0.f, 0.f);

    // time mean of each column as hi + lo: per thread, then the lanes of the
    // same column in a warp (lane bits above log2 W), then the warps in order
    if (psi_sum == nullptr) {
        // the thread's own E samples by a pairwise tree of two-sums whose
        // rounding errors are summed apart
        float2 ps[E];
        float er = 0.f, ei = 0.f;
#pragma unroll
        for (int m = 0; m < E; ++m) ps[m] = v[m];
#pragma unroll
        for (int n = E; n > 1; n = (n + 1) / 2)
#pragma unroll
            for (int m = 0; m < n / 2; ++m) {
                float e;
                two_sum(ps[m].x, ps[m + (n + 1) / 2].x, ps[m].x, e);
                er = __fadd_rn(er, e);
                two_sum(ps[m].y, ps[m + (n + 1) / 2].y, ps[m].y, e);
                ei = __fadd_rn(ei, e);
            }
        float rh, rl, ih, il;
        two_sum(ps[0].x, er, rh, rl);
        two_sum(ps[0].y, ei, ih, il);
#pragma unroll
        for (int o = 16; o >= W; o >>= 1) {
            df_add(rh, rl, __shfl_xor_sync(0xffffffffu, rh, o), __shfl_xor_sync(0xffffffffu, rl, o));
            df_add(ih, il, __shfl_xor_sync(0xffffffffu, ih, o), __shfl_xor_sync(0xffffffffu, il, o));
        }
        if ((threadIdx.x & 31) < W) part[threadIdx.x >> 5][c] = make_float4(rh, rl, ih, il);
        __syncthreads();
        if (threadIdx.x < W) {
            float4 a = part[0][threadIdx.x];
            for (int w = 1; w < Cfg::WARPS; ++w) {
                const float4 b = part[w][threadIdx.x];
                df_add(a.x, a.y, b.x, b.y);
                df_add(a.z, a.w, b.z, b.w);
            }
            float4 mm;
            df_div(a.x, a.y, (float)T, mm.x, mm.y);
            df_div(a.z, a.w, (float)T, mm.z, mm.w);
            mean[threadIdx.x] = mm;
        }
    } else if (threadIdx.x < W) {
        const double2 s = q0 + (int)threadIdx.x < nq ? psi_sum[q0 + threadIdx.x] : make_double2(0.0, 0.0);
        const double mr = s.x / T, mi = s.y / T;
        const float rh = (float)mr, ih = (float)mi;
        mean[threadIdx.x] = make_float4(rh, (float)(mr - rh), ih, (float)(mi - ih));
    }
    __syncthreads();
    const float4 mq = mean[c];
    if (t == 0 && valid && i_el) {
        const double mr = (double)mq.x + (double)mq.y, mi = (double)mq.z + (double)mq.w;
        i_el[q] = mr * mr + mi * mi;
    }
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = make_float2(__fsub_rn(__fsub_rn(v[m].x, mq.x), mq.y), __fsub_rn(__fsub_rn(v[m].y, mq.z), mq.w));

    fft::transform<T, false>(v, buf, buf, t, tw, fft::ColLayout<W>{c});

    // |Phi_p|^2 / T^2 at energy index k = (p + T/2) mod T, staged as [W][T] floats
    __syncthreads();
    float* pw = reinterpret_cast<float*>(buf);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int p = t + TPT * m;
        const int k = (p + T / 2) % T;
        float a = (v[m].x * v[m].x + v[m].y * v[m].y) * scale;
        if (kubo) a *= __ldg(kubo + k);
        pw[c * T + k] = a;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W * T; i += blockDim.x) {
        const int cc = i / T, k = i % T;
        if (q0 + cc < nq) __stcs(out + (size_t)(q0 + cc) * T + k, pw[i]);
    }
}

template <int T>
int launch_time_fft(const float2* psi, size_t ld, int nq, const double2* psi_sum, float2* tw, const float* kubo,
                    float* out, double* i_el, cudaStream_t st) {
    using Cfg = TfCfg<T>;
    tf_twiddle_kernel<T><<<4, 256, 0, st>>>(tw);
    TACAW_LAUNCH_CHECK();
    TACAW_CUDA_CHECK(ensure_smem((const void*)time_fft_power_kernel<T>, (int)Cfg::SMEM));
    const float scale = (float)(1.0 / ((double)T * (double)T));
    time_fft_power_kernel<T><<<(nq + Cfg::W - 1) / Cfg::W, Cfg::THREADS, Cfg::SMEM, st>>>(
        psi, ld, nq, psi_sum, tw, kubo, scale, out, i_el);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace

bool time_fft_size_supported(int n) {
    return n == 64 || n == 128 || n == 256 || n == 384 || n == 512 || n == 768 || n == 1024 || n == 2048 ||
           n == 4096;
}

size_t time_fft_ws_bytes(int nq, int n_t) {
    Carver cv(nullptr);
    cv.take<float2>(n_t);              // twiddles (TwSize < n_t for every plan)
    cv.take<float>(n_t);               // Kubo factors
    cv.take<double>(nq);               // I_el when the caller passes none
    cv.take<double>(normalize_ws_doubles());
    return cv.bytes();
}

int time_fft_spectrum_run(int nq, int n_t, double dt_fs, const float2* psi, size_t ld, const double2* psi_sum,
                          float* out, double* i_el, int flags, double beta, void* ws, cudaStream_t st) {
    Carver cv(ws);
    float2* tw = cv.take<float2>(n_t);
    float* kubo = cv.take<float>(n_t);
    double* el = cv.take<double>(nq);
    double* red = cv.take<double>(normalize_ws_doubles());
    double* iel = i_el ? i_el : el;
    const bool use_kubo = (flags & TACAW_KUBO) != 0;
    if (use_kubo) {
        int rc = launch_kubo(kubo, nullptr, n_t, n_t, dt_fs, beta, st);
        if (rc) return rc;
    }
    const float* kb = use_kubo ? kubo : nullptr;
    int rc = TACAW_EUNSUPPORTED;
    switch (n_t) {
        case 64: rc = launch_time_fft<64>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 128: rc = launch_time_fft<128>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 256: rc = launch_time_fft<256>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 384: rc = launch_time_fft<384>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 512: rc = launch_time_fft<512>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 768: rc = launch_time_fft<768>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 1024: rc = launch_time_fft<1024>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 2048: rc = launch_time_fft<2048>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        case 4096: rc = launch_time_fft<4096>(psi, ld, nq, psi_sum, tw, kb, out, iel, st); break;
        default: set_error("tacaw_spectrum: T = %d has no time-FFT plan", n_t); return TACAW_EUNSUPPORTED;
    }
    if (rc) return rc;
    if (flags & TACAW_NORMALIZE) {
        rc = launch_normalize(out, (size_t)nq * n_t, i_el, iel, nq, red, red + normalize_ws_doubles() - 1, st);
        if (rc) return rc;
    }
    return TACAW_OK;
}

}  // namespace tacaw
