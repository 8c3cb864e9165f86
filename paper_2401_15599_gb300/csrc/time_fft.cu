// Temporal transform on the natural energy grid as an FFT over time (the
// HBM-bound alternative to the complex GEMM of the DFT matrix, for Eq. (9)).
//
// On the natural grid E_k = h (k - T/2) / (T dt), so E_k t_n / hbar =
// 2 pi (k - T/2) n / T and
//   Phi(q, E_k) = sum_n A(q, t_n) exp(-2 pi i (k - T/2) n / T) = FFT_T[A](q)[(k - T/2) mod T],
//   I(q, E_k)   = |Phi|^2 / T^2   (times the Kubo factor when asked).
// One block takes W columns q of psi [T][nq] (time-major) and all T samples:
//  1. loads them (thread (c, t) holds times t + TPT m of column c), forms the
//     FP64 time mean m_q (fixed-order tree over the block), I_el = |m_q|^2 and
//     A = psi - m_q in FP64 rounded to float;
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
    __shared__ double2 part[Cfg::WARPS][W];
    __shared__ double2 mean[W];
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

    // FP64 time mean of each column: per thread, then the lanes of the same
    // column in a warp (lane bits above log2 W), then the warps in order
    if (psi_sum == nullptr) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            re += (double)v[m].x;
            im += (double)v[m].y;
        }
#pragma unroll
        for (int o = 16; o >= W; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if ((threadIdx.x & 31) < W) part[threadIdx.x >> 5][c] = make_double2(re, im);
        __syncthreads();
        if (threadIdx.x < W) {
            double sr = 0.0, si = 0.0;
            for (int w = 0; w < Cfg::WARPS; ++w) {
                sr += part[w][threadIdx.x].x;
                si += part[w][threadIdx.x].y;
            }
            mean[threadIdx.x] = make_double2(sr / T, si / T);
        }
    } else if (threadIdx.x < W) {
        const double2 s = q0 + (int)threadIdx.x < nq ? psi_sum[q0 + threadIdx.x] : make_double2(0.0, 0.0);
        mean[threadIdx.x] = make_double2(s.x / T, s.y / T);
    }
    __syncthreads();
    const double2 mq = mean[c];
    if (t == 0 && valid && i_el) i_el[q] = mq.x * mq.x + mq.y * mq.y;
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[m] = make_float2((float)((double)v[m].x - mq.x), (float)((double)v[m].y - mq.y));

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
