// Temporal transform of the exit waves into I(q, E) (Eq. (9): the spectrum
// is |phi_MD(q, E)|^2 by the convolution theorem, with the Kubo factor of
// Eq. (8) and the fractional-intensity normalisation after Eq. (9)).
//
//   m_q = (1/T) sum_n psi(q, t_n)                    FP64, snapshot order
//   A(q, t_n) = psi(q, t_n) - m_q                    FP64 subtract, rounded to float
//   Phi(q, E_k) = sum_n A(q, t_n) E(t_n, E_k),  E = exp(-i E_k t_n / hbar)
//   I(q, E_k) = |Phi|^2 / T^2 (* Kubo factor),  I_el(q) = |m_q|^2
//
// The transform is a complex GEMM [nq x T] x [T x n_omega].  This file holds
// the FP32 SIMT form; the DFT matrix is built in FP64 on the device (exact
// integer phase reduction on the natural grid) and rounded once to float.

#include "common.cuh"

namespace tacaw {

namespace {

// CODATA 2018: h in meV*fs and the Boltzmann constant in meV/K.

__global__ void time_sum_kernel(const float2* __restrict__ psi, size_t ld, double2* __restrict__ sum,
                                int n_t, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < n_t; ++t) {
        const float2 v = __ldg(psi + (size_t)t * ld + q);
        re += (double)v.x;
        im += (double)v.y;
    }
    sum[q] = make_double2(re, im);
}

// A = psi - sum / T in FP64, rounded to float; also I_el = |sum / T|^2.
__global__ void centre_kernel(const float2* __restrict__ psi, size_t ld, const double2* __restrict__ sum,
                              float2* __restrict__ a, double* __restrict__ i_el, int n_t, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (q >= nq) return;
    const double2 s = sum[q];
    const double inv_t = 1.0 / (double)n_t;
    const double mr = s.x * inv_t, mi = s.y * inv_t;
    const float2 v = __ldg(psi + (size_t)t * ld + q);
    a[(size_t)t * nq + q] = make_float2((float)((double)v.x - mr), (float)((double)v.y - mi));
    if (t == 0 && i_el) i_el[q] = mr * mr + mi * mi;
}

// E[n][k] = exp(-i E_k t_n / hbar) = exp(-2 pi i E_k t_n / h).
// Natural grid: E_k = h (k - T/2) / (T dt) -> phase = -2 pi ((k - T/2) n mod T) / T.
// Explicit grid: cycles = E_k t_n / h in FP64, reduced to its fractional part.
// kubo[k] = beta E_k / (1 - exp(-beta E_k)) (1 at E = 0) when requested.
__global__ void dft_table_kernel(float2* __restrict__ e, float* __restrict__ kubo,
                                 const double* __restrict__ omega, int n_t, int n_w, double dt,
                                 double beta, int t0 = 0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (k >= n_w) return;
    double s, c, ek;
    if (omega == nullptr) {
        const long long kk = (long long)k - n_t / 2;
        long long r = (kk * n) % n_t;
        if (r < 0) r += n_t;
        sincospi(-2.0 * (double)r / (double)n_t, &s, &c);
        ek = (double)kk * kPlanckMeVfs / ((double)n_t * dt);
    } else {
        ek = omega[k];
        const double cyc = ek * ((double)(t0 + n) * dt) / kPlanckMeVfs;
        const double frac = cyc - rint(cyc);
        sincospi(-2.0 * frac, &s, &c);
    }
    e[(size_t)n * n_w + k] = make_float2((float)c, (float)s);
    if (n == 0 && kubo) {
        const double be = beta * ek;
        kubo[k] = (be == 0.0) ? 1.0f : (float)(be / (-expm1(-be)));
    }
}

// I[q][k] = |sum_n A[n][q] E[n][k]|^2 * scale (* kubo[k]), FP32 SIMT; with
// phi_acc given, Phi itself is added to phi_acc[q][k] instead (time-chunked
// accumulation, tacaw_spectrum_accumulate).
constexpr int BM = 64, BN = 64, BK = 16;
__global__ void __launch_bounds__(256)
cgemm_power_kernel(const float2* __restrict__ a, const float2* __restrict__ e,
                   const float* __restrict__ kubo, float* __restrict__ out, int nq, int n_t,
                   int n_w, float scale, float2* __restrict__ phi_acc = nullptr) {
    __shared__ float2 as[BK][BM];
    __shared__ float2 es[BK][BN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int w0 = blockIdx.x * BN, q0 = blockIdx.y * BM;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int k0 = 0; k0 < n_t; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = threadIdx.x + 256 * i;
            const int kk = idx / BM, mm = idx % BM;
            const int n = k0 + kk;
            as[kk][mm] = (n < n_t && q0 + mm < nq) ? __ldg(a + (size_t)n * nq + q0 + mm)
                                                   : make_float2(0.f, 0.f);
            es[kk][mm] = (n < n_t && w0 + mm < n_w) ? __ldg(e + (size_t)n * n_w + w0 + mm)
                                                    : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[4], ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = as[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) ev[j] = es[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(av[i].x, ev[j].x, fmaf(-av[i].y, ev[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(av[i].x, ev[j].y, fmaf(av[i].y, ev[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = q0 + ty + 16 * i;
        if (q >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = w0 + tx + 16 * j;
            if (k >= n_w) continue;
            if (phi_acc) {
                float2* pp = phi_acc + (size_t)q * n_w + k;
                const float2 old = *pp;
                *pp = make_float2(old.x + acc[i][j].x, old.y + acc[i][j].y);
                continue;
            }
            float v = (acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y) * scale;
            if (kubo) v *= __ldg(kubo + k);
            out[(size_t)q * n_w + k] = v;
        }
    }
}

// Adjoint, first half: Phi = sum_n A[n][q] E[n][k] as in cgemm_power_kernel, then
// G[q][k] = (2 / T^2) dL/dI[q][k] Phi[q][k] (the gradient with respect to Phi).
__global__ void __launch_bounds__(256)
cgemm_gphi_kernel(const float2* __restrict__ a, const float2* __restrict__ e,
                  const float* __restrict__ dldi, float2* __restrict__ gphi, int nq, int n_t, int n_w,
                  float scale2) {
    __shared__ float2 as[BK][BM];
    __shared__ float2 es[BK][BN];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int w0 = blockIdx.x * BN, q0 = blockIdx.y * BM;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n_t; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = threadIdx.x + 256 * i;
            const int kk = idx / BM, mm = idx % BM;
            const int n = k0 + kk;
            as[kk][mm] = (n < n_t && q0 + mm < nq) ? __ldg(a + (size_t)n * nq + q0 + mm) : make_float2(0.f, 0.f);
            es[kk][mm] = (n < n_t && w0 + mm < n_w) ? __ldg(e + (size_t)n * n_w + w0 + mm) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[4], ev[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = as[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) ev[j] = es[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fmaf(av[i].x, ev[j].x, fmaf(-av[i].y, ev[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(av[i].x, ev[j].y, fmaf(av[i].y, ev[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int q = q0 + ty + 16 * i;
        if (q >= nq) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int k = w0 + tx + 16 * j;
            if (k >= n_w) continue;
            const float f = scale2 * __ldg(dldi + (size_t)q * n_w + k);
            gphi[(size_t)q * n_w + k] = make_float2(f * acc[i][j].x, f * acc[i][j].y);
        }
    }
}

// Adjoint, second half: gA[n][q] = sum_k conj(E[n][k]) G[q][k]  (both operands
// contiguous in k), written time-major like the exit waves.
__global__ void __launch_bounds__(256)
cgemm_back_kernel(const float2* __restrict__ e, const float2* __restrict__ gphi, float2* __restrict__ ga,
                  int nq, int n_t, int n_w) {
    __shared__ float2 es[BK][BM + 1];   // [k][n]
    __shared__ float2 gs[BK][BN + 1];   // [k][q]
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int q0 = blockIdx.x * BN, n0 = blockIdx.y * BM;
    float2 acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n_w; k0 += BK) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int idx = threadIdx.x + 256 * i;
            const int kk = idx % BK, rr = idx / BK;      // rr in [0, 64): row of the tile
            const int k = k0 + kk;
            const int n = n0 + rr, q = q0 + rr;
            es[kk][rr] = (k < n_w && n < n_t) ? __ldg(e + (size_t)n * n_w + k) : make_float2(0.f, 0.f);
            gs[kk][rr] = (k < n_w && q < nq) ? __ldg(gphi + (size_t)q * n_w + k) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float2 ev[4], gv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) ev[i] = es[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) gv[j] = gs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {   // conj(e) * g
                    acc[i][j].x = fmaf(ev[i].x, gv[j].x, fmaf(ev[i].y, gv[j].y, acc[i][j].x));
                    acc[i][j].y = fmaf(ev[i].x, gv[j].y, fmaf(-ev[i].y, gv[j].x, acc[i][j].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = n0 + ty + 16 * i;
        if (n >= n_t) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = q0 + tx + 16 * j;
            if (q < nq) ga[(size_t)n * nq + q] = acc[i][j];
        }
    }
}

// g_psi = gA - (1/T) sum_n gA  (FP64 mean), in place.
__global__ void centre_grad_kernel(float2* __restrict__ g, const double2* __restrict__ sum, int n_t, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (q >= nq) return;
    const double2 s = sum[q];
    const float2 v = g[(size_t)t * nq + q];
    g[(size_t)t * nq + q] = make_float2((float)((double)v.x - s.x / n_t), (float)((double)v.y - s.y / n_t));
}

// Deterministic FP64 sum: fixed partition into blocks, fixed order inside.
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;
__global__ void __launch_bounds__(kRedThreads)
partial_sum_kernel(const float* __restrict__ x, size_t n, double* __restrict__ partial) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    const size_t per = (n + gridDim.x - 1) / gridDim.x;
    const size_t b0 = (size_t)blockIdx.x * per, b1 = min(n, b0 + per);
    for (size_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) acc += (double)x[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kRedThreads)
total_kernel(const double* __restrict__ partial, int n_partial, const double* __restrict__ i_el,
             int nq, double* __restrict__ total) {
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n_partial; i += blockDim.x) acc += partial[i];
    if (i_el)
        for (int i = threadIdx.x; i < nq; i += blockDim.x) acc += i_el[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) total[0] = sh[0];
}

__global__ void scale_kernel(float* __restrict__ x, size_t n, double* __restrict__ i_el, int nq,
                             const double* __restrict__ total) {
    const double inv = 1.0 / total[0];
    const float finv = (float)inv;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] *= finv;
    if (i_el)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nq;
             i += (size_t)gridDim.x * blockDim.x)
            i_el[i] *= inv;
}

// kubo[k] = beta E_k / (1 - exp(-beta E_k)), 1 at E = 0 (natural grid when omega is NULL).
__global__ void kubo_kernel(float* __restrict__ kubo, const double* __restrict__ omega, int n_t, int n_w,
                            double dt, double beta) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_w) return;
    const double ek = omega ? omega[k] : (double)((long long)k - n_t / 2) * kPlanckMeVfs / ((double)n_t * dt);
    const double be = beta * ek;
    kubo[k] = (be == 0.0) ? 1.0f : (float)(be / (-expm1(-be)));
}

// A = psi - m_ref in FP64, rounded to float (a chunk of snapshots).
__global__ void centre_ref_kernel(const float2* __restrict__ psi, size_t ld, const double2* __restrict__ m_ref,
                                  float2* __restrict__ a, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int t = blockIdx.y;
    if (q >= nq) return;
    const double2 m = m_ref[q];
    const float2 v = __ldg(psi + (size_t)t * ld + q);
    a[(size_t)t * nq + q] = make_float2((float)((double)v.x - m.x), (float)((double)v.y - m.y));
}

// mean[q] = sum[q] / n (FP64).
__global__ void mean_kernel(const double2* __restrict__ sum, double2* __restrict__ mean, int n, int nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const double2 s = sum[q];
    mean[q] = make_double2(s.x / (double)n, s.y / (double)n);
}

// S[k] = sum_{n < T} exp(-i E_k n dt / hbar) in FP64, a fixed-order block sum
// per energy (the transform of a constant: what the reference mean leaves
// behind when it differs from the true mean).
__global__ void __launch_bounds__(256)
const_transform_kernel(const double* __restrict__ omega, int n_t, double dt, double2* __restrict__ s_out) {
    __shared__ double sr[256], si[256];
    const int k = blockIdx.x;
    const double ek = omega[k];
    double re = 0.0, im = 0.0;
    for (int n = threadIdx.x; n < n_t; n += blockDim.x) {
        const double cyc = ek * ((double)n * dt) / kPlanckMeVfs;
        double sn, cs;
        sincospi(-2.0 * (cyc - rint(cyc)), &sn, &cs);
        re += cs;
        im += sn;
    }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            sr[threadIdx.x] += sr[threadIdx.x + h];
            si[threadIdx.x] += si[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) s_out[k] = make_double2(sr[0], si[0]);
}

// Phi'(q, k) = Phi(q, k) - (m_q - m_ref_q) S[k] (FP64), I = |Phi'|^2 / T^2 (* kubo),
// I_el = |m_q|^2 with m_q = sum_q / T.
__global__ void finish_kernel(const float2* __restrict__ phi, const double2* __restrict__ m_ref,
                              const double2* __restrict__ sum, const double2* __restrict__ s_k,
                              const float* __restrict__ kubo, float* __restrict__ out, double* __restrict__ i_el,
                              int nq, int n_t, int n_w, double scale) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nq * n_w) return;
    const int q = (int)(i / n_w), k = (int)(i % n_w);
    const double2 sm = sum[q], mr = m_ref[q];
    const double inv_t = 1.0 / (double)n_t;
    const double dr = sm.x * inv_t - mr.x, di = sm.y * inv_t - mr.y;
    const double2 sk = s_k[k];
    const float2 p = phi[(size_t)q * n_w + k];
    const double pr = (double)p.x - (dr * sk.x - di * sk.y);
    const double pi = (double)p.y - (dr * sk.y + di * sk.x);
    double v = (pr * pr + pi * pi) * scale;
    if (kubo) v *= (double)__ldg(kubo + k);
    out[(size_t)q * n_w + k] = (float)v;
    if (k == 0 && i_el) {
        const double mx = sm.x * inv_t, my = sm.y * inv_t;
        i_el[q] = mx * mx + my * my;
    }
}

struct SpecWs {
    double2* sum;
    float2* a;
    float2* e;
    float* kubo;
    double* partial;
    double* total;
    double* i_el;
};

SpecWs carve_spec(Carver& cv, int nq, int n_t, int n_w, bool need_sum, bool need_iel) {
    SpecWs w;
    w.sum = need_sum ? cv.take<double2>(nq) : nullptr;
    w.a = cv.take<float2>((size_t)n_t * nq);
    w.e = cv.take<float2>((size_t)n_t * n_w);
    w.kubo = cv.take<float>(n_w);
    w.partial = cv.take<double>(kRedBlocks);
    w.total = cv.take<double>(1);
    w.i_el = need_iel ? cv.take<double>(nq) : nullptr;
    return w;
}

}  // namespace

int launch_time_sum(const float2* psi, size_t ld, double2* sum, int n_t, int nq, cudaStream_t st) {
    time_sum_kernel<<<(nq + 255) / 256, 256, 0, st>>>(psi, ld, sum, n_t, nq);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int launch_kubo(float* kubo, const double* omega, int n_t, int n_w, double dt, double beta,
                cudaStream_t st) {
    kubo_kernel<<<(n_w + 255) / 256, 256, 0, st>>>(kubo, omega, n_t, n_w, dt, beta);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

size_t normalize_ws_doubles() { return kRedBlocks + 1; }

// Scale I and I_el so that sum I + sum I_el = 1 (deterministic FP64 sums).
// i_el_user: caller's I_el (scaled too) or NULL; i_el: the values to add.
int launch_normalize(float* out, size_t n, double* i_el_user, const double* i_el, int nq,
                     double* partial, double* total, cudaStream_t st) {
    partial_sum_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(out, n, partial);
    TACAW_LAUNCH_CHECK();
    total_kernel<<<1, kRedThreads, 0, st>>>(partial, kRedBlocks, i_el, nq, total);
    TACAW_LAUNCH_CHECK();
    scale_kernel<<<1024, 256, 0, st>>>(out, n, i_el_user, nq, total);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

struct SpecBackWs {
    double2* sum;
    float2* a;
    float2* e;
    float2* gphi;
    double2* gsum;
};

static SpecBackWs carve_spec_back(Carver& cv, int nq, int n_t, int n_w, bool need_sum) {
    SpecBackWs w;
    w.sum = need_sum ? cv.take<double2>(nq) : nullptr;
    w.a = cv.take<float2>((size_t)n_t * nq);
    w.e = cv.take<float2>((size_t)n_t * n_w);
    w.gphi = cv.take<float2>((size_t)nq * n_w);
    w.gsum = cv.take<double2>(nq);
    return w;
}

size_t spectrum_backward_ws_bytes(int nq, int n_t, int n_w, bool have_sum) {
    Carver cv(nullptr);
    carve_spec_back(cv, nq, n_t, n_w, !have_sum);
    return cv.bytes();
}

int spectrum_backward_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                          size_t ld, const double2* psi_sum, const float* dldi, float2* gpsi, void* ws,
                          cudaStream_t st) {
    Carver cv(ws);
    SpecBackWs w = carve_spec_back(cv, nq, n_t, n_w, psi_sum == nullptr);
    const double2* sum = psi_sum;
    if (!sum) {
        time_sum_kernel<<<(nq + 255) / 256, 256, 0, st>>>(psi, ld, w.sum, n_t, nq);
        TACAW_LAUNCH_CHECK();
        sum = w.sum;
    }
    centre_kernel<<<dim3((nq + 255) / 256, n_t), 256, 0, st>>>(psi, ld, sum, w.a, nullptr, n_t, nq);
    TACAW_LAUNCH_CHECK();
    dft_table_kernel<<<dim3((n_w + 127) / 128, n_t), 128, 0, st>>>(w.e, nullptr, omega, n_t, n_w, dt_fs, 0.0);
    TACAW_LAUNCH_CHECK();
    const float scale2 = (float)(2.0 / ((double)n_t * (double)n_t));
    cgemm_gphi_kernel<<<dim3((n_w + BN - 1) / BN, (nq + BM - 1) / BM), 256, 0, st>>>(w.a, w.e, dldi, w.gphi, nq,
                                                                                     n_t, n_w, scale2);
    TACAW_LAUNCH_CHECK();
    cgemm_back_kernel<<<dim3((nq + BN - 1) / BN, (n_t + BM - 1) / BM), 256, 0, st>>>(w.e, w.gphi, gpsi, nq, n_t,
                                                                                     n_w);
    TACAW_LAUNCH_CHECK();
    time_sum_kernel<<<(nq + 255) / 256, 256, 0, st>>>(gpsi, nq, w.gsum, n_t, nq);
    TACAW_LAUNCH_CHECK();
    centre_grad_kernel<<<dim3((nq + 255) / 256, n_t), 256, 0, st>>>(gpsi, w.gsum, n_t, nq);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

size_t spectrum_tc_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int terms);
int spectrum_tc_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                    size_t ld, const double2* psi_sum, float* out, double* i_el, int flags,
                    double beta, int terms, void* ws, cudaStream_t st);

size_t time_fft_ws_bytes(int nq, int n_t);
int time_fft_spectrum_run(int nq, int n_t, double dt_fs, const float2* psi, size_t ld, const double2* psi_sum,
                          float* out, double* i_el, int flags, double beta, void* ws, cudaStream_t st);

size_t spectrum_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int precision) {
    if (precision == TACAW_BF16X3) return spectrum_tc_ws_bytes(nq, n_t, n_w, have_sum, have_iel, 2);
    if (precision == TACAW_BF16X6) return spectrum_tc_ws_bytes(nq, n_t, n_w, have_sum, have_iel, 3);
    if (precision == TACAW_FFT32) return time_fft_ws_bytes(nq, n_t);
    Carver cv(nullptr);
    carve_spec(cv, nq, n_t, n_w, !have_sum, !have_iel);
    return cv.bytes();
}

int spectrum_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                 size_t ld, const double2* psi_sum, float* out, double* i_el, int precision,
                 int flags, double temperature_K, void* ws, cudaStream_t st) {
    if (precision == TACAW_BF16X3 || precision == TACAW_BF16X6) {
        const double beta = (flags & TACAW_KUBO) ? 1.0 / (kBoltzmannMeVK * temperature_K) : 0.0;
        return spectrum_tc_run(nq, n_t, dt_fs, n_w, omega, psi, ld, psi_sum, out, i_el, flags, beta,
                               precision == TACAW_BF16X3 ? 2 : 3, ws, st);
    }
    if (precision == TACAW_FFT32) {
        const double beta = (flags & TACAW_KUBO) ? 1.0 / (kBoltzmannMeVK * temperature_K) : 0.0;
        return time_fft_spectrum_run(nq, n_t, dt_fs, psi, ld, psi_sum, out, i_el, flags, beta, ws, st);
    }
    Carver cv(ws);
    SpecWs w = carve_spec(cv, nq, n_t, n_w, psi_sum == nullptr, i_el == nullptr);
    const double2* sum = psi_sum;
    if (!sum) {
        time_sum_kernel<<<(nq + 255) / 256, 256, 0, st>>>(psi, ld, w.sum, n_t, nq);
        TACAW_LAUNCH_CHECK();
        sum = w.sum;
    }
    double* iel = i_el ? i_el : w.i_el;
    {
        dim3 grid((nq + 255) / 256, n_t);
        centre_kernel<<<grid, 256, 0, st>>>(psi, ld, sum, w.a, iel, n_t, nq);
        TACAW_LAUNCH_CHECK();
    }
    const bool kubo = (flags & TACAW_KUBO) != 0;
    const double beta = kubo ? 1.0 / (kBoltzmannMeVK * temperature_K) : 0.0;
    {
        dim3 grid((n_w + 127) / 128, n_t);
        dft_table_kernel<<<grid, 128, 0, st>>>(w.e, kubo ? w.kubo : nullptr, omega, n_t, n_w, dt_fs, beta);
        TACAW_LAUNCH_CHECK();
    }
    {
        dim3 grid((n_w + BN - 1) / BN, (nq + BM - 1) / BM);
        const float scale = (float)(1.0 / ((double)n_t * (double)n_t));
        cgemm_power_kernel<<<grid, 256, 0, st>>>(w.a, w.e, kubo ? w.kubo : nullptr, out, nq, n_t, n_w, scale);
        TACAW_LAUNCH_CHECK();
    }
    if (flags & TACAW_NORMALIZE) {
        const size_t n = (size_t)nq * n_w;
        partial_sum_kernel<<<kRedBlocks, kRedThreads, 0, st>>>(out, n, w.partial);
        TACAW_LAUNCH_CHECK();
        total_kernel<<<1, kRedThreads, 0, st>>>(w.partial, kRedBlocks, iel, nq, w.total);
        TACAW_LAUNCH_CHECK();
        scale_kernel<<<1024, 256, 0, st>>>(out, n, i_el, nq, w.total);
        TACAW_LAUNCH_CHECK();
    }
    return TACAW_OK;
}

// ------------------------------------------------------------------ time-chunked spectra
size_t spectrum_tc_accumulate_ws_bytes(int nq, int n_t, int n_w, int terms);
int spectrum_tc_accumulate_run(int nq, int t0, int n_chunk, double dt_fs, int n_w, const double* omega,
                               const float2* psi, size_t ld, const double2* m_ref, float2* phi, int terms,
                               void* ws, cudaStream_t st);

size_t spectrum_accumulate_ws_bytes(int nq, int n_chunk, int n_w, int precision) {
    if (precision == TACAW_BF16X3) return spectrum_tc_accumulate_ws_bytes(nq, n_chunk, n_w, 2);
    if (precision == TACAW_BF16X6) return spectrum_tc_accumulate_ws_bytes(nq, n_chunk, n_w, 3);
    Carver cv(nullptr);
    cv.take<float2>((size_t)n_chunk * nq);
    cv.take<float2>((size_t)n_chunk * n_w);
    return cv.bytes();
}

// phi[q][k] += sum_{j < n_chunk} (psi[j][q] - m_ref[q]) exp(-i E_k (t0 + j) dt / hbar)
int spectrum_accumulate_run(int nq, int t0, int n_chunk, double dt_fs, int n_w, const double* omega,
                            const float2* psi, size_t ld, const double2* m_ref, float2* phi, int precision,
                            void* ws, cudaStream_t st) {
    if (precision == TACAW_BF16X3 || precision == TACAW_BF16X6)
        return spectrum_tc_accumulate_run(nq, t0, n_chunk, dt_fs, n_w, omega, psi, ld, m_ref, phi,
                                          precision == TACAW_BF16X3 ? 2 : 3, ws, st);
    Carver cv(ws);
    float2* a = cv.take<float2>((size_t)n_chunk * nq);
    float2* e = cv.take<float2>((size_t)n_chunk * n_w);
    centre_ref_kernel<<<dim3((nq + 255) / 256, n_chunk), 256, 0, st>>>(psi, ld, m_ref, a, nq);
    TACAW_LAUNCH_CHECK();
    dft_table_kernel<<<dim3((n_w + 127) / 128, n_chunk), 128, 0, st>>>(e, nullptr, omega, n_chunk, n_w, dt_fs, 0.0,
                                                                      t0);
    TACAW_LAUNCH_CHECK();
    cgemm_power_kernel<<<dim3((n_w + BN - 1) / BN, (nq + BM - 1) / BM), 256, 0, st>>>(a, e, nullptr, nullptr, nq,
                                                                                    n_chunk, n_w, 0.f, phi);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int time_mean_run(int nq, int n, const double2* sum, double2* mean, cudaStream_t st) {
    mean_kernel<<<(nq + 255) / 256, 256, 0, st>>>(sum, mean, n, nq);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

size_t spectrum_finish_ws_bytes(int nq, int n_w) {
    Carver cv(nullptr);
    cv.take<double2>(n_w);
    cv.take<float>(n_w);
    cv.take<double>(kRedBlocks + 1);
    cv.take<double>(nq);
    return cv.bytes();
}

int spectrum_finish_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* phi,
                        const double2* m_ref, const double2* psi_sum, float* out, double* i_el, int flags,
                        double temperature_K, void* ws, cudaStream_t st) {
    Carver cv(ws);
    double2* s_k = cv.take<double2>(n_w);
    float* kubo = cv.take<float>(n_w);
    double* red = cv.take<double>(kRedBlocks + 1);
    double* iel_ws = cv.take<double>(nq);
    double* iel = i_el ? i_el : iel_ws;
    const_transform_kernel<<<n_w, 256, 0, st>>>(omega, n_t, dt_fs, s_k);
    TACAW_LAUNCH_CHECK();
    const bool use_kubo = (flags & TACAW_KUBO) != 0;
    if (use_kubo) {
        const double beta = 1.0 / (kBoltzmannMeVK * temperature_K);
        kubo_kernel<<<(n_w + 255) / 256, 256, 0, st>>>(kubo, omega, n_t, n_w, dt_fs, beta);
        TACAW_LAUNCH_CHECK();
    }
    const size_t n_el = (size_t)nq * n_w;
    finish_kernel<<<(unsigned)((n_el + 255) / 256), 256, 0, st>>>(phi, m_ref, psi_sum, s_k,
                                                                  use_kubo ? kubo : nullptr, out, iel, nq, n_t, n_w,
                                                                  1.0 / ((double)n_t * (double)n_t));
    TACAW_LAUNCH_CHECK();
    if (flags & TACAW_NORMALIZE) {
        int rc = launch_normalize(out, (size_t)nq * n_w, i_el, iel, nq, red, red + kRedBlocks, st);
        if (rc) return rc;
    }
    return TACAW_OK;
}

}  // namespace tacaw
