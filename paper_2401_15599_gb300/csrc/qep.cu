// Quasi-elastic (QEP / frozen-phonon) by-products of the exit waves and of the
// spectrum, as compared in the paper's first figure: the time average of
// |psi(q, t)|^2 over snapshots (the QEP diffraction pattern, Eq. (4) with
// Eq. (3)), the energy integral of I(q, E) plus the elastic part (equal to it
// on the natural grid), line profiles along theta_y = 0 with theta = lambda q,
// azimuthal averages in bins of theta, and relative differences
// (a - b) / (a + b) of two profiles.  All sums are FP64 in a fixed order.

#include <math.h>

#include "common.cuh"

namespace tacaw {

namespace {

// qep[q] = (1/n) sum_{j < n} |psi(q, t0 + j stride)|^2
__global__ void qep_kernel(const float2* __restrict__ psi, int nq, int t0, int stride, int n,
                           double* __restrict__ qep) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double acc = 0.0;
    for (int j = 0; j < n; ++j) {
        const float2 v = __ldg(psi + (size_t)(t0 + (size_t)j * stride) * nq + q);
        acc += (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    }
    qep[q] = acc / (double)n;
}

// out[q] = i_el[q] + sum_k I[q][k]: one warp per q, lanes over k, fixed-order tree
__global__ void energy_integral_kernel(const float* __restrict__ I, const double* __restrict__ i_el, int nq,
                                       int n_w, double* __restrict__ out) {
    const int q = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    double acc = 0.0;
    const float* row = I + (size_t)q * n_w;
    for (int k = lane; k < n_w; k += 32) acc += (double)__ldg(row + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[q] = acc + (i_el ? i_el[q] : 0.0);
}

// FP64 spatial frequency of FFT index k on an axis of n pixels over length len
// (the expression order of numpy.fft.fftfreq(n, d=len/n)).
__device__ double freq(int k, int n, double len) {
    const int half = (n - 1) / 2 + 1;
    const int kk = k < half ? k : k - n;
    const double d = __ddiv_rn(len, (double)n);
    return __dmul_rn((double)kk, __ddiv_rn(1.0, __dmul_rn((double)n, d)));
}

// theta = lambda |q| in mrad, evaluated as lambda * sqrt(qx^2 + qy^2) * 1000
__device__ double theta_mrad(int kx, int ky, int nx, int ny, double lx, double ly, double lam) {
    const double qx = freq(kx, nx, lx), qy = freq(ky, ny, ly);
    return __dmul_rn(__dmul_rn(lam, __dsqrt_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)))), 1000.0);
}

// line[i] = values[q(i)] along k_y = 0, i = 0 .. nx-1 in ascending theta_x
// (fftshift order: k_x = i - nx/2 wrapped), theta[i] = lambda q_x (mrad).
__global__ void line_kernel(const double* __restrict__ values, int nx, int ny, double lx, double lam,
                            double* __restrict__ line, double* __restrict__ theta) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx) return;
    int kx = i - nx / 2;
    if (kx < 0) kx += nx;
    line[i] = values[kx];
    if (theta) theta[i] = __dmul_rn(__dmul_rn(lam, freq(kx, nx, lx)), 1000.0);
}

// bin[q] = floor(theta / dtheta), or -1 beyond n_bins
__global__ void theta_bin_kernel(int nx, int ny, double lx, double ly, double lam, double dtheta,
                                 int n_bins, int* __restrict__ bin) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nx * ny) return;
    const double th = theta_mrad(q % nx, q / nx, nx, ny, lx, ly, lam);
    const double b = floor(__ddiv_rn(th, dtheta));
    bin[q] = b < (double)n_bins ? (int)b : -1;
}

// One block per bin: mean of values over the q of that bin, warps over q in a
// fixed interleave, combined in warp order.
__global__ void __launch_bounds__(256)
azimuthal_kernel(const double* __restrict__ values, const int* __restrict__ bin, int nq,
                 double* __restrict__ prof, int* __restrict__ counts) {
    __shared__ double ws[8];
    __shared__ int wc[8];
    const int b = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    int cnt = 0;
    for (int q = threadIdx.x; q < nq; q += blockDim.x)
        if (__ldg(bin + q) == b) {
            acc += __ldg(values + q);
            ++cnt;
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        ws[warp] = acc;
        wc[warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        int c = 0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
            s += ws[w];
            c += wc[w];
        }
        prof[b] = c > 0 ? s / (double)c : 0.0;
        if (counts) counts[b] = c;
    }
}

__global__ void rel_diff_kernel(const double* __restrict__ a, const double* __restrict__ b, size_t n,
                                double* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = a[i] + b[i];
    out[i] = s != 0.0 ? (a[i] - b[i]) / s : 0.0;
}

}  // namespace

int qep_run(int nq, int t0, int stride, int n, const float2* psi, double* qep, cudaStream_t st) {
    qep_kernel<<<(nq + 255) / 256, 256, 0, st>>>(psi, nq, t0, stride, n, qep);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int energy_integral_run(int nq, int n_w, const float* I, const double* i_el, double* out, cudaStream_t st) {
    energy_integral_kernel<<<(nq + 7) / 8, 256, 0, st>>>(I, i_el, nq, n_w, out);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int line_profile_run(int nx, int ny, double lx, double lam, const double* values, double* line, double* theta,
                     cudaStream_t st) {
    line_kernel<<<(nx + 127) / 128, 128, 0, st>>>(values, nx, ny, lx, lam, line, theta);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

size_t azimuthal_ws_bytes(int nq) { return ((size_t)nq * sizeof(int) + 255) / 256 * 256; }

int azimuthal_run(int nx, int ny, double lx, double ly, double lam, double dtheta, int n_bins,
                  const double* values, double* prof, int* counts, void* ws, cudaStream_t st) {
    int* bin = static_cast<int*>(ws);
    const int nq = nx * ny;
    theta_bin_kernel<<<(nq + 255) / 256, 256, 0, st>>>(nx, ny, lx, ly, lam, dtheta, n_bins, bin);
    TACAW_LAUNCH_CHECK();
    azimuthal_kernel<<<n_bins, 256, 0, st>>>(values, bin, nq, prof, counts);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int rel_diff_run(size_t n, const double* a, const double* b, double* out, cudaStream_t st) {
    rel_diff_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n, out);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace tacaw
