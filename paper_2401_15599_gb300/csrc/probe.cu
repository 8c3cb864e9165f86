// Convergent-probe incident wave (the 1 mrad convergence semi-angle probe of
// the paper's Fe simulation) for tacaw_multislice's psi_in.
//
//   Psi(q) = exp(-i pi lambda f |q|^2) exp(-2 pi i q.r_p) / sqrt(N_ap)   for theta = lambda |q| <= alpha
//   psi(r) = sum_q Psi(q) exp(2 pi i q.r)                                  (no 1/N: mean |psi|^2 = 1)
//
// Only the aperture's grid points are non-zero, so the inverse transform is a
// pruned DFT in FP64, separable over the aperture's bounding box:
//   P(k_y, x) = sum_{k_x} Psi(k_x, k_y) exp(2 pi i k_x x / nx)   (k_y in the box)
//   psi(x, y) = sum_{k_y} P(k_y, x) exp(2 pi i k_y y / ny)
// with exact twiddle arguments ((k x) mod n) / n.  The result is rounded to
// float once.

#include <math.h>

#include "common.cuh"

namespace tacaw {

namespace {

__device__ double freq(int kk, int n, double len) {   // signed index kk -> q (numpy fftfreq order of ops)
    const double d = __ddiv_rn(len, (double)n);
    return __dmul_rn((double)kk, __ddiv_rn(1.0, __dmul_rn((double)n, d)));
}

struct ProbeParams {
    int nx, ny, kx_lo, kx_hi, ky_lo, ky_hi;   // aperture bounding box of signed indices
    double lx, ly, lam, alpha_mrad, defocus, x0, y0;
};

__device__ bool inside(int kx, int ky, const ProbeParams& p, double* qx, double* qy) {
    *qx = freq(kx, p.nx, p.lx);
    *qy = freq(ky, p.ny, p.ly);
    const double th = __dmul_rn(__dmul_rn(p.lam, __dsqrt_rn(__dadd_rn(__dmul_rn(*qx, *qx), __dmul_rn(*qy, *qy)))),
                                1000.0);
    return th <= p.alpha_mrad;
}

// number of aperture points (one block)
__global__ void probe_count_kernel(ProbeParams p, int* __restrict__ count) {
    __shared__ int part[256];
    int c = 0;
    const int wx = p.kx_hi - p.kx_lo + 1, wy = p.ky_hi - p.ky_lo + 1;
    for (int e = threadIdx.x; e < wx * wy; e += blockDim.x) {
        double qx, qy;
        if (inside(p.kx_lo + e % wx, p.ky_lo + e / wx, p, &qx, &qy)) ++c;
    }
    part[threadIdx.x] = c;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) part[threadIdx.x] += part[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = part[0];
}

// e^{2 pi i k x / n} with the argument reduced exactly: k x mod n
__device__ double2 twiddle(long long k, int x, int n) {
    long long m = (k * x) % n;
    if (m < 0) m += n;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    return make_double2(c, s);
}

// P[ky - ky_lo][x] for every row of the aperture box and x
__global__ void probe_rows_kernel(ProbeParams p, const int* __restrict__ count, double2* __restrict__ P) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;                       // row index ky - ky_lo
    if (x >= p.nx) return;
    const int ky = p.ky_lo + r;
    const double inv = 1.0 / sqrt((double)*count);
    double re = 0.0, im = 0.0;
    for (int kx = p.kx_lo; kx <= p.kx_hi; ++kx) {
        double qx, qy;
        if (!inside(kx, ky, p, &qx, &qy)) continue;
        // Psi phase / pi = -(lambda f q^2 + 2 (qx x0 + qy y0))
        const double q2 = __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy));
        const double ph = -(p.lam * p.defocus * q2 + 2.0 * (qx * p.x0 + qy * p.y0));
        double s, c;
        sincospi(ph, &s, &c);
        const double2 w = twiddle(kx, x, p.nx);
        re += c * w.x - s * w.y;
        im += c * w.y + s * w.x;
    }
    P[(size_t)r * p.nx + x] = make_double2(re * inv, im * inv);
}

// psi[y][x] = sum over aperture rows of P[row][x] e^{2 pi i ky y / ny}
__global__ void probe_cols_kernel(ProbeParams p, const double2* __restrict__ P, float2* __restrict__ psi) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= p.nx) return;
    double re = 0.0, im = 0.0;
    for (int r = 0; r <= p.ky_hi - p.ky_lo; ++r) {
        const double2 v = P[(size_t)r * p.nx + x];
        const double2 w = twiddle(p.ky_lo + r, y, p.ny);
        re += v.x * w.x - v.y * w.y;
        im += v.x * w.y + v.y * w.x;
    }
    psi[(size_t)y * p.nx + x] = make_float2((float)re, (float)im);
}

ProbeParams make_probe(int nx, int ny, double lx, double ly, double lam, double alpha, double defocus, double x0,
                       double y0) {
    ProbeParams p;
    p.nx = nx;
    p.ny = ny;
    p.lx = lx;
    p.ly = ly;
    p.lam = lam;
    p.alpha_mrad = alpha;
    p.defocus = defocus;
    p.x0 = x0;
    p.y0 = y0;
    // |q| <= alpha / (1000 lambda): |k| <= that * length (one spare index for rounding),
    // the whole axis -n/2 .. (n-1)/2 when that reaches the Nyquist index
    const double qa = alpha / (1000.0 * lam);
    const double rx = floor(qa * lx) + 1.0, ry = floor(qa * ly) + 1.0;
    p.kx_lo = rx >= nx / 2 ? -(nx / 2) : -(int)rx;
    p.kx_hi = rx >= nx / 2 ? (nx - 1) / 2 : (int)rx;
    p.ky_lo = ry >= ny / 2 ? -(ny / 2) : -(int)ry;
    p.ky_hi = ry >= ny / 2 ? (ny - 1) / 2 : (int)ry;
    return p;
}

}  // namespace

size_t probe_ws_bytes(int nx, int ny, double lx, double ly, double lam, double alpha) {
    const ProbeParams p = make_probe(nx, ny, lx, ly, lam, alpha, 0.0, 0.0, 0.0);
    Carver cv(nullptr);
    cv.take<int>(1);
    cv.take<double2>((size_t)(p.ky_hi - p.ky_lo + 1) * nx);
    return cv.bytes();
}

int probe_run(int nx, int ny, double lx, double ly, double lam, double alpha, double defocus, double x0, double y0,
              float2* psi, void* ws, cudaStream_t st) {
    const ProbeParams p = make_probe(nx, ny, lx, ly, lam, alpha, defocus, x0, y0);
    Carver cv(ws);
    int* count = cv.take<int>(1);
    double2* P = cv.take<double2>((size_t)(p.ky_hi - p.ky_lo + 1) * nx);
    probe_count_kernel<<<1, 256, 0, st>>>(p, count);
    TACAW_LAUNCH_CHECK();
    probe_rows_kernel<<<dim3((nx + 127) / 128, p.ky_hi - p.ky_lo + 1), 128, 0, st>>>(p, count, P);
    TACAW_LAUNCH_CHECK();
    probe_cols_kernel<<<dim3((nx + 127) / 128, ny), 128, 0, st>>>(p, P, psi);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace tacaw
