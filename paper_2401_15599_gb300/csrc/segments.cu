// Spectra averaged over sets of consecutive snapshots (the averaging over
// trajectory segments described after Eq. (9): each set of seg_len snapshots,
// offset by hop from the previous one, is transformed as a trajectory of its
// own and the resulting I(q, E) and elastic parts are averaged).
//
// Per set the regular spectrum path runs on the set's rows of psi (time-major,
// so a set is a contiguous block) into a per-set buffer; a kernel adds it to
// an FP64 accumulator.  The final kernel divides by the number of sets,
// applies the Kubo factor (Eq. (8)) and writes FP32; the normalisation after
// Eq. (9) then acts on the averages.

#include "common.cuh"

namespace tacaw {

size_t spectrum_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int precision);
int spectrum_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                 size_t ld, const double2* psi_sum, float* out, double* i_el, int precision,
                 int flags, double temperature_K, void* ws, cudaStream_t st);
int launch_kubo(float* kubo, const double* omega, int n_t, int n_w, double dt, double beta,
                cudaStream_t st);
int launch_normalize(float* out, size_t n, double* i_el_user, const double* i_el, int nq,
                     double* partial, double* total, cudaStream_t st);
size_t normalize_ws_doubles();

namespace {

__global__ void add_set_kernel(double* __restrict__ acc, const float* __restrict__ x, size_t n,
                               double* __restrict__ acc_el, const double* __restrict__ x_el, int nq) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc[i] += (double)x[i];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nq; i += stride)
        acc_el[i] += x_el[i];
}

// out[q][k] = acc[q][k] / n_sets * kubo[k];  el[q] = acc_el[q] / n_sets
__global__ void finish_kernel(float* __restrict__ out, const double* __restrict__ acc, size_t n, int n_w,
                              const float* __restrict__ kubo, double inv_sets, double* __restrict__ el,
                              const double* __restrict__ acc_el, int nq) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        float v = (float)(acc[i] * inv_sets);
        if (kubo) v *= kubo[i % (size_t)n_w];
        out[i] = v;
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)nq; i += stride)
        el[i] = acc_el[i] * inv_sets;
}

struct SegWs {
    double* acc;
    double* acc_el;
    float* set_i;
    double* set_el;
    double* el;
    float* kubo;
    double* red;
    void* spec;
};

SegWs carve_seg(Carver& cv, int nq, int seg_len, int n_w, int precision) {
    SegWs w;
    w.acc = cv.take<double>((size_t)nq * n_w);
    w.acc_el = cv.take<double>(nq);
    w.set_i = cv.take<float>((size_t)nq * n_w);
    w.set_el = cv.take<double>(nq);
    w.el = cv.take<double>(nq);
    w.kubo = cv.take<float>(n_w);
    w.red = cv.take<double>(normalize_ws_doubles());
    w.spec = cv.take<unsigned char>(spectrum_ws_bytes(nq, seg_len, n_w, false, true, precision));
    return w;
}

}  // namespace

size_t spectrum_segments_ws_bytes(int nq, int seg_len, int n_w, int precision) {
    Carver cv(nullptr);
    carve_seg(cv, nq, seg_len, n_w, precision);
    return cv.bytes();
}

int spectrum_segments_run(int nq, double dt_fs, int seg_len, int hop, int n_sets, int n_w,
                          const double* omega, const float2* psi, float* out, double* i_el, int precision,
                          int flags, double temperature_K, void* ws, cudaStream_t st) {
    Carver cv(ws);
    SegWs w = carve_seg(cv, nq, seg_len, n_w, precision);
    const size_t n = (size_t)nq * n_w;
    TACAW_CUDA_CHECK(cudaMemsetAsync(w.acc, 0, n * sizeof(double), st));
    TACAW_CUDA_CHECK(cudaMemsetAsync(w.acc_el, 0, (size_t)nq * sizeof(double), st));
    for (int g = 0; g < n_sets; ++g) {
        const float2* set = psi + (size_t)g * hop * nq;
        int rc = spectrum_run(nq, seg_len, dt_fs, n_w, omega, set, (size_t)nq, nullptr, w.set_i, w.set_el,
                              precision, 0, 0.0, w.spec, st);
        if (rc) return rc;
        add_set_kernel<<<1024, 256, 0, st>>>(w.acc, w.set_i, n, w.acc_el, w.set_el, nq);
        TACAW_LAUNCH_CHECK();
    }
    const bool kubo = (flags & TACAW_KUBO) != 0;
    if (kubo) {
        int rc = launch_kubo(w.kubo, omega, seg_len, n_w, dt_fs, 1.0 / (kBoltzmannMeVK * temperature_K), st);
        if (rc) return rc;
    }
    double* el = i_el ? i_el : w.el;
    finish_kernel<<<1024, 256, 0, st>>>(out, w.acc, n, n_w, kubo ? w.kubo : nullptr, 1.0 / n_sets, el,
                                        w.acc_el, nq);
    TACAW_LAUNCH_CHECK();
    if (flags & TACAW_NORMALIZE) {
        int rc = launch_normalize(out, n, i_el, el, nq, w.red, w.red + normalize_ws_doubles() - 1, st);
        if (rc) return rc;
    }
    return TACAW_OK;
}

}  // namespace tacaw
