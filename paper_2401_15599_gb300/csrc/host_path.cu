// tacaw_time_to_spectrum_host: the whole path of the procedure after Eq. (9)
// in one call, from positions in host memory to I(q, E) in host memory: per
// batch of snapshots the positions are copied to the device on a copy stream
// (two staging buffers, so the copy of batch b + 1 overlaps the work on batch
// b), then slice potentials and multislice (FP64 running sum of the exit
// waves); then the temporal transform on the natural energy grid, and the
// copies of I and I_el back to the host, all on the caller's stream.

#include <algorithm>

#include "common.cuh"

namespace tacaw {

int potential_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, size_t* bytes);
int potential_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos, const int* species,
                  int n_species, const float* amp_sigma, float* V, void* ws, cudaStream_t st);
size_t multislice_ws_bytes(const tacaw_grid& g);
size_t multislice_queue_ws_bytes(const tacaw_job* jobs, int n_jobs);
int multislice_queue_run(const tacaw_job* jobs, int n_jobs, int wave, int span, void* ws, cudaStream_t st);
int multislice_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in, float2* psi_q,
                   double2* psi_sum, void* ws, cudaStream_t st, int flags);
size_t spectrum_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int precision);
int spectrum_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi, size_t ld,
                 const double2* psi_sum, float* out, double* i_el, int precision, int flags, double temperature_K,
                 void* ws, cudaStream_t st);

namespace {

struct HostPathWs {
    float* pos[2];
    float* V;
    float2* psi;
    double2* psi_sum;
    float* I;
    double* I_el;
    void *ws_pot, *ws_ms, *ws_spec;
    size_t b_pot, b_ms, b_spec;
};

HostPathWs carve_host_path(Carver& cv, const tacaw_grid& g, int n_t, int n_atoms, int batch, int precision) {
    HostPathWs w;
    const size_t nq = (size_t)g.nx * g.ny;
    for (int i = 0; i < 2; ++i) w.pos[i] = cv.take<float>((size_t)batch * n_atoms * 3);
    w.V = cv.take<float>((size_t)batch * g.n_slices * nq);
    w.psi = cv.take<float2>((size_t)n_t * nq);
    w.psi_sum = cv.take<double2>(nq);
    w.I = cv.take<float>(nq * (size_t)n_t);
    w.I_el = cv.take<double>(nq);
    potential_ws_bytes(g, batch, n_atoms, &w.b_pot);
    tacaw_job job;                                   // the work-queue multislice of one batch
    job.grid = g;
    job.n_t = batch;
    job.V = nullptr;
    job.psi_in = nullptr;
    job.psi_q = nullptr;
    job.psi_sum = nullptr;
    w.b_ms = std::max(multislice_ws_bytes(g), multislice_queue_ws_bytes(&job, 1));
    w.b_spec = spectrum_ws_bytes((int)nq, n_t, n_t, true, true, precision);
    w.ws_pot = cv.take<unsigned char>(w.b_pot);
    w.ws_ms = cv.take<unsigned char>(w.b_ms);
    w.ws_spec = cv.take<unsigned char>(w.b_spec);
    return w;
}

}  // namespace

size_t host_path_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, int batch, int precision) {
    Carver cv(nullptr);
    carve_host_path(cv, g, n_t, n_atoms, batch, precision);
    return cv.bytes();
}

int host_path_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos_host, const int* species,
                  int n_species, const float* amp_sigma, double dt_fs, int batch, int ms_flags, int precision,
                  int flags, double temperature_K, float* I_host, double* I_el_host, void* ws, cudaStream_t st) {
    Carver cv(ws);
    HostPathWs w = carve_host_path(cv, g, n_t, n_atoms, batch, precision);
    const size_t nq = (size_t)g.nx * g.ny;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // start, ready[2], free[2]
    int rc = TACAW_OK;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    cudaEvent_t start = ev[0], *ready = ev + 1, *freed = ev + 3;
    const int n_b = (n_t + batch - 1) / batch;
    auto issue = [&](int b) -> cudaError_t {     // positions of batch b into staging slot b & 1
        const int t0 = b * batch, nb = (t0 + batch <= n_t) ? batch : n_t - t0, slot = b & 1;
        cudaError_t r = cudaSuccess;
        if (b >= 2) r = cudaStreamWaitEvent(cs, freed[slot], 0);   // the potential of batch b - 2 has read it
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(w.pos[slot], pos_host + (size_t)t0 * n_atoms * 3, (size_t)nb * n_atoms * 3 * sizeof(float),
                                cudaMemcpyHostToDevice, cs);
        if (r == cudaSuccess) r = cudaEventRecord(ready[slot], cs);
        return r;
    };
    if (e == cudaSuccess) e = cudaMemsetAsync(w.psi_sum, 0, nq * sizeof(double2), st);
    if (e == cudaSuccess) e = cudaEventRecord(start, st);                  // earlier work on st comes first
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, start, 0);
    if (e == cudaSuccess) e = issue(0);
    for (int b = 0; b < n_b && e == cudaSuccess && rc == TACAW_OK; ++b) {
        if (b + 1 < n_b) e = issue(b + 1);
        const int t0 = b * batch, nb = (t0 + batch <= n_t) ? batch : n_t - t0, slot = b & 1;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ready[slot], 0);
        if (e != cudaSuccess) break;
        rc = potential_run(g, nb, n_atoms, w.pos[slot], species, n_species, amp_sigma, w.V, w.ws_pot, st);
        if (rc) break;
        e = cudaEventRecord(freed[slot], st);
        if (e != cudaSuccess) break;
        if (ms_flags & TACAW_MS_QUEUE) {
            tacaw_job job;
            job.grid = g;
            job.n_t = nb;
            job.V = w.V;
            job.psi_in = nullptr;
            job.psi_q = w.psi + (size_t)t0 * nq;
            job.psi_sum = w.psi_sum;
            rc = multislice_queue_run(&job, 1, 0, 0, w.ws_ms, st);
        } else {
            rc = multislice_run(g, nb, w.V, nullptr, w.psi + (size_t)t0 * nq, w.psi_sum, w.ws_ms, st, ms_flags);
        }
    }
    if (rc == TACAW_OK && e == cudaSuccess)
        rc = spectrum_run((int)nq, n_t, dt_fs, n_t, nullptr, w.psi, nq, w.psi_sum, w.I, w.I_el, precision, flags,
                          temperature_K, w.ws_spec, st);
    if (rc == TACAW_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(I_host, w.I, nq * (size_t)n_t * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (rc == TACAW_OK && e == cudaSuccess && I_el_host)
        e = cudaMemcpyAsync(I_el_host, w.I_el, nq * sizeof(double), cudaMemcpyDeviceToHost, st);
    // resources are released once their pending work completes
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (cs) cudaStreamDestroy(cs);
    if (rc) return rc;
    TACAW_CUDA_CHECK(e);
    return TACAW_OK;
}

}  // namespace tacaw
