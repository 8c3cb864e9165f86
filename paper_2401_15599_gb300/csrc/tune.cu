// Autotuning of the multislice: how many snapshots one tacaw_multislice call
// advances together (and, through `flags`, which variant of the passes it uses, or the work queue).  The slice step is two passes over
// the batch's waves, so the batch sets how much of the wave stays in L2 between
// the row and the column pass (32 snapshots of 512^2 are 64 MB) and how many
// blocks each launch has.  The tuner times the real entry point on the
// caller's buffers for each candidate and reports the device time per snapshot.

#include "common.cuh"

namespace tacaw {

size_t multislice_ws_bytes(const tacaw_grid& g);
int multislice_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                   float2* psi_q, double2* psi_sum, void* ws, cudaStream_t st, int flags);
int multislice_queue_run(const tacaw_job* jobs, int n_jobs, int wave, int span, void* ws, cudaStream_t st);

// One timed call: the staged passes with `flags`, or (TACAW_MS_QUEUE) the
// work-queue multislice with its default wave and span.
static int tune_call(const tacaw_grid& g, int n_t, const float* V, float2* psi_q, void* ws, cudaStream_t st,
                     int flags) {
    if (flags & TACAW_MS_QUEUE) {
        tacaw_job job;
        job.grid = g;
        job.n_t = n_t;
        job.V = V;
        job.psi_in = nullptr;
        job.psi_q = psi_q;
        job.psi_sum = nullptr;
        return multislice_queue_run(&job, 1, 0, 0, ws, st);
    }
    return multislice_run(g, n_t, V, nullptr, psi_q, nullptr, ws, st, flags);
}

int tune_multislice_run(const tacaw_grid& g, const float* V, float2* psi_q, const int* cand, int n_cand,
                        int reps, int flags, float* ms_per_snapshot, int* best, void* ws, cudaStream_t st) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    TACAW_CUDA_CHECK(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        TACAW_CUDA_CHECK(ce);
    }
    int rc = TACAW_OK;
    float best_ms = 0.f;
    for (int i = 0; i < n_cand && rc == TACAW_OK; ++i) {
        rc = tune_call(g, cand[i], V, psi_q, ws, st, flags);     // warm-up
        if (rc) break;
        ce = cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == TACAW_OK && ce == cudaSuccess; ++r)
            rc = tune_call(g, cand[i], V, psi_q, ws, st, flags);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, st);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
        if (ce != cudaSuccess) {
            set_error("tacaw_tune_multislice: %s", cudaGetErrorString(ce));
            rc = TACAW_ECUDA;
            break;
        }
        ms_per_snapshot[i] = ms / ((float)reps * (float)cand[i]);
        if (i == 0 || ms_per_snapshot[i] < best_ms) {
            best_ms = ms_per_snapshot[i];
            *best = cand[i];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace tacaw
