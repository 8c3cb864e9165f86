// C-ABI entry points of libtacaw (declared in include/tacaw.h): argument
// validation, workspace queries and dispatch to the kernels.  Everything is
// enqueued on the caller's stream; nothing here allocates device memory.

#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "common.cuh"

namespace tacaw {

// ------------------------------------------------------------------ errors
static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = '\0'; }

// -------------------------------------------------------- beam constants
// CODATA 2018: Planck constant, speed of light, electron rest mass and
// elementary charge (SI).
void beam_constants(double kev, double* lambda_A, double* sigma_e) {
    const double h = 6.62607015e-34, c = 299792458.0, m0 = 9.1093837015e-31, e = 1.602176634e-19;
    const double eu = kev * 1e3 * e;                         // kinetic energy, J
    const double p = sqrt(2.0 * m0 * eu * (1.0 + eu / (2.0 * m0 * c * c)));
    const double lam_m = h / p;
    const double gamma = 1.0 + eu / (m0 * c * c);
    *lambda_A = lam_m * 1e10;
    *sigma_e = 2.0 * M_PI * gamma * m0 * e * lam_m / (h * h) * 1e-10;
}

// declared in the kernel files
bool multislice_size_supported(int n);
size_t multislice_ws_bytes(const tacaw_grid& g);
int multislice_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                   float2* psi_q, double2* psi_sum, void* ws, cudaStream_t st, int flags);
int potential_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, size_t* bytes);
int potential_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos, const int* species,
                  int n_species, const float* amp_sigma, float* V, void* ws, cudaStream_t st);
size_t spectrum_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int precision);
size_t spectrum_backward_ws_bytes(int nq, int n_t, int n_w, bool have_sum);
int spectrum_backward_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                          size_t ld, const double2* psi_sum, const float* dldi, float2* gpsi, void* ws,
                          cudaStream_t st);
size_t multislice_backward_ws_bytes(const tacaw_grid& g, int n_t, int every);
size_t multislice_batch_ws_bytes(const tacaw_job* jobs, int n_jobs);
int multislice_batch_run(const tacaw_job* jobs, int n_jobs, void* ws, cudaStream_t st);
size_t multislice_queue_ws_bytes(const tacaw_job* jobs, int n_jobs);
int multislice_queue_run(const tacaw_job* jobs, int n_jobs, int wave, int span, void* ws, cudaStream_t st);
int multislice_backward_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                            const float2* g_exit, float* dV, int every, void* ws, cudaStream_t st);
int potential_backward_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, int n_species, size_t* bytes);
int potential_backward_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos,
                           const int* species, int n_species, const float* amp_sigma, const float* dV,
                           double* grad, void* ws, cudaStream_t st);
int spectrum_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                 size_t ld, const double2* psi_sum, float* out, double* i_el, int precision,
                 int flags, double temperature_K, void* ws, cudaStream_t st);

size_t spectrum_segments_ws_bytes(int nq, int seg_len, int n_w, int precision);
int spectrum_segments_run(int nq, double dt_fs, int seg_len, int hop, int n_sets, int n_w,
                          const double* omega, const float2* psi, float* out, double* i_el, int precision,
                          int flags, double temperature_K, void* ws, cudaStream_t st);

int qep_run(int nq, int t0, int stride, int n, const float2* psi, double* qep, cudaStream_t st);
int energy_integral_run(int nq, int n_w, const float* I, const double* i_el, double* out, cudaStream_t st);
int line_profile_run(int nx, int ny, double lx, double lam, const double* values, double* line, double* theta,
                     cudaStream_t st);
size_t azimuthal_ws_bytes(int nq);
int azimuthal_run(int nx, int ny, double lx, double ly, double lam, double dtheta, int n_bins,
                  const double* values, double* prof, int* counts, void* ws, cudaStream_t st);
int rel_diff_run(size_t n, const double* a, const double* b, double* out, cudaStream_t st);

size_t probe_ws_bytes(int nx, int ny, double lx, double ly, double lam, double alpha);
int probe_run(int nx, int ny, double lx, double ly, double lam, double alpha, double defocus, double x0, double y0,
              float2* psi, void* ws, cudaStream_t st);

bool time_fft_size_supported(int n);

size_t host_path_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, int batch, int precision);
int host_path_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos_host, const int* species,
                  int n_species, const float* amp_sigma, double dt_fs, int batch, int ms_flags, int precision,
                  int flags, double temperature_K, float* I_host, double* I_el_host, void* ws, cudaStream_t st);

size_t spectrum_accumulate_ws_bytes(int nq, int n_chunk, int n_w, int precision);
int spectrum_accumulate_run(int nq, int t0, int n_chunk, double dt_fs, int n_w, const double* omega,
                            const float2* psi, size_t ld, const double2* m_ref, float2* phi, int precision,
                            void* ws, cudaStream_t st);
int time_mean_run(int nq, int n, const double2* sum, double2* mean, cudaStream_t st);
size_t spectrum_finish_ws_bytes(int nq, int n_w);
int spectrum_finish_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* phi,
                        const double2* m_ref, const double2* psi_sum, float* out, double* i_el, int flags,
                        double temperature_K, void* ws, cudaStream_t st);

int tune_multislice_run(const tacaw_grid& g, const float* V, float2* psi_q, const int* cand, int n_cand,
                        int reps, int flags, float* ms_per_snapshot, int* best, void* ws, cudaStream_t st);

static int check_grid(const tacaw_grid* g, const char* fn) {
    TACAW_REQUIRE(g != nullptr, TACAW_EINVAL, "%s: grid is NULL", fn);
    TACAW_REQUIRE(g->nx > 0 && g->ny > 0 && g->n_slices > 0 && g->n_slices <= 65535, TACAW_EINVAL,
                  "%s: nx, ny must be positive and n_slices in [1, 65535]", fn);
    TACAW_REQUIRE(g->lx > 0 && g->ly > 0 && g->dz > 0 && isfinite(g->lx) && isfinite(g->ly) &&
                      isfinite(g->dz) && isfinite(g->z0),
                  TACAW_EINVAL, "%s: lx, ly, dz must be positive and finite", fn);
    TACAW_REQUIRE(g->kev > 0 && isfinite(g->kev), TACAW_EINVAL, "%s: kev must be positive", fn);
    TACAW_REQUIRE(g->bandlimit > 0 && isfinite(g->bandlimit), TACAW_EINVAL,
                  "%s: bandlimit must be positive", fn);
    return TACAW_OK;
}

static int check_ws(void* ws, size_t* ws_bytes, size_t need, const char* fn, bool* query) {
    TACAW_REQUIRE(ws_bytes != nullptr, TACAW_EINVAL, "%s: ws_bytes is NULL", fn);
    if (ws == nullptr) {
        *ws_bytes = need;
        *query = true;
        return TACAW_OK;
    }
    *query = false;
    TACAW_REQUIRE(*ws_bytes >= need, TACAW_ENOMEM, "%s: workspace of %zu bytes, %zu needed", fn,
                  *ws_bytes, need);
    TACAW_REQUIRE(((uintptr_t)ws & 255) == 0, TACAW_EINVAL, "%s: workspace must be 256-byte aligned",
                  fn);
    return TACAW_OK;
}

}  // namespace tacaw

using namespace tacaw;

extern "C" {

const char* tacaw_last_error(void) { return g_err; }

int32_t tacaw_version(void) { return 100; }

int tacaw_beam_constants(double kev, double* lambda_A, double* sigma_e) {
    clear_error();
    TACAW_REQUIRE(kev > 0 && isfinite(kev) && lambda_A && sigma_e, TACAW_EINVAL,
                  "tacaw_beam_constants: bad argument");
    beam_constants(kev, lambda_A, sigma_e);
    return TACAW_OK;
}

int tacaw_potential(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms, const float* pos,
                    const int32_t* species, int32_t n_species, const float* amp_sigma, float* V,
                    void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_potential";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(n_t >= 0 && n_t <= 65535, TACAW_EINVAL, "%s: n_t must be in [0, 65535]", fn);
    TACAW_REQUIRE(n_atoms >= 0, TACAW_EINVAL, "%s: n_atoms must be >= 0", fn);
    TACAW_REQUIRE(n_species >= 1 && n_species <= TACAW_MAX_SPECIES && amp_sigma, TACAW_EINVAL,
                  "%s: need 1..%d species with amp_sigma", fn, TACAW_MAX_SPECIES);
    size_t need = 0;
    potential_ws_bytes(*grid, n_t, n_atoms, &need);
    bool query = false;
    rc = check_ws(ws, ws_bytes, need, fn, &query);
    if (rc || query) return rc;
    if (n_t == 0) return TACAW_OK;
    TACAW_REQUIRE(V != nullptr && (n_atoms == 0 || (pos && species)), TACAW_EINVAL,
                  "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return potential_run(*grid, n_t, n_atoms, pos, species, n_species, amp_sigma, V, ws,
                         (cudaStream_t)stream);
}

int tacaw_multislice(const tacaw_grid* grid, int32_t n_t, const float* V, const void* psi_in,
                     void* psi_q, void* psi_sum, int32_t flags, void* ws, size_t* ws_bytes,
                     void* stream) {
    clear_error();
    const char* fn = "tacaw_multislice";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(multislice_size_supported(grid->nx) && multislice_size_supported(grid->ny),
                  TACAW_EUNSUPPORTED, "%s: nx = %d, ny = %d not in {64, 128, 256, 384, 512, 768, 1024}", fn,
                  grid->nx, grid->ny);
    TACAW_REQUIRE(n_t >= 0 && n_t <= 65535, TACAW_EINVAL, "%s: n_t must be in [0, 65535]", fn);
    TACAW_REQUIRE((flags & ~(TACAW_MS_WARP_ROWS | TACAW_MS_BLOCK_COLS | TACAW_MS_QUEUE)) == 0, TACAW_EINVAL,
                  "%s: unknown flags", fn);
    const bool queue = (flags & TACAW_MS_QUEUE) != 0;
    TACAW_REQUIRE(!queue || flags == TACAW_MS_QUEUE, TACAW_EINVAL,
                  "%s: TACAW_MS_QUEUE takes no other flag", fn);
    TACAW_REQUIRE(!queue || grid->nx == grid->ny, TACAW_EUNSUPPORTED,
                  "%s: the work-queue pass needs a square grid (nx = %d, ny = %d)", fn, grid->nx, grid->ny);
    tacaw_job job;
    job.grid = *grid;
    job.n_t = n_t;
    job.V = V;
    job.psi_in = psi_in;
    job.psi_q = psi_q;
    job.psi_sum = psi_sum;
    bool query = false;
    rc = check_ws(ws, ws_bytes, queue ? multislice_queue_ws_bytes(&job, 1) : multislice_ws_bytes(*grid), fn,
                  &query);
    if (rc || query) return rc;
    if (n_t == 0) return TACAW_OK;
    TACAW_REQUIRE(V && psi_q, TACAW_EINVAL, "%s: NULL array", fn);
    TACAW_REQUIRE(!queue || (reinterpret_cast<uintptr_t>(V) % 16 == 0 && reinterpret_cast<uintptr_t>(psi_q) % 16 == 0),
                  TACAW_EINVAL, "%s: TACAW_MS_QUEUE needs 16-byte aligned V and psi_q", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    if (queue) return multislice_queue_run(&job, 1, 0, 0, ws, (cudaStream_t)stream);
    return multislice_run(*grid, n_t, V, (const float2*)psi_in, (float2*)psi_q, (double2*)psi_sum,
                          ws, (cudaStream_t)stream, flags);
}

int tacaw_multislice_batch(const tacaw_job* jobs, int32_t n_jobs, void* ws, size_t* ws_bytes,
                           void* stream) {
    clear_error();
    const char* fn = "tacaw_multislice_batch";
    TACAW_REQUIRE(jobs != nullptr && n_jobs >= 0, TACAW_EINVAL, "%s: bad job list", fn);
    for (int j = 0; j < n_jobs; ++j) {
        int rc = check_grid(&jobs[j].grid, fn);
        if (rc) return rc;
        TACAW_REQUIRE(multislice_size_supported(jobs[j].grid.nx) && multislice_size_supported(jobs[j].grid.ny),
                      TACAW_EUNSUPPORTED, "%s: job %d: nx = %d, ny = %d not supported", fn, j,
                      jobs[j].grid.nx, jobs[j].grid.ny);
        TACAW_REQUIRE(jobs[j].n_t >= 0 && jobs[j].n_t <= 65535, TACAW_EINVAL,
                      "%s: job %d: n_t must be in [0, 65535]", fn, j);
        TACAW_REQUIRE(jobs[j].n_t == 0 || (jobs[j].V && jobs[j].psi_q), TACAW_EINVAL,
                      "%s: job %d: NULL array", fn, j);
    }
    bool query = false;
    int rc = check_ws(ws, ws_bytes, multislice_batch_ws_bytes(jobs, n_jobs), fn, &query);
    if (rc || query) return rc;
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return multislice_batch_run(jobs, n_jobs, ws, (cudaStream_t)stream);
}

int tacaw_multislice_queue(const tacaw_job* jobs, int32_t n_jobs, int32_t wave_snapshots, int32_t item_span,
                           void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_multislice_queue";
    TACAW_REQUIRE(jobs != nullptr && n_jobs >= 0, TACAW_EINVAL, "%s: bad job list", fn);
    TACAW_REQUIRE(wave_snapshots >= 0, TACAW_EINVAL, "%s: wave_snapshots must be >= 0", fn);
    TACAW_REQUIRE(item_span >= 0, TACAW_EINVAL, "%s: item_span must be >= 0", fn);
    long long total = 0;
    for (int j = 0; j < n_jobs; ++j) {
        int rc = check_grid(&jobs[j].grid, fn);
        if (rc) return rc;
        TACAW_REQUIRE(multislice_size_supported(jobs[j].grid.nx) && jobs[j].grid.nx == jobs[j].grid.ny,
                      TACAW_EUNSUPPORTED, "%s: job %d: nx = %d, ny = %d: needs a square grid of a supported size",
                      fn, j, jobs[j].grid.nx, jobs[j].grid.ny);
        TACAW_REQUIRE(jobs[j].n_t >= 0 && jobs[j].n_t <= (1 << 24), TACAW_EINVAL,
                      "%s: job %d: n_t must be in [0, 2^24]", fn, j);
        TACAW_REQUIRE(jobs[j].n_t == 0 || (jobs[j].V && jobs[j].psi_q), TACAW_EINVAL,
                      "%s: job %d: NULL array", fn, j);
        total += jobs[j].n_t;
    }
    TACAW_REQUIRE(total <= (1 << 28), TACAW_EINVAL, "%s: at most 2^28 snapshots in one call", fn);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, multislice_queue_ws_bytes(jobs, n_jobs), fn, &query);
    if (rc || query) return rc;
    for (int j = 0; j < n_jobs; ++j)
        TACAW_REQUIRE(jobs[j].n_t == 0 || (reinterpret_cast<uintptr_t>(jobs[j].V) % 16 == 0 &&
                                           reinterpret_cast<uintptr_t>(jobs[j].psi_q) % 16 == 0),
                      TACAW_EINVAL, "%s: job %d: V and psi_q must be 16-byte aligned", fn, j);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return multislice_queue_run(jobs, n_jobs, wave_snapshots, item_span, ws, (cudaStream_t)stream);
}

int tacaw_spectrum(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega, const double* omega_meV,
                   const void* psi, const void* psi_sum, float* I, double* I_el, int32_t precision,
                   int32_t flags, double temperature_K, void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_spectrum";
    TACAW_REQUIRE(nq > 0 && n_t > 0 && n_t <= 65535 && n_omega > 0, TACAW_EINVAL,
                  "%s: nq, n_omega must be positive and n_t in [1, 65535]", fn);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE(omega_meV != nullptr || n_omega == n_t, TACAW_EINVAL,
                  "%s: the natural grid (omega NULL) has n_omega == T", fn);
    TACAW_REQUIRE(precision == TACAW_FP32 || precision == TACAW_BF16X3 || precision == TACAW_BF16X6 ||
                      precision == TACAW_FFT32, TACAW_EINVAL,
                  "%s: unknown precision %d", fn, precision);
    TACAW_REQUIRE((flags & ~(TACAW_KUBO | TACAW_NORMALIZE)) == 0, TACAW_EINVAL, "%s: unknown flags",
                  fn);
    TACAW_REQUIRE(!(flags & TACAW_KUBO) || (temperature_K > 0 && isfinite(temperature_K)),
                  TACAW_EINVAL, "%s: the Kubo factor needs a positive temperature", fn);
    TACAW_REQUIRE((precision != TACAW_BF16X3 && precision != TACAW_BF16X6) || n_omega <= 32640, TACAW_EUNSUPPORTED,
                  "%s: the tensor-core path takes at most 32640 energies", fn);
    TACAW_REQUIRE(precision != TACAW_FFT32 || omega_meV == nullptr, TACAW_EINVAL,
                  "%s: TACAW_FFT32 computes the natural grid only (omega must be NULL)", fn);
    TACAW_REQUIRE(precision != TACAW_FFT32 || time_fft_size_supported(n_t), TACAW_EUNSUPPORTED,
                  "%s: TACAW_FFT32 has no plan for T = %d", fn, n_t);
    bool query = false;
    int rc = check_ws(ws, ws_bytes,
                      spectrum_ws_bytes(nq, n_t, n_omega, psi_sum != nullptr, I_el != nullptr,
                                        precision),
                      fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(psi && I, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return spectrum_run(nq, n_t, dt_fs, n_omega, omega_meV, (const float2*)psi, (size_t)nq,
                        (const double2*)psi_sum, I, I_el, precision, flags, temperature_K, ws,
                        (cudaStream_t)stream);
}

int tacaw_time_to_spectrum_host(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms, const float* pos_host,
                                const int32_t* species, int32_t n_species, const float* amp_sigma, double dt_fs,
                                int32_t batch, int32_t ms_flags, int32_t precision, int32_t flags,
                                double temperature_K, float* I_host, double* I_el_host, void* ws, size_t* ws_bytes,
                                void* stream) {
    clear_error();
    const char* fn = "tacaw_time_to_spectrum_host";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(multislice_size_supported(grid->nx) && multislice_size_supported(grid->ny), TACAW_EUNSUPPORTED,
                  "%s: nx = %d, ny = %d not in {64, 128, 256, 384, 512, 768, 1024}", fn, grid->nx, grid->ny);
    TACAW_REQUIRE(n_t >= 1 && n_t <= 65535 && n_atoms >= 0 && batch >= 1, TACAW_EINVAL,
                  "%s: need n_t in [1, 65535], n_atoms >= 0 and batch >= 1", fn);
    TACAW_REQUIRE(n_species >= 1 && n_species <= TACAW_MAX_SPECIES && amp_sigma, TACAW_EINVAL,
                  "%s: need 1..%d species with amp_sigma", fn, TACAW_MAX_SPECIES);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE((ms_flags & ~(TACAW_MS_WARP_ROWS | TACAW_MS_BLOCK_COLS | TACAW_MS_QUEUE)) == 0, TACAW_EINVAL,
                  "%s: unknown multislice flags", fn);
    TACAW_REQUIRE(!(ms_flags & TACAW_MS_QUEUE) || (ms_flags == TACAW_MS_QUEUE && grid->nx == grid->ny), TACAW_EINVAL,
                  "%s: TACAW_MS_QUEUE alone, on a square grid", fn);
    TACAW_REQUIRE(precision == TACAW_FP32 || precision == TACAW_BF16X3 || precision == TACAW_BF16X6 ||
                      precision == TACAW_FFT32, TACAW_EINVAL, "%s: unknown precision %d", fn, precision);
    TACAW_REQUIRE(precision != TACAW_FFT32 || time_fft_size_supported(n_t), TACAW_EUNSUPPORTED,
                  "%s: TACAW_FFT32 has no plan for T = %d", fn, n_t);
    TACAW_REQUIRE((precision != TACAW_BF16X3 && precision != TACAW_BF16X6) || n_t <= 32640, TACAW_EUNSUPPORTED,
                  "%s: the tensor-core path takes at most 32640 energies", fn);
    TACAW_REQUIRE((flags & ~(TACAW_KUBO | TACAW_NORMALIZE)) == 0, TACAW_EINVAL, "%s: unknown flags", fn);
    TACAW_REQUIRE(!(flags & TACAW_KUBO) || (temperature_K > 0 && isfinite(temperature_K)), TACAW_EINVAL,
                  "%s: the Kubo factor needs a positive temperature", fn);
    const int b = batch < n_t ? batch : n_t;
    bool query = false;
    rc = check_ws(ws, ws_bytes, host_path_ws_bytes(*grid, n_t, n_atoms, b, precision), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(pos_host && I_host && (n_atoms == 0 || species), TACAW_EINVAL, "%s: NULL array", fn);
    const int frc = inject_launch_fault(fn);
    if (frc) return frc;
    return host_path_run(*grid, n_t, n_atoms, pos_host, species, n_species, amp_sigma, dt_fs, b, ms_flags, precision,
                         flags, temperature_K, I_host, I_el_host, ws, (cudaStream_t)stream);
}

int tacaw_time_mean(int32_t nq, int32_t n, const void* psi_sum, void* mean, void* stream) {
    clear_error();
    const char* fn = "tacaw_time_mean";
    TACAW_REQUIRE(nq > 0 && n > 0, TACAW_EINVAL, "%s: nq and n must be positive", fn);
    TACAW_REQUIRE(psi_sum && mean, TACAW_EINVAL, "%s: NULL array", fn);
    const int frc = inject_launch_fault(fn);
    if (frc) return frc;
    return time_mean_run(nq, n, (const double2*)psi_sum, (double2*)mean, (cudaStream_t)stream);
}

int tacaw_spectrum_accumulate(int32_t nq, int32_t t0, int32_t n_chunk, double dt_fs, int32_t n_omega,
                              const double* omega_meV, const void* psi, const void* m_ref, void* phi,
                              int32_t precision, void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_spectrum_accumulate";
    TACAW_REQUIRE(nq > 0 && n_chunk > 0 && n_chunk <= 65535 && n_omega > 0 && t0 >= 0, TACAW_EINVAL,
                  "%s: need nq, n_omega > 0, t0 >= 0 and n_chunk in [1, 65535]", fn);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE(omega_meV != nullptr, TACAW_EINVAL, "%s: the energies are required", fn);
    TACAW_REQUIRE(precision == TACAW_FP32 || precision == TACAW_BF16X3 || precision == TACAW_BF16X6, TACAW_EINVAL,
                  "%s: precision must be TACAW_FP32, TACAW_BF16X3 or TACAW_BF16X6", fn);
    TACAW_REQUIRE(precision == TACAW_FP32 || n_omega <= 32640, TACAW_EUNSUPPORTED,
                  "%s: the tensor-core path takes at most 32640 energies", fn);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, spectrum_accumulate_ws_bytes(nq, n_chunk, n_omega, precision), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(psi && m_ref && phi, TACAW_EINVAL, "%s: NULL array", fn);
    const int frc = inject_launch_fault(fn);
    if (frc) return frc;
    return spectrum_accumulate_run(nq, t0, n_chunk, dt_fs, n_omega, omega_meV, (const float2*)psi, (size_t)nq,
                                   (const double2*)m_ref, (float2*)phi, precision, ws, (cudaStream_t)stream);
}

int tacaw_spectrum_finish(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega, const double* omega_meV,
                          const void* phi, const void* m_ref, const void* psi_sum, float* I, double* I_el,
                          int32_t flags, double temperature_K, void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_spectrum_finish";
    TACAW_REQUIRE(nq > 0 && n_t > 0 && n_omega > 0, TACAW_EINVAL, "%s: nq, n_t, n_omega must be positive", fn);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE(omega_meV != nullptr, TACAW_EINVAL, "%s: the energies are required", fn);
    TACAW_REQUIRE((flags & ~(TACAW_KUBO | TACAW_NORMALIZE)) == 0, TACAW_EINVAL, "%s: unknown flags", fn);
    TACAW_REQUIRE(!(flags & TACAW_KUBO) || (temperature_K > 0 && isfinite(temperature_K)), TACAW_EINVAL,
                  "%s: the Kubo factor needs a positive temperature", fn);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, spectrum_finish_ws_bytes(nq, n_omega), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(phi && m_ref && psi_sum && I, TACAW_EINVAL, "%s: NULL array", fn);
    const int frc = inject_launch_fault(fn);
    if (frc) return frc;
    return spectrum_finish_run(nq, n_t, dt_fs, n_omega, omega_meV, (const float2*)phi, (const double2*)m_ref,
                               (const double2*)psi_sum, I, I_el, flags, temperature_K, ws, (cudaStream_t)stream);
}

int tacaw_spectrum_segments(int32_t nq, int32_t n_t, double dt_fs, int32_t seg_len, int32_t hop,
                            int32_t n_sets, int32_t n_omega, const double* omega_meV, const void* psi,
                            float* I, double* I_el, int32_t precision, int32_t flags, double temperature_K,
                            void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_spectrum_segments";
    TACAW_REQUIRE(nq > 0 && n_omega > 0 && seg_len > 0 && seg_len <= 65535 && hop > 0 && seg_len <= n_t,
                  TACAW_EINVAL, "%s: need nq, n_omega, hop > 0 and 1 <= seg_len <= min(T, 65535)", fn);
    const long long most = ((long long)n_t - seg_len) / hop + 1;
    const int sets = n_sets == 0 ? (int)(most < 0x7fffffff ? most : 0x7fffffff) : n_sets;
    TACAW_REQUIRE(sets >= 1 && sets <= most, TACAW_EINVAL,
                  "%s: n_sets = %d, but only %lld sets of %d snapshots offset by %d fit in %d", fn, n_sets,
                  most, seg_len, hop, n_t);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE(omega_meV != nullptr || n_omega == seg_len, TACAW_EINVAL,
                  "%s: the natural grid (omega NULL) has n_omega == seg_len", fn);
    TACAW_REQUIRE(precision == TACAW_FP32 || precision == TACAW_BF16X3 || precision == TACAW_BF16X6 ||
                      precision == TACAW_FFT32, TACAW_EINVAL,
                  "%s: unknown precision %d", fn, precision);
    TACAW_REQUIRE((flags & ~(TACAW_KUBO | TACAW_NORMALIZE)) == 0, TACAW_EINVAL, "%s: unknown flags", fn);
    TACAW_REQUIRE(!(flags & TACAW_KUBO) || (temperature_K > 0 && isfinite(temperature_K)), TACAW_EINVAL,
                  "%s: the Kubo factor needs a positive temperature", fn);
    TACAW_REQUIRE((precision != TACAW_BF16X3 && precision != TACAW_BF16X6) || n_omega <= 32640, TACAW_EUNSUPPORTED,
                  "%s: the tensor-core path takes at most 32640 energies", fn);
    TACAW_REQUIRE(precision != TACAW_FFT32 || omega_meV == nullptr, TACAW_EINVAL,
                  "%s: TACAW_FFT32 computes the natural grid only (omega must be NULL)", fn);
    TACAW_REQUIRE(precision != TACAW_FFT32 || time_fft_size_supported(seg_len), TACAW_EUNSUPPORTED,
                  "%s: TACAW_FFT32 has no plan for seg_len = %d", fn, seg_len);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, spectrum_segments_ws_bytes(nq, seg_len, n_omega, precision), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(psi && I, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return spectrum_segments_run(nq, dt_fs, seg_len, hop, sets, n_omega, omega_meV, (const float2*)psi, I, I_el,
                                 precision, flags, temperature_K, ws, (cudaStream_t)stream);
}

int tacaw_spectrum_backward(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega,
                            const double* omega_meV, const void* psi, const void* psi_sum,
                            const float* dL_dI, void* dL_dpsi, void* ws, size_t* ws_bytes,
                            void* stream) {
    clear_error();
    const char* fn = "tacaw_spectrum_backward";
    TACAW_REQUIRE(nq > 0 && n_t > 0 && n_t <= 65535 && n_omega > 0, TACAW_EINVAL,
                  "%s: nq, n_omega must be positive and n_t in [1, 65535]", fn);
    TACAW_REQUIRE(dt_fs > 0 && isfinite(dt_fs), TACAW_EINVAL, "%s: dt must be positive", fn);
    TACAW_REQUIRE(omega_meV != nullptr || n_omega == n_t, TACAW_EINVAL,
                  "%s: the natural grid (omega NULL) has n_omega == T", fn);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, spectrum_backward_ws_bytes(nq, n_t, n_omega, psi_sum != nullptr), fn,
                      &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(psi && dL_dI && dL_dpsi, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return spectrum_backward_run(nq, n_t, dt_fs, n_omega, omega_meV, (const float2*)psi, (size_t)nq,
                                 (const double2*)psi_sum, dL_dI, (float2*)dL_dpsi, ws, (cudaStream_t)stream);
}

int tacaw_multislice_backward(const tacaw_grid* grid, int32_t n_t, const float* V, const void* psi_in,
                              const void* dL_dpsi_q, float* dL_dV, int32_t ckpt_every, void* ws,
                              size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_multislice_backward";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(multislice_size_supported(grid->nx) && multislice_size_supported(grid->ny),
                  TACAW_EUNSUPPORTED, "%s: nx = %d, ny = %d not in {64, 128, 256, 384, 512, 768, 1024}", fn,
                  grid->nx, grid->ny);
    TACAW_REQUIRE(n_t >= 0 && n_t <= 65535, TACAW_EINVAL, "%s: n_t must be in [0, 65535]", fn);
    int every = ckpt_every;
    if (every <= 0) every = (int)ceil(sqrt((double)grid->n_slices));
    if (every > grid->n_slices) every = grid->n_slices;
    bool query = false;
    rc = check_ws(ws, ws_bytes, multislice_backward_ws_bytes(*grid, n_t, every), fn, &query);
    if (rc || query) return rc;
    if (n_t == 0) return TACAW_OK;
    TACAW_REQUIRE(V && dL_dpsi_q && dL_dV, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return multislice_backward_run(*grid, n_t, V, (const float2*)psi_in, (const float2*)dL_dpsi_q, dL_dV,
                                   every, ws, (cudaStream_t)stream);
}

int tacaw_potential_backward(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms, const float* pos,
                             const int32_t* species, int32_t n_species, const float* amp_sigma,
                             const float* dL_dV, double* dL_damp_sigma, void* ws, size_t* ws_bytes,
                             void* stream) {
    clear_error();
    const char* fn = "tacaw_potential_backward";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(n_t >= 1 && n_t <= 65535, TACAW_EINVAL, "%s: n_t must be in [1, 65535]", fn);
    TACAW_REQUIRE(n_atoms >= 0, TACAW_EINVAL, "%s: n_atoms must be >= 0", fn);
    TACAW_REQUIRE(n_species >= 1 && n_species <= TACAW_MAX_SPECIES && amp_sigma, TACAW_EINVAL,
                  "%s: need 1..%d species with amp_sigma", fn, TACAW_MAX_SPECIES);
    size_t need = 0;
    potential_backward_ws_bytes(*grid, n_t, n_atoms, n_species, &need);
    bool query = false;
    rc = check_ws(ws, ws_bytes, need, fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(dL_dV && dL_damp_sigma && (n_atoms == 0 || (pos && species)), TACAW_EINVAL,
                  "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return potential_backward_run(*grid, n_t, n_atoms, pos, species, n_species, amp_sigma, dL_dV,
                                  dL_damp_sigma, ws, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ QEP by-products
int tacaw_qep_intensity(int32_t nq, int32_t n_t, int32_t t0, int32_t stride, int32_t n, const void* psi,
                        double* qep, void* stream) {
    clear_error();
    const char* fn = "tacaw_qep_intensity";
    TACAW_REQUIRE(nq > 0 && n_t > 0 && t0 >= 0 && stride >= 1, TACAW_EINVAL,
                  "%s: need nq, n_t > 0, t0 >= 0, stride >= 1", fn);
    const long long most = t0 < n_t ? ((long long)n_t - 1 - t0) / stride + 1 : 0;
    const long long use = n == 0 ? most : n;
    TACAW_REQUIRE(use >= 1 && use <= most, TACAW_EINVAL,
                  "%s: %d snapshots from %d every %d do not fit in %d", fn, n, t0, stride, n_t);
    TACAW_REQUIRE(psi && qep, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return qep_run(nq, t0, stride, (int)use, (const float2*)psi, qep, (cudaStream_t)stream);
}

int tacaw_energy_integral(int32_t nq, int32_t n_omega, const float* I, const double* I_el, double* out,
                          void* stream) {
    clear_error();
    const char* fn = "tacaw_energy_integral";
    TACAW_REQUIRE(nq > 0 && n_omega > 0, TACAW_EINVAL, "%s: nq and n_omega must be positive", fn);
    TACAW_REQUIRE(I && out, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return energy_integral_run(nq, n_omega, I, I_el, out, (cudaStream_t)stream);
}

int tacaw_line_profile(int32_t nx, int32_t ny, double lx, double lambda_A, const double* values, double* line,
                       double* theta_mrad, void* stream) {
    clear_error();
    const char* fn = "tacaw_line_profile";
    TACAW_REQUIRE(nx > 0 && ny > 0 && lx > 0 && isfinite(lx) && lambda_A > 0 && isfinite(lambda_A), TACAW_EINVAL,
                  "%s: need nx, ny, lx, lambda > 0", fn);
    TACAW_REQUIRE(values && line, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return line_profile_run(nx, ny, lx, lambda_A, values, line, theta_mrad, (cudaStream_t)stream);
}

int tacaw_azimuthal_profile(int32_t nx, int32_t ny, double lx, double ly, double lambda_A, double dtheta_mrad,
                            int32_t n_bins, const double* values, double* profile, int32_t* counts, void* ws,
                            size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_azimuthal_profile";
    TACAW_REQUIRE(nx > 0 && ny > 0 && (long long)nx * ny <= 0x7fffffff && n_bins > 0 && lx > 0 && ly > 0 &&
                      isfinite(lx) && isfinite(ly) && lambda_A > 0 && isfinite(lambda_A) && dtheta_mrad > 0 &&
                      isfinite(dtheta_mrad),
                  TACAW_EINVAL, "%s: need positive sizes, lengths, lambda and bin width", fn);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, azimuthal_ws_bytes(nx * ny), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(values && profile, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return azimuthal_run(nx, ny, lx, ly, lambda_A, dtheta_mrad, n_bins, values, profile, counts, ws,
                         (cudaStream_t)stream);
}

int tacaw_relative_difference(int64_t n, const double* a, const double* b, double* out, void* stream) {
    clear_error();
    const char* fn = "tacaw_relative_difference";
    TACAW_REQUIRE(n >= 0, TACAW_EINVAL, "%s: n must be >= 0", fn);
    if (n == 0) return TACAW_OK;
    TACAW_REQUIRE(a && b && out, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return rel_diff_run((size_t)n, a, b, out, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ convergent probe
int tacaw_probe(int32_t nx, int32_t ny, double lx, double ly, double kev, double alpha_mrad, double defocus_A,
                double x0_A, double y0_A, void* psi, void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_probe";
    TACAW_REQUIRE(nx > 0 && ny > 0 && ny <= 65535 && lx > 0 && ly > 0 && isfinite(lx) && isfinite(ly), TACAW_EINVAL,
                  "%s: need nx > 0, 0 < ny <= 65535 and positive lengths", fn);
    TACAW_REQUIRE(kev > 0 && isfinite(kev) && alpha_mrad >= 0 && isfinite(alpha_mrad) && isfinite(defocus_A) &&
                      isfinite(x0_A) && isfinite(y0_A),
                  TACAW_EINVAL, "%s: need kev > 0, alpha >= 0 and finite defocus and position", fn);
    double lam = 0.0, sig = 0.0;
    beam_constants(kev, &lam, &sig);
    bool query = false;
    int rc = check_ws(ws, ws_bytes, probe_ws_bytes(nx, ny, lx, ly, lam, alpha_mrad), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(psi, TACAW_EINVAL, "%s: NULL array", fn);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return probe_run(nx, ny, lx, ly, lam, alpha_mrad, defocus_A, x0_A, y0_A, (float2*)psi, ws,
                     (cudaStream_t)stream);
}

// ------------------------------------------------------------------ autotuning
int tacaw_tune_multislice(const tacaw_grid* grid, int32_t max_batch, const float* V, void* psi_q,
                          const int32_t* candidates, int32_t n_candidates, int32_t reps, int32_t flags,
                          float* ms_per_snapshot, int32_t* best_batch, void* ws, size_t* ws_bytes, void* stream) {
    clear_error();
    const char* fn = "tacaw_tune_multislice";
    int rc = check_grid(grid, fn);
    if (rc) return rc;
    TACAW_REQUIRE(multislice_size_supported(grid->nx) && multislice_size_supported(grid->ny), TACAW_EUNSUPPORTED,
                  "%s: nx = %d, ny = %d not in {64, 128, 256, 384, 512, 768, 1024}", fn, grid->nx, grid->ny);
    TACAW_REQUIRE(max_batch >= 1 && max_batch <= 65535 && n_candidates >= 1 && reps >= 1 && reps <= 1000,
                  TACAW_EINVAL, "%s: need 1 <= max_batch <= 65535, n_candidates >= 1, 1 <= reps <= 1000", fn);
    TACAW_REQUIRE((flags & ~(TACAW_MS_WARP_ROWS | TACAW_MS_BLOCK_COLS | TACAW_MS_QUEUE)) == 0, TACAW_EINVAL,
                  "%s: unknown flags", fn);
    const bool queue = (flags & TACAW_MS_QUEUE) != 0;
    TACAW_REQUIRE(!queue || (flags == TACAW_MS_QUEUE && grid->nx == grid->ny), TACAW_EINVAL,
                  "%s: TACAW_MS_QUEUE alone, on a square grid", fn);
    tacaw_job job;                                       // workspace of the largest queue call
    job.grid = *grid;
    job.n_t = max_batch;
    job.V = V;
    job.psi_in = nullptr;
    job.psi_q = psi_q;
    job.psi_sum = nullptr;
    bool query = false;
    rc = check_ws(ws, ws_bytes, queue ? multislice_queue_ws_bytes(&job, 1) : multislice_ws_bytes(*grid), fn, &query);
    if (rc || query) return rc;
    TACAW_REQUIRE(V && psi_q && candidates && ms_per_snapshot && best_batch, TACAW_EINVAL, "%s: NULL array", fn);
    TACAW_REQUIRE(!queue || (reinterpret_cast<uintptr_t>(V) % 16 == 0 && reinterpret_cast<uintptr_t>(psi_q) % 16 == 0),
                  TACAW_EINVAL, "%s: TACAW_MS_QUEUE needs 16-byte aligned V and psi_q", fn);
    for (int i = 0; i < n_candidates; ++i)
        TACAW_REQUIRE(candidates[i] >= 1 && candidates[i] <= max_batch, TACAW_EINVAL,
                      "%s: candidate %d = %d outside [1, max_batch = %d]", fn, i, candidates[i], max_batch);
    {
        const int frc = inject_launch_fault(fn);
        if (frc) return frc;
    }
    return tune_multislice_run(*grid, V, (float2*)psi_q, candidates, n_candidates, reps, flags, ms_per_snapshot,
                               best_batch, ws, (cudaStream_t)stream);
}

}  // extern "C"
