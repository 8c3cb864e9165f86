/*
 * tacaw.h -- C-ABI of libtacaw, the GB300 (sm_103a) hot path of the
 * time-auto-correlation method for angle-resolved phonon / magnon EELS and
 * EEGS (Castellanos-Reyes, Zeiger, Rusz, arXiv 2401.15599).
 *
 * The path follows the paper's two-step procedure (the paragraphs after
 * Eq. (9)): for every snapshot of a trajectory, build the slice potentials of
 * that configuration and propagate a plane wave through them by multislice;
 * stack the exit waves phi_MD(q, t), Fourier transform over time, take
 * |.|^2 (Eq. (9), via the convolution theorem), optionally apply the Kubo
 * detailed-balance factor (Eq. (8)) and the fractional-intensity
 * normalisation (the unnumbered equation after Eq. (9)).  The elastic
 * (time-averaged) wave is removed before the temporal transform and returned
 * separately (the paper keeps the elastic channel at E = 0 in its spectra).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Array arguments are DEVICE pointers owned by the caller unless a comment
 *   says "host".  The library never frees them and keeps no reference to
 *   them after the call returns.
 * - `stream` is a cudaStream_t cast to void*; NULL means the legacy default
 *   stream.  Work is enqueued asynchronously on that stream; outputs are
 *   valid once the stream reaches that point.
 * - Scratch memory comes only from the caller: `ws` (device) and
 *   `*ws_bytes`.  Call once with ws == NULL to receive the required size in
 *   *ws_bytes (nothing is computed then); then call again with a buffer of at
 *   least that size.  No call allocates device memory.
 * - Return value: TACAW_OK (0) on success or a negative TACAW_E* code;
 *   tacaw_last_error() gives a message for the calling thread.  Argument
 *   errors are detected on the host before anything is enqueued.
 * - Complex numbers are (re, im) pairs of float (float2) or double (double2).
 * - Layouts are row-major, last index fastest.  Wave arrays are [ny][nx];
 *   q-space arrays are in FFT order (index k <-> frequency k for k < n/2,
 *   k - n otherwise; q = frequency / L).
 */
#ifndef TACAW_H
#define TACAW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TACAW_OK 0
#define TACAW_EINVAL (-1)       /* bad argument (detected on the host) */
#define TACAW_ECUDA (-2)        /* a CUDA runtime call or launch failed */
#define TACAW_ENOMEM (-3)       /* workspace smaller than required */
#define TACAW_ETIMEOUT (-4)     /* a bounded device wait gave up (reported by tacaw_status) */
#define TACAW_EUNSUPPORTED (-5) /* size or option not supported by this build */

/* precision of the temporal transform (tacaw_spectrum) */
#define TACAW_FP32 0            /* FP32 SIMT complex GEMM */
#define TACAW_BF16X3 1          /* split BF16 (hi+lo), 3 products, FP32 accumulation: for timing
                                   comparisons only -- its ~2^-16 error relative to sum |A||e|
                                   exceeds 2e-5 of I in the weak outer energy bands; use
                                   TACAW_BF16X6 for explicit energy grids */
#define TACAW_FFT32 2           /* natural grid only: FP32 FFT over time (T in 64..1024 as for
                                   tacaw_multislice, or 2048, 4096) */
#define TACAW_BF16X6 3          /* split BF16 (three terms), 6 products, FP32 accumulation */

/* flags of tacaw_multislice */
#define TACAW_MS_WARP_ROWS 1    /* 512-point rows: row pass with one warp per row (16 values per
                                   thread) instead of two; same results to rounding, chosen by
                                   the autotuner where faster; ignored for other sizes */
#define TACAW_MS_BLOCK_COLS 2   /* 512-point columns: one block per column block instead of the
                                   persistent column pass with TMA-staged tiles; identical
                                   results; ignored for other sizes */
#define TACAW_MS_QUEUE 4        /* square grids: all slices in one persistent launch over a device
                                   work queue (tacaw_multislice_queue with one job and the default
                                   wave); identical results; alone, not with the flags above; the
                                   workspace then also holds the queue's counters */

/* flags of tacaw_spectrum */
#define TACAW_KUBO 1            /* multiply by beta E / (1 - exp(-beta E)), Eq. (8) */
#define TACAW_NORMALIZE 2       /* scale I and I_el so sum I + sum I_el = 1 */

/*
 * Simulation box and beam.  Lengths in Angstrom, beam energy in keV.
 * Pixel (i, j) sits at (i * lx / nx, j * ly / ny).  Slice s covers
 * [z0 + s dz, z0 + (s + 1) dz); for splitting atoms the first slice reaches
 * -inf and the last +inf.  `bandlimit` is the fraction of the Nyquist radius
 * min(nx / 2lx, ny / 2ly) kept by the propagator (2/3 is the usual choice).
 */
typedef struct tacaw_grid {
    int32_t nx, ny;
    double lx, ly;
    int32_t n_slices;
    double dz, z0;
    double kev;
    double bandlimit;
} tacaw_grid;

/* Message of the last failing call on this thread ("" if none). */
const char* tacaw_last_error(void);

/* Library version as major * 10000 + minor * 100 + patch. */
int32_t tacaw_version(void);

/*
 * Bounded device waits and their status (the paper has no counterpart: this
 * is the library's failure reporting).  Kernels that wait on the GPU for
 * asynchronous copies or tensor-core work (the multislice row pass after the
 * first slice, the split-BF16 temporal transform) give up after a bounded
 * number of polls instead of spinning forever; they then stop, leave their
 * outputs incomplete and set a per-device status flag.  Calls return before
 * their kernels run, so the flag cannot be their return value:
 *
 * tacaw_status(stream): waits for `stream` (NULL: the legacy default stream),
 *   reads the flag of the current device and clears it.  Returns TACAW_OK, or
 *   TACAW_ETIMEOUT if any bounded wait gave up since the flag was last read
 *   (the outputs of the calls enqueued since then are incomplete);
 *   TACAW_ECUDA if the device cannot be reached.  Blocks the calling thread:
 *   not for use during stream capture.
 *
 * tacaw_set_wait_limit(polls): polls >= 0 sets the number of polls of every
 *   bounded data wait of the multislice row pass enqueued afterwards in this
 *   process (0 gives up at once: for tests of the timeout path); polls < 0
 *   restores the default (about a second).  A CUDA graph keeps the limit
 *   that was in force when it was captured.  Always returns TACAW_OK.
 *
 * Host-side fault injection for tests: the environment variable TACAW_FAULT
 * (comma-separated) makes "launch" fail every computing entry point with
 * TACAW_ECUDA just before it would enqueue work, "symbol" fail the lookup of
 * the library's device variables (TACAW_ECUDA), and "timeout" make
 * tacaw_status return TACAW_ETIMEOUT without touching the device.  It is read
 * on every call.
 */
int tacaw_status(void* stream);
int tacaw_set_wait_limit(int64_t polls);

/*
 * Relativistic wavelength lambda (Angstrom) and interaction constant sigma_e
 * (rad / (V Angstrom)) at beam energy `kev` (host outputs).  The paper
 * defers to standard multislice (Cowley-Moodie); these are the textbook
 * values lambda = h / sqrt(2 m0 e U (1 + eU / 2 m0 c^2)) and
 * sigma_e = 2 pi gamma m0 e lambda / h^2.
 */
int tacaw_beam_constants(double kev, double* lambda_A, double* sigma_e);

/*
 * Slice potentials of T configurations (the scattering potential of a
 * configuration tau that the multislice step of the procedure after Eq. (9)
 * propagates through).
 *
 *   v_s(r) = sum_a amp_a exp(-|r - R_a|^2 / (2 s_a^2)) w_s(z_a)
 *
 * over atoms whose minimum-image lateral offsets satisfy |dx|, |dy| <= 6 s_a (each atom an
 * isotropic 3-D Gaussian whose z-projection peaks at amp_a, in V*A), with
 * w_s(z) = (erf((z_{s+1} - z)/(sqrt2 s)) - erf((z_s - z)/(sqrt2 s))) / 2 the
 * fraction of the atom inside slice s (0 if the slice misses
 * [z - 6 s, z + 6 s]).  Requires 6 s_a < min(lx, ly) / 2.
 *
 * pos       [T][n_atoms][3] float, Angstrom (any values; wrapped laterally)
 * species   [n_atoms] int32 in [0, n_species); out-of-range entries give EINVAL
 *           only if detected -- the kernel skips atoms with a bad species
 * amp_sigma HOST [n_species][2] float: amplitude (V*A), width s (A);
 *           n_species <= TACAW_MAX_SPECIES
 * V         out [T][n_slices][ny][nx] float, V*A
 * Deterministic: identical configurations give bit-identical V (each pixel
 * is an FP32 sum over the atoms in a fixed order: by slab, then by bin, then
 * in input order); listing the same atoms in another order changes only that
 * rounding order.
 * Errors: EINVAL for bad sizes or pointers; EUNSUPPORTED for nx or ny above
 * 65535, or when the binning tables exceed shared memory (too many slices, or
 * more than 128 neighbouring bins per tile: widths too large for the slice
 * thickness or the pixel size); ENOMEM for a short workspace.
 */
#define TACAW_MAX_SPECIES 8
int tacaw_potential(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms,
                    const float* pos, const int32_t* species, int32_t n_species,
                    const float* amp_sigma, float* V, void* ws, size_t* ws_bytes,
                    void* stream);

/*
 * Multislice propagation of one incident wave through each of T snapshots
 * (second step of the procedure after Eq. (9)).  For every snapshot:
 *   psi_0 = psi_in (real space) or the unit plane wave;
 *   for s = 0 .. n_slices-1:
 *     chi = exp(i sigma_e v_s) psi_s,  Chi = F2[chi] (unitary: 1/(nx ny)),
 *     Chi' = BL(q) exp(-i pi lambda dz |q|^2) Chi,  psi_{s+1} = F2^-1[Chi'];
 *   the exit wave is Chi' of the last slice, returned in q-space.
 *
 * V        [T][n_slices][ny][nx] float, V*A (as written by tacaw_potential)
 * psi_in   [ny][nx] float2 real-space incident wave, or NULL for psi = 1
 * psi_q    out [T][ny][nx] float2, exit waves in q-space, FFT order; also
 *          used as the working buffer (no other scratch for the waves)
 * psi_sum  in/out [ny][nx] double2 running sum over snapshots, or NULL; when
 *          given, sum_t psi_q(t) is ADDED to it in FP64 (snapshot order)
 * flags    0, TACAW_MS_WARP_ROWS and / or TACAW_MS_BLOCK_COLS (variants of the
 *          passes' thread layout and staging, for the autotuner), or
 *          TACAW_MS_QUEUE alone (square grids)
 * Supported sizes: nx, ny in {64, 128, 256, 384, 512, 768, 1024}.
 */
int tacaw_multislice(const tacaw_grid* grid, int32_t n_t, const float* V,
                     const void* psi_in, void* psi_q, void* psi_sum, int32_t flags,
                     void* ws, size_t* ws_bytes, void* stream);

/*
 * tacaw_multislice without a workspace, for callers that cannot allocate
 * device memory at all (for example a plug-in whose host application owns
 * every device allocation, or a real-time service that forbids allocation
 * after start-up).  The paper has no counterpart: this is a deployment
 * convenience.  Same arguments, results and supported sizes as
 * tacaw_multislice, minus ws / ws_bytes; it calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *
 * Scratch lives in one fixed 64 KiB device array inside the library (enough
 * for every supported grid, up to 1024 x 1024); each GPU that loads the
 * library holds it until the process exits (the tables of the largest grid,
 * 1024 x 1024, take 37120 bytes).  A grid needing more is rejected with
 * TACAW_EINVAL.  The first call in a CUDA context looks up the array's device
 * address there (cudaGetSymbolAddress) and keeps it for that context; make
 * that first call before any stream capture, and again after a device reset.  All calls on a device share the array and
 * rewrite it at the start of each call: calls whose kernels overlap on the GPU
 * (concurrent streams or graph replays) race and must be serialised.
 */
int tacaw_multislice_static(const tacaw_grid* grid, int32_t n_t, const float* V,
                            const void* psi_in, void* psi_q, void* psi_sum, int32_t flags,
                            void* stream);

/*
 * Energy-resolved intensity from exit waves (Eq. (9) with Eq. (8) and the
 * normalisation after it).  With A(q, t_n) = psi(q, t_n) - m_q and
 * m_q = (1/T) sum_n psi(q, t_n) (FP64):
 *
 *   Phi(q, E_k) = sum_n A(q, t_n) exp(-i E_k t_n / hbar),  t_n = n dt
 *   I(q, E_k)   = |Phi(q, E_k)|^2 / T^2,   I_el(q) = |m_q|^2
 *
 * E > 0 is energy loss.  Natural grid (omega_meV == NULL, n_omega == T):
 * E_k = h (k - T/2) / (T dt), k = 0 .. T-1 (ascending).
 *
 * nq         number of q-points (columns of psi)
 * psi        [T][nq] float2 exit waves (time-major, e.g. tacaw_multislice's
 *            psi_q viewed as [T][ny*nx])
 * psi_sum    [nq] double2 sum_t psi, or NULL to compute it here (FP64)
 * omega_meV  DEVICE [n_omega] double energies in meV, or NULL for the natural grid
 * I          out [nq][n_omega] float
 * I_el       out [nq] double, or NULL
 * precision  TACAW_FP32, TACAW_BF16X3, TACAW_BF16X6 (three-term split, for the
 *            bands where the two-term split's ~2^-16 relative error matters), or
 *            TACAW_FFT32 (natural grid only, T in
 *            {64, 128, 256, 384, 512, 768, 1024, 2048, 4096}: one FP32 FFT over
 *            time per q instead of the DFT-matrix GEMM; with it psi_sum, when
 *            given, supplies the mean, else the mean is an FP64 block sum)
 * flags      TACAW_KUBO | TACAW_NORMALIZE (temperature_K used by KUBO)
 */
int tacaw_spectrum(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega,
                   const double* omega_meV, const void* psi, const void* psi_sum,
                   float* I, double* I_el, int32_t precision, int32_t flags,
                   double temperature_K, void* ws, size_t* ws_bytes, void* stream);

/*
 * The whole path in one call, from host positions to host I(q, E): the
 * procedure after Eq. (9) for a trajectory of T snapshots -- per batch of
 * `batch` snapshots, the positions are copied to the device on a copy stream
 * of the library's own (two staging buffers: the copy of the next batch
 * overlaps the work on this one), then tacaw_potential and tacaw_multislice
 * (ms_flags) with the FP64 running sum; then tacaw_spectrum on the natural
 * energy grid (precision, flags, temperature_K as there); then I and I_el are
 * copied back on `stream`.  Outputs are valid once `stream` reaches the end of
 * the call.
 *
 * pos_host   HOST [T][n_atoms][3] float (page-locked memory lets the copies
 *            overlap the compute; pageable memory works but serialises them)
 * species    DEVICE [n_atoms] int32; amp_sigma HOST [n_species][2] as for
 *            tacaw_potential
 * I_host     HOST out [nx*ny][T] float;  I_el_host HOST out [nx*ny] double or NULL
 * Workspace (device): the staging buffers, one batch of potentials, all exit
 * waves, the device I and the workspaces of the three calls; query with
 * ws == NULL.  Creates and destroys one stream and five events per call (not
 * for stream capture).  Errors as for the three calls it chains.
 */
int tacaw_time_to_spectrum_host(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms, const float* pos_host,
                                const int32_t* species, int32_t n_species, const float* amp_sigma, double dt_fs,
                                int32_t batch, int32_t ms_flags, int32_t precision, int32_t flags,
                                double temperature_K, float* I_host, double* I_el_host, void* ws, size_t* ws_bytes,
                                void* stream);

/*
 * Time-chunked spectra: Eq. (9) for a trajectory whose exit waves are never
 * all resident at once (long trajectories, many jobs), or whose snapshots are
 * spread over several GPUs.  With A = psi - m the inelastic transform is
 * linear in the snapshots, so it can be summed chunk by chunk; the mean m is
 * only known at the end, so every chunk is centred on a reference mean m_ref
 * (any fixed estimate, e.g. the mean of the first chunk, or the exact mean
 * when it is known) and the finishing call removes the rest in FP64:
 *
 *   Phi_ref(q, E_k) = sum_n (psi(q, t_n) - m_ref_q) exp(-i E_k t_n / hbar)
 *   Phi(q, E_k)     = Phi_ref(q, E_k) - (m_q - m_ref_q) S(E_k),
 *   S(E)            = sum_{n < T} exp(-i E t_n / hbar),   m_q = psi_sum_q / T
 *
 * Centring on a close reference keeps the summed terms small (the inelastic
 * signal is a small difference of large terms, as for tacaw_spectrum).
 *
 * tacaw_time_mean: mean [nq] double2 = psi_sum [nq] double2 / n (FP64).
 *
 * tacaw_spectrum_accumulate: phi [nq][n_omega] float2 (in/out) +=
 *   sum_{j < n_chunk} (psi[j][q] - m_ref[q]) exp(-i E_k (t0 + j) dt / hbar),
 *   for the chunk psi [n_chunk][nq] float2 of snapshots t0 .. t0 + n_chunk - 1;
 *   omega_meV DEVICE [n_omega] (required; pass the natural energies for the
 *   natural grid of the whole trajectory); precision TACAW_FP32, TACAW_BF16X6
 *   or TACAW_BF16X3 (as for tacaw_spectrum).  Workspace: query with ws == NULL.
 *
 * tacaw_spectrum_finish: I [nq][n_omega] float = |Phi|^2 / T^2 (times the Kubo
 *   factor with TACAW_KUBO), I_el [nq] double = |m|^2 (or NULL), from the
 *   accumulated phi, the m_ref used for every chunk and psi_sum = sum over all
 *   T snapshots (FP64); TACAW_NORMALIZE as in tacaw_spectrum (over these nq).
 *   S(E) and the correction are FP64.  Workspace: query with ws == NULL.
 * Errors: TACAW_EINVAL for sizes, NULL arrays, missing energies, unknown
 * precision or flags; TACAW_EUNSUPPORTED above 32640 energies on tensor cores.
 */
int tacaw_time_mean(int32_t nq, int32_t n, const void* psi_sum, void* mean, void* stream);
int tacaw_spectrum_accumulate(int32_t nq, int32_t t0, int32_t n_chunk, double dt_fs, int32_t n_omega,
                              const double* omega_meV, const void* psi, const void* m_ref, void* phi,
                              int32_t precision, void* ws, size_t* ws_bytes, void* stream);
int tacaw_spectrum_finish(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega, const double* omega_meV,
                          const void* phi, const void* m_ref, const void* psi_sum, float* I, double* I_el,
                          int32_t flags, double temperature_K, void* ws, size_t* ws_bytes, void* stream);

/*
 * Spectrum averaged over sets of consecutive snapshots (the averaging over
 * segments of one trajectory described after Eq. (9); the paper averages,
 * e.g., 79 sets of 100 snapshots offset by 50).  Set g = 0 .. n_sets-1 holds
 * snapshots g*hop .. g*hop + seg_len - 1 and is a trajectory of its own:
 *
 *   m_g(q)     = (1/seg_len) sum_n psi(q, t_{g hop + n})          (FP64)
 *   I_g(q, E)  = |sum_n (psi - m_g)(q, t_{g hop + n}) exp(-i E n dt / hbar)|^2 / seg_len^2
 *   I(q, E)    = (1/n_sets) sum_g I_g(q, E),   I_el(q) = (1/n_sets) sum_g |m_g(q)|^2
 *
 * (time measured from the start of each set: the start only adds a phase).
 * TACAW_KUBO and TACAW_NORMALIZE act on the averages as in tacaw_spectrum.
 *
 * nq, dt_fs  as in tacaw_spectrum; psi [n_t][nq] float2 exit waves (DEVICE)
 * seg_len    snapshots per set, 1 <= seg_len <= min(n_t, 65535)
 * hop        offset between the first snapshots of consecutive sets, >= 1
 * n_sets     number of sets, 1 .. (n_t - seg_len) / hop + 1; 0 = all that fit
 * omega_meV  DEVICE [n_omega] energies, or NULL for the natural grid of one
 *            set: n_omega == seg_len, E_k = h (k - seg_len/2) / (seg_len dt)
 * I          out [nq][n_omega] float;  I_el out [nq] double, or NULL
 * precision  TACAW_FP32, TACAW_BF16X3, TACAW_BF16X6 or TACAW_FFT32 (the per-set transform); sums over
 *            sets are FP64.
 * Errors: TACAW_EINVAL for sizes, sets that do not fit, unknown flags or
 * precision; TACAW_EUNSUPPORTED above 32640 energies with TACAW_BF16X3.
 */
int tacaw_spectrum_segments(int32_t nq, int32_t n_t, double dt_fs, int32_t seg_len, int32_t hop,
                            int32_t n_sets, int32_t n_omega, const double* omega_meV, const void* psi,
                            float* I, double* I_el, int32_t precision, int32_t flags,
                            double temperature_K, void* ws, size_t* ws_bytes, void* stream);

/*
 * Quasi-elastic (QEP / frozen-phonon) by-products, the quantities the paper
 * compares in its first figure (diffraction pattern of the time-averaged
 * intensity, energy integral of the spectrum, line profiles along
 * theta_y = 0, relative differences).  All arrays are DEVICE pointers; sums
 * are FP64 in a fixed order, so results do not vary between runs.
 *
 * tacaw_qep_intensity: the QEP pattern of a subset of snapshots (Eq. (4) with
 *   Eq. (3): |psi|^2 averaged over configurations), e.g. every 40th snapshot
 *   for a "100 snapshots every 1 ps" QEP of a 25 fs trajectory:
 *     qep[q] = (1/n) sum_{j < n} |psi(q, t0 + j stride)|^2
 *   psi [n_t][nq] float2; n = 0 takes every snapshot t0, t0 + stride, ... < n_t.
 *   TACAW_EINVAL when the snapshots do not fit.
 *
 * tacaw_energy_integral: out[q] = I_el[q] + sum_k I[q][k] (I [nq][n_omega]
 *   float, I_el [nq] double or NULL).  On the natural grid it equals the QEP
 *   pattern of all snapshots (Parseval).
 *
 * tacaw_line_profile: the profile along k_y = 0 of values [ny][nx] (FFT
 *   order, double): line[i] = values[k_x(i)], k_x(i) = i - nx/2 (mod nx), in
 *   ascending theta_x = lambda q_x; theta_mrad [nx] receives theta_x in mrad
 *   (or NULL).  q_x = k/lx as numpy's fftfreq.
 *
 * tacaw_azimuthal_profile: mean of values [ny][nx] (FFT order, double) over
 *   the q with theta = lambda |q| (mrad, FP64) in [b dtheta, (b+1) dtheta),
 *   b = 0 .. n_bins-1 -> profile [n_bins] (0 for an empty bin); counts
 *   [n_bins] int32 receives the number of q per bin (or NULL).  lambda_A is
 *   given by the caller (e.g. from tacaw_beam_constants).  Workspace: one
 *   int32 per q (query with ws == NULL).
 *
 * tacaw_relative_difference: out[i] = (a[i] - b[i]) / (a[i] + b[i]) (0 where
 *   a + b = 0), the "difference divided by sum" of two profiles, n doubles.
 */
int tacaw_qep_intensity(int32_t nq, int32_t n_t, int32_t t0, int32_t stride, int32_t n, const void* psi,
                        double* qep, void* stream);
int tacaw_energy_integral(int32_t nq, int32_t n_omega, const float* I, const double* I_el, double* out,
                          void* stream);
int tacaw_line_profile(int32_t nx, int32_t ny, double lx, double lambda_A, const double* values,
                       double* line, double* theta_mrad, void* stream);
int tacaw_azimuthal_profile(int32_t nx, int32_t ny, double lx, double ly, double lambda_A,
                            double dtheta_mrad, int32_t n_bins, const double* values, double* profile,
                            int32_t* counts, void* ws, size_t* ws_bytes, void* stream);
int tacaw_relative_difference(int64_t n, const double* a, const double* b, double* out, void* stream);

/*
 * Convergent-probe incident wave for tacaw_multislice's psi_in (the paper's
 * Fe set-up uses a 200 kV probe with a 1 mrad convergence semi-angle):
 *
 *   Psi(q) = exp(-i pi lambda f |q|^2) exp(-2 pi i q.r_p) / sqrt(N_ap)
 *            for the N_ap grid points with theta = lambda |q| <= alpha, else 0
 *   psi(r) = sum_q Psi(q) exp(2 pi i q.r)   (no 1/N, so mean |psi|^2 = 1 like
 *            the unit plane wave)
 *
 * theta in mrad is evaluated in FP64 as lambda * sqrt(qx^2 + qy^2) * 1000 with
 * q = k / l (numpy fftfreq order) and lambda from tacaw_beam_constants(kev).
 * A positive defocus f (Angstrom) equals free propagation through f with the
 * multislice propagator; r_p = (x0, y0) (Angstrom) is the probe position.
 * The transform is a pruned FP64 DFT over the aperture's points, rounded to
 * float once.  psi: out DEVICE [ny][nx] float2 (real space).  Workspace:
 * query with ws == NULL.  TACAW_EINVAL for non-positive sizes or energy,
 * alpha < 0 or non-finite values.
 */
int tacaw_probe(int32_t nx, int32_t ny, double lx, double ly, double kev, double alpha_mrad,
                double defocus_A, double x0_A, double y0_A, void* psi, void* ws, size_t* ws_bytes,
                void* stream);

/*
 * Autotuning of the snapshot batch (the paper has no counterpart; it serves
 * the batched and long-trajectory drivers).  Times tacaw_multislice with a
 * plane wave on the caller's potentials V [max_batch][n_slices][ny][nx] (DEVICE)
 * into psi_q [max_batch][ny][nx] (DEVICE, overwritten) for n_candidates
 * snapshot batches candidates[i] (HOST, each in [1, max_batch]): one warm-up
 * call, then `reps` timed calls per candidate (CUDA events on `stream`), every
 * call with the tacaw_multislice `flags` given (so the caller can compare the
 * variants of the passes as well; TACAW_MS_QUEUE times the work-queue
 * multislice with its default wave and span).
 * ms_per_snapshot [n_candidates] (HOST out) receives the device time per
 * snapshot of each; *best_batch (HOST out) the fastest candidate.  Blocks the
 * calling thread until the timings are read (not for stream capture).
 * Workspace as tacaw_multislice with n_t = max_batch and these flags (query
 * with ws == NULL).  TACAW_EINVAL for bad
 * sizes, TACAW_EUNSUPPORTED for grid sizes tacaw_multislice does not take.
 */
int tacaw_tune_multislice(const tacaw_grid* grid, int32_t max_batch, const float* V, void* psi_q,
                          const int32_t* candidates, int32_t n_candidates, int32_t reps, int32_t flags,
                          float* ms_per_snapshot, int32_t* best_batch, void* ws, size_t* ws_bytes,
                          void* stream);

/*
 * Adjoint of tacaw_spectrum (flags 0) for gradient-based fitting: given
 * dL/dI (real, [nq][n_omega]) returns the gradient with respect to psi in
 * the PyTorch convention for complex inputs (dL/dRe + i dL/dIm):
 *   g_Phi = (2 / T^2) dL/dI * Phi,   g_A(q, n) = sum_k g_Phi(q, k) exp(+i E_k t_n / hbar),
 *   g_psi(q, n) = g_A(q, n) - (1/T) sum_n' g_A(q, n')   (centring is self-adjoint).
 * dL_dpsi out [T][nq] float2 (FP32 SIMT).  Other arguments as in tacaw_spectrum.
 */
int tacaw_spectrum_backward(int32_t nq, int32_t n_t, double dt_fs, int32_t n_omega,
                            const double* omega_meV, const void* psi, const void* psi_sum,
                            const float* dL_dI, void* dL_dpsi,
                            void* ws, size_t* ws_bytes, void* stream);

/*
 * Many independent multislice jobs of uneven size in one call (independent
 * trajectories, or segments of one trajectory, as the paper averages over).
 * Each job is a tacaw_multislice call: its own grid (sizes as supported by
 * tacaw_multislice), snapshot count, potentials, incident wave, exit waves
 * and optional FP64 running sum.  Slice steps of jobs with the same grid
 * size share kernel launches (at most TACAW_MAX_BATCH jobs and 65535
 * snapshots per launch), so short and small jobs ride along with large ones;
 * the call only enqueues kernels and is suited to CUDA graph capture (make
 * one call outside capture first so per-kernel attributes are set).
 * jobs: HOST array; the pointers inside are device pointers.
 */
#define TACAW_MAX_BATCH 64
typedef struct tacaw_job {
    tacaw_grid grid;
    int32_t n_t;
    const float* V;      /* [n_t][n_slices][ny][nx] */
    const void* psi_in;  /* [ny][nx] float2 or NULL */
    void* psi_q;         /* out [n_t][ny][nx] float2 */
    void* psi_sum;       /* in/out [ny][nx] double2 or NULL */
} tacaw_job;

int tacaw_multislice_batch(const tacaw_job* jobs, int32_t n_jobs, void* ws, size_t* ws_bytes,
                           void* stream);

/*
 * The jobs of tacaw_multislice_batch (square grids only) through one
 * persistent launch per grid size that takes its work from a device queue
 * instead of two launches per slice.  Every snapshot is an independent
 * multislice run (second step of the procedure after Eq. (9)); a queue item
 * is one pass (row: x transforms and transmission; column: y transforms and
 * propagator with band limit) of one slice over item_span rows or columns
 * of one snapshot.  Items run job by job and, within a job, in waves of
 * `wave_snapshots` snapshots: slice 0 row items of the whole wave, its column
 * items, slice 1, and so on, so a wave's exit-wave buffers stay in L2 between
 * the passes.  An item starts when the items it depends on (the previous
 * pass of the same snapshot) have finished: device-side counters, waits
 * bounded by the limit of tacaw_set_wait_limit (default a few seconds each);
 * a wait that gives up stops the launch and makes tacaw_status report
 * TACAW_ETIMEOUT.  Results are bit-identical to tacaw_multislice_batch and
 * to tacaw_multislice for each job.
 * jobs            HOST array as for tacaw_multislice_batch (n_t up to 2^24 per
 *                 job, 2^28 in all); grids with nx == ny in the supported sizes;
 *                 V and psi_q 16-byte aligned
 * wave_snapshots  snapshots per wave, or 0: as many as fit about 128 MiB of
 *                 exit waves (64 at 512^2)
 * item_span       rows or columns per item: a multiple of the rows one block
 *                 transforms at once (256 / (N / values per thread): 4 at
 *                 512^2) that divides N; 0 or any other value: 16 (the
 *                 block's rows where those exceed 16)
 * Workspace: the per-job tables of tacaw_multislice plus 8 bytes per snapshot
 * and 16 bytes of queue state.  Errors: TACAW_EUNSUPPORTED for a grid that is
 * not square or not a supported size, TACAW_EINVAL for bad counts or NULL
 * arrays.  Enqueues only (memsets and kernels): suited to CUDA graph capture
 * after one call outside capture.
 */
int tacaw_multislice_queue(const tacaw_job* jobs, int32_t n_jobs, int32_t wave_snapshots, int32_t item_span,
                           void* ws, size_t* ws_bytes, void* stream);

/*
 * Adjoint of tacaw_multislice for gradient-based fitting (PyTorch convention
 * for complex quantities: g = dL/dRe + i dL/dIm).  Given the gradient with
 * respect to the exit waves, reverses every slice step of the forward:
 *   g_X = conj(P BL) g_Y,  g_chi = F2^H g_X / (nx ny),
 *   dL/dv_s = sigma_e Im(g_chi conj(chi)),  g_psi = exp(-i sigma_e v_s) g_chi,
 *   g_Y(previous slice) = F2 g_psi.
 * The forward waves are recomputed from checkpoints stored every
 * `ckpt_every` slices (<= 0: ceil(sqrt(n_slices))), so the workspace holds
 * about (n_slices / ckpt_every + ckpt_every + 2) wave sets of [T][ny][nx].
 *
 * V          [T][n_slices][ny][nx] float, the forward's slice potentials
 * psi_in     [ny][nx] float2 incident wave of the forward, or NULL (plane wave)
 * dL_dpsi_q  [T][ny][nx] float2 gradient with respect to the exit waves
 * dL_dV      out [T][n_slices][ny][nx] float
 */
int tacaw_multislice_backward(const tacaw_grid* grid, int32_t n_t, const float* V,
                              const void* psi_in, const void* dL_dpsi_q, float* dL_dV,
                              int32_t ckpt_every, void* ws, size_t* ws_bytes, void* stream);

/*
 * Adjoint of tacaw_potential for the per-species Gaussian parameters: with
 * P = exp(-rho^2 / 2 s^2) inside the 6 s cut-off and g = dL/dv_s,
 *   dL/d amp = sum g P w_s,   dL/d s = sum g amp P (rho^2 / s^3 w_s + dw_s/ds)
 * summed over pixels, slices, atoms of the species and the T snapshots (the
 * cut-offs are held fixed).  Block totals are kept in FP64; the result is
 * reproducible up to the FP64 rounding of the order in which candidate
 * atoms are added.
 *
 * pos, species, amp_sigma as in tacaw_potential; dL_dV [T][n_slices][ny][nx];
 * dL_damp_sigma out DEVICE [n_species][2] double (d amp, d s), overwritten.
 */
int tacaw_potential_backward(const tacaw_grid* grid, int32_t n_t, int32_t n_atoms,
                             const float* pos, const int32_t* species, int32_t n_species,
                             const float* amp_sigma, const float* dL_dV, double* dL_damp_sigma,
                             void* ws, size_t* ws_bytes, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TACAW_H */
