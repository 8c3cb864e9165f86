// Multislice slice step as two fused passes per slice over the wave held in
// the exit-wave buffer itself (second step of the procedure after Eq. (9);
// textbook multislice: transmit, Fourier transform, propagate, inverse).
//
// With F2 = Fy Fx, one slice  psi_{s+1} = F2^-1[ P BL F2[ t_s psi_s ] ] is
// split into
//   row pass    (along x):  Fx^-1 -> multiply by t_s = exp(i sigma_e v_s) -> Fx
//   column pass (along y):  Fy -> multiply by P BL / (nx ny) -> Fy^-1
// so between passes the wave is stored "hybrid" as (k_x, y).  The first row
// pass starts from the real-space incident wave (no inverse transform); the
// last column pass skips Fy^-1 and leaves the exit wave in q-space.
// Each pass reads and writes every point once (8 + 8 bytes per point), the
// row pass also reads v_s (4 bytes per point): 36 bytes per point and slice
// for a dense wave.  The band limit zeroes a third of the k_x columns, which
// neither pass reads or writes, so at 512^2 with the 2/3 limit the passes
// move 4 + 16 f_col + 16 f_blk = 25.4 bytes per point and slice (f_col: kept
// columns, f_blk: column-pass blocks holding a kept column).

#include <cuda.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "tc.cuh"

namespace tacaw {

// Raise a kernel's dynamic shared-memory limit once per device (later calls,
// including calls made while a stream is being captured, skip the driver call).
cudaError_t ensure_smem(const void* kernel, int bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int& have = done[{kernel, dev}];
    if (have >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// Blocks of `kernel` resident on the whole device at once (occupancy times
// SM count), computed once per kernel, size and device.
cudaError_t resident_blocks(const void* kernel, int threads, int smem, int* out) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    const auto key = std::make_tuple(kernel, threads, smem, dev);
    auto it = done.find(key);
    if (it != done.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    int per_sm = 0, n_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    *out = done[key] = per_sm * n_sm;
    return cudaSuccess;
}

namespace {

constexpr int kRowThreads = 256;

// Tables computed in FP64 on the device once per call (into the workspace):
//   twx, twy: per-stage twiddle tables of the nx / ny FFT plans (rounded to float),
//   px[kx] = exp(-i pi lambda dz qx^2), py[ky] = exp(-i pi lambda dz qy^2) / (nx ny),
//   kymax[kx] = largest |ky| index with qx^2 + qy^2 <= qmax^2 (-1 if none),
//   kymax[nx] = K, the largest |kx| index with qx^2 <= qmax^2: the columns
//     kx <= K and kx >= nx - K are the ones the band limit keeps ("kept columns").
// The band limit zeroes every other column of the hybrid (k_x, y) wave, so the
// passes skip them: the row pass neither reads nor writes them, the column pass
// does not transform them (it writes their zeros only into the exit wave).
// q = k * (1 / (n * (L / n))) with k the signed FFT frequency index: the same
// FP64 expression sequence as numpy.fft.fftfreq(n, d=L/n), evaluated without
// FMA contraction so the band-limit decision is bit-identical to it.
__device__ double fft_freq(int k, int n, double len) {
    const int half = (n - 1) / 2 + 1;
    const int kk = k < half ? k : k - n;
    const double d = __ddiv_rn(len, (double)n);
    const double val = __ddiv_rn(1.0, __dmul_rn((double)n, d));
    return __dmul_rn((double)kk, val);
}

__device__ void fill_plan_twiddles(int n, float2* tw, int tid, int nthr) {
    switch (n) {
        case 64: fft::fill_twiddles<64>(tw, tid, nthr); break;
        case 128: fft::fill_twiddles<128>(tw, tid, nthr); break;
        case 256: fft::fill_twiddles<256>(tw, tid, nthr); break;
        case 512: fft::fill_twiddles<512>(tw, tid, nthr); break;
        case 1024: fft::fill_twiddles<1024>(tw, tid, nthr); break;
        case 384: fft::fill_twiddles<384>(tw, tid, nthr); break;
        case 768: fft::fill_twiddles<768>(tw, tid, nthr); break;
    }
}

// Copy a plan's twiddle table into shared memory (made visible by the
// barrier at the start of the first transform).
template <int N>
__device__ __forceinline__ void stage_twiddles(float2* dst, const float2* __restrict__ src) {
    for (int i = threadIdx.x; i < fft::TwSize<N>::value; i += blockDim.x) dst[i] = __ldg(src + i);
}

__global__ void ms_setup_kernel(float2* twx, float2* twy, float2* px, float2* py, int* kymax,
                                int nx, int ny, double lx, double ly, double lam_dz,
                                double qmax2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0) {
        fill_plan_twiddles(nx, twx, threadIdx.x, blockDim.x);
        fill_plan_twiddles(ny, twy, threadIdx.x, blockDim.x);
    }
    if (i < nx) {
        double s, c;
        const double qx = fft_freq(i, nx, lx);
        const double qx2 = __dmul_rn(qx, qx);
        sincospi(-lam_dz * qx2, &s, &c);
        px[i] = make_float2((float)c, (float)s);
        int kmax = -1;
        for (int k = 0; k <= ny / 2; ++k) {  // |q_y| grows with k: stop at the first miss
            const double qy = fft_freq(k, ny, ly);
            if (__dadd_rn(qx2, __dmul_rn(qy, qy)) <= qmax2) kmax = k; else break;
        }
        kymax[i] = kmax;
    }
    if (i == 0) {                        // K: the same FP64 test with q_y = 0
        int kk = -1;
        for (int k = 0; k <= nx / 2; ++k) {
            const double q = fft_freq(k, nx, lx);
            if (__dadd_rn(__dmul_rn(q, q), 0.0) <= qmax2) kk = k; else break;
        }
        kymax[nx] = kk;
    }
    if (i < ny) {
        double s, c;
        const double qy = fft_freq(i, ny, ly);
        sincospi(-lam_dz * __dmul_rn(qy, qy), &s, &c);
        const double inv_n = 1.0 / ((double)nx * (double)ny);
        py[i] = make_float2((float)(c * inv_n), (float)(s * inv_n));
    }
}

// Row pass body for one row: (k_x, y) row -> Fx^-1 (mode 0; mode 1 starts from
// the unit plane wave, mode 2 from psi_in) -> multiply by exp(i sigma v) -> Fx.
__device__ __forceinline__ bool kept_column(int kx, int nx, int K) { return kx <= K || kx >= nx - K; }

template <int NX>
__device__ __forceinline__ void row_body(float2* __restrict__ rowp, const float* __restrict__ vrow,
                                         const float2* __restrict__ inrow, int mode, float sigma, int K,
                                         float2* b0, float2* b1, const float2* tw, int t, int row) {
    using namespace fft;
    constexpr int E = Plan<NX>::E;
    constexpr int TPT = NX / E;
    const PadRowLayout lay{row * PaddedLen<NX>::value};
    float2 v[E];
    if (mode == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = kept_column(t + TPT * m, NX, K) ? rowp[t + TPT * m] : make_float2(0.f, 0.f);
        transform<NX, true>(v, b0, b1, t, tw, lay);
    } else if (mode == 1) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = make_float2(1.f, 0.f);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = inrow[t + TPT * m];
    }
    float x[E];
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sigma * __ldcs(vrow + t + TPT * m);
    transmit<E>(v, x);
    transform<NX, false>(v, b0, b1, t, tw, lay);
#pragma unroll
    for (int m = 0; m < E; ++m)
        if (kept_column(t + TPT * m, NX, K)) rowp[t + TPT * m] = v[m];
}

// Row pass: ROWS rows of one snapshot per block.  With ahead > 0 (16-byte
// aligned buffers) thread 0 first asks L2 for the block's potential rows and
// for the rows of the block `ahead` places later in launch order (about one
// wave of resident blocks later), so their loads find the data in L2.
template <int NX>
__global__ void __launch_bounds__(kRowThreads)
row_pass_kernel(float2* __restrict__ psi, const float* __restrict__ V,
                const float2* __restrict__ psi_in, const float2* __restrict__ twx,
                const int* __restrict__ kymax, int ny, int n_slices, int s, float sigma, int mode,
                int ahead) {
    constexpr int TPT = NX / fft::Plan<NX>::E;
    constexpr int ROWS = kRowThreads / TPT;
    constexpr int PL = fft::PaddedLen<NX>::value;
    extern __shared__ float2 smem[];
    float2* tw = smem + 2 * ROWS * PL;
    if (ahead > 0 && threadIdx.x == 0) {
        prefetch_l2_bulk(V + (((size_t)blockIdx.y * n_slices + s) * ny + (size_t)blockIdx.x * ROWS) * NX,
                         ROWS * NX * sizeof(float));
        const size_t nxt = (size_t)blockIdx.y * gridDim.x + blockIdx.x + ahead;
        if (nxt < (size_t)gridDim.x * gridDim.y) {
            const size_t by = nxt / gridDim.x, y0 = (nxt % gridDim.x) * ROWS;
            prefetch_l2_bulk(V + ((by * n_slices + s) * ny + y0) * NX, ROWS * NX * sizeof(float));
            if (mode == 0) prefetch_l2_bulk(psi + (by * ny + y0) * NX, ROWS * NX * sizeof(float2));
        }
    }
    stage_twiddles<NX>(tw, twx);
    const int t = threadIdx.x % TPT;
    const int row = threadIdx.x / TPT;
    const int y = blockIdx.x * ROWS + row;
    const size_t snap = blockIdx.y;
    row_body<NX>(psi + (snap * ny + y) * NX, V + ((snap * n_slices + s) * ny + y) * NX,
                 psi_in ? psi_in + (size_t)y * NX : nullptr, mode, sigma, __ldg(kymax + NX), smem,
                 smem + ROWS * PL, tw, t, row);
}


// Staged row pass for slices after the first (hybrid (k_x, y) input): a
// persistent grid in which each block walks row groups (ROWS rows of one
// snapshot) and, while it transforms one group, has bulk asynchronous copies
// (cp.async.bulk, completion on an mbarrier) bring the kept columns of the next
// group's wave rows and its potential rows into the other half of a two-stage
// shared-memory ring.  The stage being transformed doubles as the FFT's
// exchange buffer (one-buffer mode).  Same arithmetic as row_body, so the
// results are identical.  The waits for a group's data give up after
// `polls` polls: the block then sets the status flag *err, stops, and waits
// (with a fixed long bound) for the copy it is waiting on, so no copy lands in
// shared memory after the block has exited.  A group's copy is issued once
// every thread has passed the wait of the group before (the barrier after that
// wait), when the stage it refills is free, so at most one copy is in flight
// at a wait and a group ends without a barrier of its own.
// The barrier of one row's transform threads: a named barrier per row when a
// row spans several warps, the warp itself when it spans one or part of one.
template <int TPT>
__device__ __forceinline__ auto row_sync_of(int row) {
    static_assert(TPT <= 32 || (TPT % 32 == 0 && kRowThreads / TPT <= 15), "named barrier per row");
    if constexpr (TPT >= 64) return fft::NamedSync{1 + row, TPT};
    else return fft::WarpSync{};
}

// P is the transform plan: Plan<NX> (for 512 points: 8 values per thread, two
// warps per row) or WarpPlan<NX> (16 values per thread, one warp per row).
// Blocks per SM the staged row pass's register budget targets: four for the
// 8-value plans (their shared memory allows four), two for the 16- and
// 24-value plans (at most 128 registers a thread).
template <class P>
struct RowStagedMinBlocks { static constexpr int value = P::E == 8 ? 4 : 2; };

template <int NX, class P>
__global__ void __launch_bounds__(kRowThreads, RowStagedMinBlocks<P>::value)
row_pass_staged_kernel(float2* __restrict__ psi, const float* __restrict__ V, const float2* __restrict__ twx,
                       const int* __restrict__ kymax, int ny, int n_slices, int s, float sigma, int n_groups,
                       int* __restrict__ err, uint32_t polls) {
    using namespace fft;
    constexpr int E = P::E;
    constexpr int TPT = NX / E;
    constexpr int ROWS = kRowThreads / TPT;
    constexpr int PL = PaddedLen<NX>::value;            // a row's slot: the padded exchange layout
    constexpr int PSI_BYTES = ROWS * PL * (int)sizeof(float2);
    constexpr int V_BYTES = ROWS * NX * (int)sizeof(float);
    constexpr int STAGE = PSI_BYTES + V_BYTES;
    extern __shared__ __align__(128) unsigned char stage_raw[];
    float2* tw = reinterpret_cast<float2*>(stage_raw + 2 * STAGE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(stage_raw + 2 * STAGE + TwSize<NX>::value * sizeof(float2));
    const int groups_per_snap = ny / ROWS;
    const int K = __ldg(kymax + NX);
    // kept columns [0, a) and [b, NX), both ends even so every copy is 16-byte aligned
    int a = K + 1;
    a += a & 1;
    if (a > NX) a = NX;
    int b = NX - K;
    b -= b & 1;
    if (b < a) b = a;
    const uint32_t tx_bytes = (uint32_t)(ROWS * (a + NX - b) * (int)sizeof(float2) + V_BYTES);
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    stage_twiddles<NX>(tw, twx);
    __syncthreads();
    // the twiddles of one stage in which all of a thread's butterflies share
    // jm stay in registers for every group (plans of 8 or 16 values; the
    // 24-value plans have no registers to spare)
    using RT = typename std::conditional<(P::E <= 16), RegTwOf<P, NX>, NoRegTw>::type;
    RT rt{};
    if constexpr (P::E <= 16) rt = load_reg_tw<P, NX>(tw, threadIdx.x % TPT);
    auto issue = [&](int snap, int gi, int st) {   // thread 0: group gi of snapshot snap
        const int y0 = gi * ROWS;
        unsigned char* dst = stage_raw + st * STAGE;
        fence_proxy_async_smem();                  // the stage was FFT scratch two groups ago
        tc::mbar_arrive_expect_tx(&bar[st], tx_bytes);
        const float2* src = psi + ((size_t)snap * ny + y0) * NX;
        for (int r = 0; r < ROWS; ++r) {
            bulk_copy_g2s(dst + (size_t)r * PL * sizeof(float2), src + (size_t)r * NX, a * sizeof(float2), &bar[st]);
            if (b < NX)
                bulk_copy_g2s(dst + ((size_t)r * PL + b) * sizeof(float2), src + (size_t)r * NX + b,
                              (NX - b) * sizeof(float2), &bar[st]);
        }
        bulk_copy_g2s(dst + PSI_BYTES, V + (((size_t)snap * n_slices + s) * ny + y0) * NX, V_BYTES, &bar[st]);
    };
    const int t = threadIdx.x % TPT;
    const int row = threadIdx.x / TPT;
    // group g = snap * groups_per_snap + gi advances by gridDim.x groups, tracked without divisions
    const int step_snap = (int)gridDim.x / groups_per_snap, step_gi = (int)gridDim.x % groups_per_snap;
    int snap = (int)blockIdx.x / groups_per_snap, gi = (int)blockIdx.x % groups_per_snap;
    if (threadIdx.x == 0 && (int)blockIdx.x < n_groups) issue(snap, gi, 0);
    int it = 0;
    bool timed_out = false;                        // at a timeout: a copy in flight into stage it & 1
    for (int g = blockIdx.x; g < n_groups; g += gridDim.x, ++it) {
        const int st = it & 1;
        const bool ok = tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, polls);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        float2* rowp = psi + ((size_t)snap * ny + gi * ROWS + row) * NX;
        snap += step_snap;                         // (snap, gi): the next group
        gi += step_gi;
        if (gi >= groups_per_snap) {
            gi -= groups_per_snap;
            ++snap;
        }
        // every thread has left the previous group, so its stage takes the next copy
        if (threadIdx.x == 0 && g + (int)gridDim.x < n_groups) issue(snap, gi, st ^ 1);
        float2* buf = reinterpret_cast<float2*>(stage_raw + st * STAGE);
        const float* vrow = reinterpret_cast<const float*>(stage_raw + st * STAGE + PSI_BYTES) + row * NX;
        const PadRowLayout lay{row * PL};
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = kept_column(t + TPT * m, NX, K) ? buf[row * PL + t + TPT * m] : make_float2(0.f, 0.f);
        const auto row_sync = row_sync_of<TPT>(row);   // a row's transforms touch only its own row
        transform_plan<P, NX, true>(v, buf, buf, t, tw, lay, row_sync, rt);
        float x[E];
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = sigma * vrow[t + TPT * m];
        transmit<E>(v, x);
        transform_plan<P, NX, false>(v, buf, buf, t, tw, lay, row_sync, rt);
#pragma unroll
        for (int m = 0; m < E; ++m)
            if (kept_column(t + TPT * m, NX, K)) rowp[t + TPT * m] = v[m];
    }
    if (timed_out && threadIdx.x == 0) {
        atomicExch(err, 1);
        // drain: the copy into stage it & 1 (whose wait gave up; the next group's
        // copy is issued only after that wait) completes once its bytes land
        const int st = it & 1;
        for (int k = 0; k < 64 && !tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, 1u << 20); ++k) {
        }
    }
}

// Exchange layouts of the one-warp-per-row pass and of the staged column pass:
// at 512 points those without half-warp bank collisions (fft::PadRowLayout512,
// PadColLayout512, whose slots are longer), else the Pad16 layouts.
template <int N>
using WarpRowLay = typename std::conditional<N == 512, fft::PadRowLayout512, fft::PadRowLayout>::type;
template <int N, int W>
using StagedColLay = typename std::conditional<N == 512, fft::PadColLayout512<W>, fft::PadColLayout<W>>::type;

// Staged row pass with one warp per row (plans of TPT = 32 threads): every
// warp walks its own rows with its own two-stage ring and mbarriers, so the
// warps of a block never wait on one another.  Lane 0 issues the bulk copies
// of the warp's next row (its kept columns and potential row) once every lane
// has passed the wait for the current one (__syncwarp), when the stage that
// copy refills is free.  Same arithmetic as row_body, so the results are
// identical.  A wait that gives up after `polls` polls sets *err; the warp
// stops and waits (with a fixed long bound) for the copy it was waiting on.
template <int NX, class P>
__global__ void __launch_bounds__(kRowThreads, RowStagedMinBlocks<P>::value)
row_pass_warp_kernel(float2* __restrict__ psi, const float* __restrict__ V, const float2* __restrict__ twx,
                     const int* __restrict__ kymax, int ny, int n_slices, int s, float sigma, int n_rows,
                     int* __restrict__ err, uint32_t polls) {
    using namespace fft;
    constexpr int E = P::E;
    constexpr int TPT = NX / E;
    static_assert(TPT == 32, "one warp per row");
    constexpr int WARPS = kRowThreads / 32;
    using Lay = WarpRowLay<NX>;
    constexpr int PL = Lay::template slot<NX>();
    constexpr int PSI_BYTES = PL * (int)sizeof(float2);
    constexpr int STAGE = PSI_BYTES + NX * (int)sizeof(float);   // one row: padded wave slot, then v_s
    extern __shared__ __align__(128) unsigned char wstage_raw[];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    unsigned char* mine = wstage_raw + (size_t)warp * 2 * STAGE;
    float2* tw = reinterpret_cast<float2*>(wstage_raw + (size_t)WARPS * 2 * STAGE);
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + TwSize<NX>::value) + 2 * warp;
    const int K = __ldg(kymax + NX);
    int a = K + 1;                                 // kept columns [0, a) and [b, NX), 16-byte aligned copies
    a += a & 1;
    if (a > NX) a = NX;
    int b = NX - K;
    b -= b & 1;
    if (b < a) b = a;
    const uint32_t tx_bytes = (uint32_t)((a + NX - b) * (int)sizeof(float2) + NX * (int)sizeof(float));
    if (lane == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    stage_twiddles<NX>(tw, twx);
    __syncthreads();                               // twiddles and barrier initialisation visible
    using RT = RegTwOf<P, NX>;
    const RT rt = load_reg_tw<P, NX>(tw, lane);
    auto issue = [&](int snap, int y, int st) {    // lane 0
        unsigned char* dst = mine + st * STAGE;
        fence_proxy_async_smem();                  // the stage was FFT scratch two rows ago
        tc::mbar_arrive_expect_tx(&bar[st], tx_bytes);
        const float2* src = psi + ((size_t)snap * ny + y) * NX;
        bulk_copy_g2s(dst, src, a * sizeof(float2), &bar[st]);
        if (b < NX) bulk_copy_g2s(dst + (size_t)b * sizeof(float2), src + b, (NX - b) * sizeof(float2), &bar[st]);
        bulk_copy_g2s(dst + PSI_BYTES, V + (((size_t)snap * n_slices + s) * ny + y) * NX, NX * sizeof(float),
                      &bar[st]);
    };
    // row r = snap * ny + y advances by `step` rows, tracked without divisions
    const int step = gridDim.x * WARPS;
    const int step_snap = step / ny, step_y = step % ny;
    const int r0 = blockIdx.x * WARPS + warp;
    int snap = r0 / ny, y = r0 % ny;
    if (lane == 0 && r0 < n_rows) issue(snap, y, 0);
    int it = 0;
    bool timed_out = false;
    for (int r = r0; r < n_rows; r += step, ++it) {
        const int st = it & 1;
        const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, polls));
        if (!ok) {
            timed_out = true;
            break;
        }
        float2* rowp = psi + ((size_t)snap * ny + y) * NX;
        snap += step_snap;                         // (snap, y): the next row
        y += step_y;
        if (y >= ny) {
            y -= ny;
            ++snap;
        }
        // every lane has left the previous row, so its stage takes the next copy
        if (lane == 0 && r + step < n_rows) issue(snap, y, st ^ 1);
        float2* buf = reinterpret_cast<float2*>(mine + st * STAGE);
        const float* vrow = reinterpret_cast<const float*>(mine + st * STAGE + PSI_BYTES);
        const Lay lay{0};
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = kept_column(lane + TPT * m, NX, K) ? buf[lane + TPT * m] : make_float2(0.f, 0.f);
        transform_plan<P, NX, true>(v, buf, buf, lane, tw, lay, WarpSync{}, rt);
        float x[E];
#pragma unroll
        for (int m = 0; m < E; ++m) x[m] = sigma * vrow[lane + TPT * m];
        transmit<E>(v, x);
        transform_plan<P, NX, false>(v, buf, buf, lane, tw, lay, WarpSync{}, rt);
#pragma unroll
        for (int m = 0; m < E; ++m)
            if (kept_column(lane + TPT * m, NX, K)) rowp[lane + TPT * m] = v[m];
        __syncwarp();                              // the stage is refilled after the next wait
    }
    if (timed_out && lane == 0) {
        atomicExch(err, 1);
        const int st = it & 1;
        for (int k = 0; k < 64 && !tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, 1u << 20); ++k) {
        }
    }
}

// Jobs of one batched launch (all of the same grid size): block row y of the
// launch belongs to job j with start[j] <= blockIdx.y < start[j + 1].
constexpr int kMaxBatch = 64;
struct RowJobs {
    int n;
    int start[kMaxBatch + 1];
    float2* psi[kMaxBatch];
    const float* V[kMaxBatch];
    const float2* psi_in[kMaxBatch];
    const int* kymax[kMaxBatch];
    int n_slices[kMaxBatch];
    int mode[kMaxBatch];
    float sigma[kMaxBatch];
};

__device__ __forceinline__ int find_job(const int* start, int n, int gy) {
    int j = 0;
    while (j + 1 < n && start[j + 1] <= gy) ++j;
    return j;
}

template <int NX>
__global__ void __launch_bounds__(kRowThreads)
row_batch_kernel(const __grid_constant__ RowJobs jobs, const float2* __restrict__ twx, int ny, int s) {
    constexpr int TPT = NX / fft::Plan<NX>::E;
    constexpr int ROWS = kRowThreads / TPT;
    constexpr int PL = fft::PaddedLen<NX>::value;
    extern __shared__ float2 smem[];
    float2* tw = smem + 2 * ROWS * PL;
    stage_twiddles<NX>(tw, twx);
    const int t = threadIdx.x % TPT;
    const int row = threadIdx.x / TPT;
    const int y = blockIdx.x * ROWS + row;
    const int j = find_job(jobs.start, jobs.n, blockIdx.y);
    const size_t snap = blockIdx.y - jobs.start[j];
    const float2* pin = jobs.psi_in[j];
    row_body<NX>(jobs.psi[j] + (snap * ny + y) * NX, jobs.V[j] + ((snap * jobs.n_slices[j] + s) * ny + y) * NX,
                 pin ? pin + (size_t)y * NX : nullptr, jobs.mode[j], jobs.sigma[j], __ldg(jobs.kymax[j] + NX),
                 smem, smem + ROWS * PL, tw, t, row);
}

// W columns per column-pass block and the blocks per SM the register budget
// targets.  At 512 rows four 256-thread blocks of 4 columns per SM ran faster
// than two 512-thread blocks of 8 (narrower barriers; fewer band-limited
// columns transformed) and than eight blocks of 2 (half-sector loads, spills).
template <int NY>
struct ColCfg {
    static constexpr int W = (NY >= 1024) ? 8 : (NY >= 512 ? 4 : 16);
    static constexpr int kMinBlocks = (NY >= 1024) ? 1 : (NY >= 512 ? 4 : 2);
};
// ny must be a multiple of the rows handled per row-pass block
static_assert(kRowThreads / (384 / 24) == 16 && kRowThreads / (768 / 24) == 8, "row tiles");

// Column pass body for W adjacent columns of one snapshot.
//   forward  (CONJ = false, FFT_IN = true):  Fy -> x P BL / (nx ny) -> Fy^-1 (unless `last`)
//   adjoint  (CONJ = true):  [Fy] -> x conj(P BL) / (nx ny) -> Fy^-1, where the leading
//   Fy is skipped (FFT_IN = false) when the input is already in q-space.
template <int NY, bool CONJ, bool FFT_IN>
__device__ __forceinline__ void col_body(float2* __restrict__ col, int nx, int kx,
                                         const float2* __restrict__ px, const float2* __restrict__ py,
                                         const int* __restrict__ kymax, int last, float2* b0, float2* b1,
                                         const float2* tw, int t, int c) {
    using namespace fft;
    constexpr int E = Plan<NY>::E;
    constexpr int TPT = NY / E;
    constexpr int W = ColCfg<NY>::W;
    const PadColLayout<W> lay{c};
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = col[(size_t)(t + TPT * m) * nx];
    if (FFT_IN) transform<NY, false>(v, b0, b1, t, tw, lay);
    const float2 pxv = __ldg(px + kx);
    const int kmax = __ldg(kymax + kx);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int ky = t + TPT * m;
        const int aky = ky < NY / 2 ? ky : NY - ky;
        const float2 p = cmul(pxv, __ldg(py + ky));
        v[m] = (aky <= kmax) ? (CONJ ? cmulc(v[m], p) : cmul(v[m], p)) : make_float2(0.f, 0.f);
    }
    if (!last) transform<NY, true>(v, b0, b1, t, tw, lay);
#pragma unroll
    for (int m = 0; m < E; ++m) col[(size_t)(t + TPT * m) * nx] = v[m];
}

// A column block whose W columns the band limit all drops: nothing to
// transform; after the last slice it writes their zeros into the exit wave.
// Returns true when the block is done (uniform over the block).
template <int NY>
__device__ __forceinline__ bool dropped_block(float2* __restrict__ col, int nx, int kx0, int K, int last,
                                              int t) {
    constexpr int TPT = NY / fft::Plan<NY>::E;
    constexpr int W = ColCfg<NY>::W;
    if (kx0 <= K || kx0 + W - 1 >= nx - K) return false;
    if (last) {
#pragma unroll
        for (int m = 0; m < fft::Plan<NY>::E; ++m) col[(size_t)(t + TPT * m) * nx] = make_float2(0.f, 0.f);
    }
    return true;
}

// Column pass: W columns of one snapshot per block.
template <int NY, bool CONJ, bool FFT_IN>
__global__ void __launch_bounds__(ColCfg<NY>::W * (NY / fft::Plan<NY>::E), ColCfg<NY>::kMinBlocks)
col_pass_kernel(float2* __restrict__ psi, const float2* __restrict__ twy,
                const float2* __restrict__ px, const float2* __restrict__ py,
                const int* __restrict__ kymax, int nx, int last) {
    constexpr int W = ColCfg<NY>::W;
    constexpr int PL = fft::PaddedLen<NY>::value;
    extern __shared__ float2 smem[];
    float2* tw = smem + 2 * W * PL;
    const int c = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int kx = blockIdx.x * W + c;
    const size_t snap = blockIdx.y;
    const int K = __ldg(kymax + nx);
    if (dropped_block<NY>(psi + snap * NY * (size_t)nx + kx, nx, blockIdx.x * W, K, last, t))
        return;
    stage_twiddles<NY>(tw, twy);
    col_body<NY, CONJ, FFT_IN>(psi + snap * NY * (size_t)nx + kx, nx, kx, px, py, kymax, last, smem,
                               smem + W * PL, tw, t, c);
}

// Staged column pass of the forward slice step (Fy -> x P BL / (nx ny) -> Fy^-1,
// or no Fy^-1 after the last slice): a persistent grid in which each block
// walks the column blocks that hold a kept column (W columns of one snapshot;
// the band-limited blocks are never read), and while it transforms one, TMA
// brings the next block's NY x W tile into the other half of a two-stage
// shared-memory ring (two boxes of NY/2 rows; the tile arrives dense, row by
// row, which is the order in which a warp's 8 rows x W columns read it).  The
// stage being transformed doubles as the exchange buffer.  Same arithmetic as
// col_body, so the results are identical.  The waits give up after `polls`
// polls like the staged row pass's (status flag, then a drain of the stage
// waited on; the next tile is issued after the barrier that follows a wait).
template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::W * (NY / fft::Plan<NY>::E), ColCfg<NY>::kMinBlocks)
col_pass_staged_kernel(const __grid_constant__ CUtensorMap map, float2* __restrict__ psi,
                       const float2* __restrict__ twy, const float2* __restrict__ px, const float2* __restrict__ py,
                       const int* __restrict__ kymax, int nx, int n_t, int last, int* __restrict__ err,
                       uint32_t polls) {
    using namespace fft;
    constexpr int E = Plan<NY>::E;
    constexpr int TPT = NY / E;
    constexpr int W = ColCfg<NY>::W;
    using Lay = StagedColLay<NY, W>;
    constexpr int STAGE = Lay::template slot<NY>() * W;  // float2 per stage: the padded exchange layout
    constexpr uint32_t STAGE_BYTES = NY * W * sizeof(float2);   // what TMA brings (dense)
    extern __shared__ __align__(128) float2 cstage[];
    float2* tw = cstage + 2 * STAGE;
    uint64_t* bar = reinterpret_cast<uint64_t*>(tw + TwSize<NY>::value);
    const int c = threadIdx.x % W;
    const int t = threadIdx.x / W;
    // kept column blocks: [0, n_lo) and [nb - n_hi, nb) of the nb = nx / W blocks
    const int K = __ldg(kymax + nx);
    const int nb = nx / W;
    const int n_lo = K / W + 1;
    int hi0 = (nx - K - W + 1 + W - 1) / W;              // first block with a column >= nx - K
    if (hi0 < n_lo) hi0 = n_lo;
    const int n_kept = n_lo + (nb - hi0);
    const long long n_items = (long long)n_t * n_kept;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    stage_twiddles<NY>(tw, twy);
    __syncthreads();
    const RegTwOf<Plan<NY>, NY> rt = load_reg_tw<Plan<NY>, NY>(tw, t);
    // item i = snap * n_kept + j is column block j of the kept blocks of snapshot
    // snap; the position advances by gridDim.x items per step, tracked without
    // divisions in the loop
    auto kept_block = [&](int j) { return j < n_lo ? j : hi0 + (j - n_lo); };
    const int step_snap = (int)(gridDim.x / (unsigned)n_kept), step_j = (int)(gridDim.x % (unsigned)n_kept);
    auto advance = [&](int& snap, int& j) {
        snap += step_snap;
        j += step_j;
        if (j >= n_kept) {
            j -= n_kept;
            ++snap;
        }
    };
    auto issue = [&](int snap, int j, int st) {           // thread 0
        const int kb = kept_block(j);
        float2* dst = cstage + st * STAGE;
        fence_proxy_async_smem();                        // the stage was exchange scratch two items ago
        tc::mbar_arrive_expect_tx(&bar[st], STAGE_BYTES);
        tc::tma_load_2d(dst, &map, &bar[st], kb * W, snap * NY);
        tc::tma_load_2d(dst + (NY / 2) * W, &map, &bar[st], kb * W, snap * NY + NY / 2);
    };
    int snap = (int)(blockIdx.x / (unsigned)n_kept), j = (int)(blockIdx.x % (unsigned)n_kept);
    if (threadIdx.x == 0 && (long long)blockIdx.x < n_items) issue(snap, j, 0);
    int it = 0;
    bool timed_out = false;
    for (long long i = blockIdx.x; i < n_items; i += gridDim.x, ++it) {
        const int st = it & 1;
        const bool ok = tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, polls);
        if (__syncthreads_or(!ok)) {
            timed_out = true;
            break;
        }
        const int kb = kept_block(j);
        const int cur_snap = snap;
        advance(snap, j);                                // (snap, j): the next item
        // every thread has left the previous item, so its stage takes the next tile
        if (threadIdx.x == 0 && i + gridDim.x < n_items) issue(snap, j, st ^ 1);
        const int kx = kb * W + c;
        float2* buf = cstage + st * STAGE;
        const Lay lay{c};
        float2 v[E];
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = buf[(t + TPT * m) * W + c];
        transform_plan<Plan<NY>, NY, false>(v, buf, buf, t, tw, lay, BlockSync{}, rt);
        const float2 pxv = __ldg(px + kx);
        const int kmax = __ldg(kymax + kx);
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int ky = t + TPT * m;
            const int aky = ky < NY / 2 ? ky : NY - ky;
            v[m] = (aky <= kmax) ? cmul(v[m], cmul(pxv, __ldg(py + ky))) : make_float2(0.f, 0.f);
        }
        if (!last) transform_plan<Plan<NY>, NY, true>(v, buf, buf, t, tw, lay, BlockSync{}, rt);
        float2* col = psi + (size_t)cur_snap * NY * nx + kx;
#pragma unroll
        for (int m = 0; m < E; ++m) col[(size_t)(t + TPT * m) * nx] = v[m];
    }
    if (timed_out && threadIdx.x == 0) {
        atomicExch(err, 1);
        const int st = it & 1;
        for (int k = 0; k < 64 && !tc::mbar_wait_quiet(&bar[st], (it >> 1) & 1, 1u << 20); ++k) {
        }
    }
}

// After the last slice: zeros into the exit wave's band-limited column blocks
// (the staged column pass never touches them).
template <int NY>
__global__ void zero_dropped_kernel(float2* __restrict__ psi, const int* __restrict__ kymax, int nx) {
    constexpr int W = ColCfg<NY>::W;
    const int K = __ldg(kymax + nx);
    const int n_lo = K / W + 1;
    int hi0 = (nx - K - W + 1 + W - 1) / W;
    if (hi0 < n_lo) hi0 = n_lo;
    const int x = n_lo * W + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (x >= hi0 * W) return;
    float2* p = psi + (size_t)blockIdx.y * NY * nx + x;
    for (int y = 0; y < NY; ++y) p[(size_t)y * nx] = make_float2(0.f, 0.f);
}

struct ColJobs {
    int n;
    int start[kMaxBatch + 1];
    float2* psi[kMaxBatch];
    const float2* px[kMaxBatch];
    const float2* py[kMaxBatch];
    const int* kymax[kMaxBatch];
    int last[kMaxBatch];
};

template <int NY>
__global__ void __launch_bounds__(ColCfg<NY>::W * (NY / fft::Plan<NY>::E), ColCfg<NY>::kMinBlocks)
col_batch_kernel(const __grid_constant__ ColJobs jobs, const float2* __restrict__ twy, int nx) {
    constexpr int W = ColCfg<NY>::W;
    constexpr int PL = fft::PaddedLen<NY>::value;
    extern __shared__ float2 smem[];
    float2* tw = smem + 2 * W * PL;
    const int c = threadIdx.x % W;
    const int t = threadIdx.x / W;
    const int kx = blockIdx.x * W + c;
    const int j = find_job(jobs.start, jobs.n, blockIdx.y);
    const size_t snap = blockIdx.y - jobs.start[j];
    if (dropped_block<NY>(jobs.psi[j] + snap * NY * (size_t)nx + kx, nx, blockIdx.x * W,
                          __ldg(jobs.kymax[j] + nx), jobs.last[j], t))
        return;
    stage_twiddles<NY>(tw, twy);
    col_body<NY, false, true>(jobs.psi[j] + snap * NY * (size_t)nx + kx, nx, kx, jobs.px[j], jobs.py[j],
                              jobs.kymax[j], jobs.last[j], smem, smem + W * PL, tw, t, c);
}

// Adjoint row pass of slice s.  g holds the gradient (k_x, y) rows after the
// adjoint column pass; `state` the forward wave entering slice s in the same
// hybrid form (mode 0), or the incident wave is the unit plane wave (mode 1)
// / psi_in (mode 2).  With chi = t psi, t = exp(i sigma v):
//   g_chi = Fx^-1 g,  dL/dv = sigma Im(g_chi conj(chi)),  g_psi = conj(t) g_chi,
// and g_psi is transformed back with Fx (unless fft_out == 0: slice 0, real space).
template <int NX>
__global__ void __launch_bounds__(kRowThreads)
row_back_kernel(float2* __restrict__ g, const float2* __restrict__ state, const float* __restrict__ V,
                float* __restrict__ dV, const float2* __restrict__ psi_in,
                const float2* __restrict__ twx, const int* __restrict__ kymax, int ny, int n_slices, int s,
                float sigma, int mode, int fft_out) {
    using namespace fft;
    constexpr int E = Plan<NX>::E;
    constexpr int TPT = NX / E;
    constexpr int ROWS = kRowThreads / TPT;
    constexpr int PL = PaddedLen<NX>::value;
    extern __shared__ float2 smem[];
    float2* b0 = smem;
    float2* b1 = smem + ROWS * PL;
    float2* tw = smem + 2 * ROWS * PL;
    stage_twiddles<NX>(tw, twx);

    const int t = threadIdx.x % TPT;
    const int row = threadIdx.x / TPT;
    const int y = blockIdx.x * ROWS + row;
    const size_t snap = blockIdx.y;
    float2* grow = g + (snap * ny + y) * NX;
    const size_t vrow_off = ((snap * n_slices + s) * ny + y) * NX;
    const PadRowLayout lay{row * PL};

    // g and the hybrid state hold data only in the kept columns
    const int K = __ldg(kymax + NX);
    float2 gv[E], sv[E];
#pragma unroll
    for (int m = 0; m < E; ++m)
        gv[m] = kept_column(t + TPT * m, NX, K) ? grow[t + TPT * m] : make_float2(0.f, 0.f);
    transform<NX, true>(gv, b0, b1, t, tw, lay);
    if (mode == 0) {
        const float2* srow = state + (snap * ny + y) * NX;
#pragma unroll
        for (int m = 0; m < E; ++m)
            sv[m] = kept_column(t + TPT * m, NX, K) ? srow[t + TPT * m] : make_float2(0.f, 0.f);
        transform<NX, true>(sv, b0, b1, t, tw, lay);
    } else if (mode == 1) {
#pragma unroll
        for (int m = 0; m < E; ++m) sv[m] = make_float2(1.f, 0.f);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) sv[m] = psi_in[(size_t)y * NX + t + TPT * m];
    }
#pragma unroll
    for (int m = 0; m < E; ++m) {
        float sn, cs;
        phase_sincos(sigma * __ldg(V + vrow_off + t + TPT * m), &sn, &cs);
        const float2 tt = make_float2(cs, sn);
        const float2 chi = cmul(tt, sv[m]);
        const float2 gc = cmulc(gv[m], chi);            // g_chi conj(chi)
        dV[vrow_off + t + TPT * m] = sigma * gc.y;
        gv[m] = cmulc(gv[m], tt);                       // conj(t) g_chi
    }
    if (fft_out) transform<NX, false>(gv, b0, b1, t, tw, lay);
#pragma unroll
    for (int m = 0; m < E; ++m)
        if (!fft_out || kept_column(t + TPT * m, NX, K)) grow[t + TPT * m] = gv[m];
}

// psi_sum[q] += sum_t psi[t][q], FP64, snapshots added in order.
__global__ void snapshot_sum_kernel(const float2* __restrict__ psi, double2* __restrict__ sum,
                                    int n_t, size_t nq) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    double re = 0.0, im = 0.0;
    for (int t = 0; t < n_t; ++t) {
        const float2 v = __ldg(psi + (size_t)t * nq + q);
        re += (double)v.x;
        im += (double)v.y;
    }
    double2 acc = sum[q];
    acc.x += re;
    acc.y += im;
    sum[q] = acc;
}

// The staged row pass (slices after the first) with plan P.
template <int NX, class P>
cudaError_t launch_row_staged(float2* psi, const float* V, const float2* twx, const int* kymax, int ny, int n_t,
                              int n_slices, int s, float sigma, WaitCtl wc, cudaStream_t st, bool* launched) {
    constexpr int TPT = NX / P::E;
    constexpr int ROWS = kRowThreads / TPT;
    *launched = false;
    // one warp per row: warps with rings of their own (row_pass_warp_kernel)
    constexpr bool kWarp = TPT == 32;
    const void* kern;
    if constexpr (kWarp) kern = (const void*)row_pass_warp_kernel<NX, P>;
    else kern = (const void*)row_pass_staged_kernel<NX, P>;
    constexpr int PL = kWarp ? WarpRowLay<NX>::template slot<NX>() : fft::PaddedLen<NX>::value;
    const size_t smem = 2 * (size_t)ROWS * (PL * sizeof(float2) + NX * sizeof(float)) +
                        fft::TwSize<NX>::value * sizeof(float2) + (kWarp ? 2 * ROWS : 2) * sizeof(uint64_t);
    cudaError_t e = ensure_smem(kern, (int)smem);
    if (e != cudaSuccess) return e;
    int resident = 0;
    e = resident_blocks(kern, kRowThreads, (int)smem, &resident);
    if (e != cudaSuccess) return e;
    const long long groups = (long long)(ny / ROWS) * n_t;
    if (groups * ROWS > 0x7fffffffLL - (1LL << 24) || ny % ROWS != 0) return cudaSuccess;   // int counters
    const int n_groups = (int)groups;
    const int blocks = resident < n_groups ? resident : n_groups;
    if constexpr (kWarp)
        row_pass_warp_kernel<NX, P><<<blocks, kRowThreads, smem, st>>>(psi, V, twx, kymax, ny, n_slices, s, sigma,
                                                                      n_groups * ROWS, wc.flag, wc.polls);
    else
        row_pass_staged_kernel<NX, P><<<blocks, kRowThreads, smem, st>>>(psi, V, twx, kymax, ny, n_slices, s, sigma,
                                                                        n_groups, wc.flag, wc.polls);
    *launched = true;
    return cudaGetLastError();
}

// Row pass of slice s.  warp_rows: for 512-point rows, the staged pass with
// one warp per row (WarpPlan) instead of two.
template <int NX>
cudaError_t launch_row(float2* psi, const float* V, const float2* psi_in, const float2* twx,
                       const int* kymax, int ny, int n_t, int n_slices, int s, float sigma, int mode,
                       WaitCtl wc, bool warp_rows, cudaStream_t st) {
    constexpr int TPT = NX / fft::Plan<NX>::E;
    constexpr int ROWS = kRowThreads / TPT;
    if (mode == 0 && fft::Plan<NX>::E == 8 && reinterpret_cast<uintptr_t>(psi) % 16 == 0 &&
        reinterpret_cast<uintptr_t>(V) % 16 == 0) {
        bool launched = false;
        cudaError_t e;
        if constexpr (NX == 512) {
            if (warp_rows) e = launch_row_staged<NX, fft::WarpPlan<NX>>(psi, V, twx, kymax, ny, n_t, n_slices, s,
                                                                      sigma, wc, st, &launched);
            else e = launch_row_staged<NX, fft::Plan<NX>>(psi, V, twx, kymax, ny, n_t, n_slices, s, sigma, wc, st,
                                                         &launched);
        } else {
            e = launch_row_staged<NX, fft::Plan<NX>>(psi, V, twx, kymax, ny, n_t, n_slices, s, sigma, wc, st,
                                                    &launched);
        }
        if (e != cudaSuccess || launched) return e;
    }
    const size_t smem = (2 * ROWS * fft::PaddedLen<NX>::value + fft::TwSize<NX>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)row_pass_kernel<NX>, (int)smem);
    if (e != cudaSuccess) return e;
    int ahead = 0;
    if (reinterpret_cast<uintptr_t>(psi) % 16 == 0 && reinterpret_cast<uintptr_t>(V) % 16 == 0) {
        e = resident_blocks((const void*)row_pass_kernel<NX>, kRowThreads, (int)smem, &ahead);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(ny / ROWS, n_t);
    row_pass_kernel<NX><<<grid, kRowThreads, smem, st>>>(psi, V, psi_in, twx, kymax, ny, n_slices, s, sigma,
                                                          mode, ahead);
    return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of the waves [rows][nx] of 8-byte complex values with a box of
// box_x columns x box_y rows (no swizzle); false if the driver cannot encode it.
bool encode_wave_map(CUtensorMap* map, const void* ptr, int nx, long long rows, int box_x, int box_y) {
    static EncodeTiledFn fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        looked = true;
    }
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)nx * 8};
    const cuuint32_t box[2] = {(cuuint32_t)box_x, (cuuint32_t)box_y};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The staged column pass of the forward step (512-point columns); *launched is
// false when it does not apply (then the per-block pass runs).
template <int NY>
cudaError_t launch_col_staged(float2* psi, const float2* twy, const float2* px, const float2* py, const int* kymax,
                              int nx, int n_t, int last, WaitCtl wc, cudaStream_t st, bool* launched) {
    constexpr int TPT = NY / fft::Plan<NY>::E;
    constexpr int W = ColCfg<NY>::W;
    *launched = false;
    if (wc.flag == nullptr || reinterpret_cast<uintptr_t>(psi) % 16 != 0 || nx % W != 0) return cudaSuccess;
    CUtensorMap map;
    if (!encode_wave_map(&map, psi, nx, (long long)n_t * NY, W, NY / 2)) return cudaSuccess;
    const size_t smem = (2 * (size_t)W * StagedColLay<NY, W>::template slot<NY>() + fft::TwSize<NY>::value) *
                            sizeof(float2) + 2 * sizeof(uint64_t);
    cudaError_t e = ensure_smem((const void*)col_pass_staged_kernel<NY>, (int)smem);
    if (e != cudaSuccess) return e;
    int resident = 0;
    e = resident_blocks((const void*)col_pass_staged_kernel<NY>, W * TPT, (int)smem, &resident);
    if (e != cudaSuccess) return e;
    const long long items = (long long)n_t * (nx / W);   // at most: the kernel walks the kept blocks only
    const int blocks = (long long)resident < items ? resident : (int)items;
    col_pass_staged_kernel<NY><<<blocks, W * TPT, smem, st>>>(map, psi, twy, px, py, kymax, nx, n_t, last, wc.flag,
                                                              wc.polls);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (last) {
        zero_dropped_kernel<NY><<<dim3((nx + 127) / 128, n_t), 128, 0, st>>>(psi, kymax, nx);
        e = cudaGetLastError();
    }
    *launched = true;
    return e;
}

template <int NY, bool CONJ, bool FFT_IN>
cudaError_t launch_col_t(float2* psi, const float2* twy, const float2* px, const float2* py,
                         const int* kymax, int nx, int n_t, int last, cudaStream_t st) {
    constexpr int TPT = NY / fft::Plan<NY>::E;
    constexpr int W = ColCfg<NY>::W;
    const size_t smem = (2 * W * fft::PaddedLen<NY>::value + fft::TwSize<NY>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)col_pass_kernel<NY, CONJ, FFT_IN>, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nx / W, n_t);
    col_pass_kernel<NY, CONJ, FFT_IN><<<grid, W * TPT, smem, st>>>(psi, twy, px, py, kymax, nx, last);
    return cudaGetLastError();
}

// dir 0: forward; 1: adjoint with a leading Fy; 2: adjoint of q-space input (no leading Fy)
template <int NY>
cudaError_t launch_col(float2* psi, const float2* twy, const float2* px, const float2* py,
                       const int* kymax, int nx, int n_t, int last, cudaStream_t st, int dir = 0,
                       WaitCtl wc = WaitCtl{nullptr, 0}) {
    if constexpr (NY == 512) {
        if (dir == 0) {
            bool launched = false;
            cudaError_t e = launch_col_staged<NY>(psi, twy, px, py, kymax, nx, n_t, last, wc, st, &launched);
            if (e != cudaSuccess || launched) return e;
        }
    }
    if (dir == 0) return launch_col_t<NY, false, true>(psi, twy, px, py, kymax, nx, n_t, last, st);
    if (dir == 1) return launch_col_t<NY, true, true>(psi, twy, px, py, kymax, nx, n_t, last, st);
    return launch_col_t<NY, true, false>(psi, twy, px, py, kymax, nx, n_t, last, st);
}

template <int NX>
cudaError_t launch_row_back(float2* g, const float2* state, const float* V, float* dV,
                            const float2* psi_in, const float2* twx, const int* kymax, int ny, int n_t,
                            int n_slices, int s, float sigma, int mode, int fft_out, cudaStream_t st) {
    constexpr int TPT = NX / fft::Plan<NX>::E;
    constexpr int ROWS = kRowThreads / TPT;
    const size_t smem = (2 * ROWS * fft::PaddedLen<NX>::value + fft::TwSize<NX>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)row_back_kernel<NX>, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ny / ROWS, n_t);
    row_back_kernel<NX><<<grid, kRowThreads, smem, st>>>(g, state, V, dV, psi_in, twx, kymax, ny, n_slices,
                                                          s, sigma, mode, fft_out);
    return cudaGetLastError();
}

#define TACAW_SIZE_SWITCH(n, CALL)                  \
    switch (n) {                                    \
        case 64: { constexpr int N_ = 64; CALL; }   \
        case 128: { constexpr int N_ = 128; CALL; } \
        case 256: { constexpr int N_ = 256; CALL; } \
        case 384: { constexpr int N_ = 384; CALL; } \
        case 512: { constexpr int N_ = 512; CALL; } \
        case 768: { constexpr int N_ = 768; CALL; } \
        case 1024: { constexpr int N_ = 1024; CALL; } \
    }

cudaError_t dispatch_row(int nx, float2* psi, const float* V, const float2* psi_in, const float2* twx,
                         const int* kymax, int ny, int n_t, int n_slices, int s, float sigma, int mode,
                         WaitCtl wc, cudaStream_t st, bool warp_rows = false) {
    TACAW_SIZE_SWITCH(nx, return launch_row<N_>(psi, V, psi_in, twx, kymax, ny, n_t, n_slices, s, sigma, mode, wc,
                                                warp_rows, st));
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_col(int ny, float2* psi, const float2* twy, const float2* px, const float2* py,
                         const int* kymax, int nx, int n_t, int last, cudaStream_t st, int dir = 0,
                         WaitCtl wc = WaitCtl{nullptr, 0}) {
    switch (ny) {
        case 64: return launch_col<64>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
        case 128: return launch_col<128>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
        case 256: return launch_col<256>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
        case 512: return launch_col<512>(psi, twy, px, py, kymax, nx, n_t, last, st, dir, wc);
        case 1024: return launch_col<1024>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
        case 384: return launch_col<384>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
        case 768: return launch_col<768>(psi, twy, px, py, kymax, nx, n_t, last, st, dir);
    }
    return cudaErrorInvalidValue;
}

template <int NX>
cudaError_t launch_row_batch(const RowJobs& jobs, const float2* twx, int ny, int total, int s, cudaStream_t st) {
    constexpr int TPT = NX / fft::Plan<NX>::E;
    constexpr int ROWS = kRowThreads / TPT;
    const size_t smem = (2 * ROWS * fft::PaddedLen<NX>::value + fft::TwSize<NX>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)row_batch_kernel<NX>, (int)smem);
    if (e != cudaSuccess) return e;
    row_batch_kernel<NX><<<dim3(ny / ROWS, total), kRowThreads, smem, st>>>(jobs, twx, ny, s);
    return cudaGetLastError();
}

template <int NY>
cudaError_t launch_col_batch(const ColJobs& jobs, const float2* twy, int nx, int total, cudaStream_t st) {
    constexpr int TPT = NY / fft::Plan<NY>::E;
    constexpr int W = ColCfg<NY>::W;
    const size_t smem = (2 * W * fft::PaddedLen<NY>::value + fft::TwSize<NY>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)col_batch_kernel<NY>, (int)smem);
    if (e != cudaSuccess) return e;
    col_batch_kernel<NY><<<dim3(nx / W, total), W * TPT, smem, st>>>(jobs, twy, nx);
    return cudaGetLastError();
}

cudaError_t dispatch_row_batch(int nx, const RowJobs& jobs, const float2* twx, int ny, int total, int s,
                               cudaStream_t st) {
    TACAW_SIZE_SWITCH(nx, return launch_row_batch<N_>(jobs, twx, ny, total, s, st));
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_col_batch(int ny, const ColJobs& jobs, const float2* twy, int nx, int total,
                               cudaStream_t st) {
    TACAW_SIZE_SWITCH(ny, return launch_col_batch<N_>(jobs, twy, nx, total, st));
    return cudaErrorInvalidValue;
}

cudaError_t dispatch_row_back(int nx, float2* g, const float2* state, const float* V, float* dV,
                              const float2* psi_in, const float2* twx, const int* kymax, int ny, int n_t,
                              int n_slices, int s, float sigma, int mode, int fft_out, cudaStream_t st) {
    TACAW_SIZE_SWITCH(nx, return launch_row_back<N_>(g, state, V, dV, psi_in, twx, kymax, ny, n_t, n_slices, s,
                                                     sigma, mode, fft_out, st));
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ work queue
// Persistent multislice over a device work queue, for jobs whose grids are
// square (nx = ny = N).  An item is one pass of one slice over kQSpan rows
// (row item) or kQSpan columns (column item) of one snapshot; a resident
// grid of 256-thread blocks takes items from a global counter in a fixed
// order.  The order runs the snapshots of a job in waves of `wave` snapshots:
// within a wave, slice 0 row items of every snapshot, then slice 0 column
// items, then slice 1 row items, and so on, so between the passes of a
// snapshot the blocks touch only the wave's other snapshots and the wave's
// waves stay in L2.  A row item of slice s needs the column items of slice
// s - 1 of its snapshot, a column item the row items of slice s: per-snapshot
// counters of finished items (release after the item's stores, acquire before
// its loads).  Every item an item waits on comes earlier in the order and is
// held by a running block, so the waits end; each is bounded all the same
// (then the status flag and the call's abort word are set and every block
// leaves).  Results equal the per-slice launches' bit for bit: same plans,
// twiddles, layouts and per-point arithmetic.
constexpr int kQThreads = 256;
constexpr int kQMaxJobs = 64;
constexpr int kQSpan = 16;               // default rows (row item) or columns (column item) per item

template <int N>
struct QCfg {
    static constexpr int E = fft::Plan<N>::E;
    static constexpr int TPT = N / E;                 // threads per transform
    static constexpr int ROWS = kQThreads / TPT;      // rows per row tile = columns per column tile
    static constexpr int SPAN = ROWS > kQSpan ? ROWS : kQSpan;   // default span
    // row-tile exchange layout: for the 24-value plans (two blocks per SM whatever the stage size)
    // the second and later exchanges as p + 8 (p / 64), free of half-warp bank collisions; the
    // 8-value plans keep p + p / 16 everywhere (longer rows would cost them a resident block)
    using RowLay = typename std::conditional<E == 24, fft::PadRowL<fft::Pad16, fft::Pad64x8>, fft::PadRowLayout>::type;
    static constexpr int PL = RowLay::template slot<N>();
    static_assert(PL % 2 == 0, "16-byte aligned rows");
    static constexpr int MIN_BLOCKS = E > 8 ? 2 : 4;    // resident blocks per SM the registers allow
    static_assert(ROWS * TPT == kQThreads && N % SPAN == 0, "queue tiles");
    // a span (rows or columns per item) is a multiple of ROWS that divides N
    static constexpr bool valid_span(int span) { return span >= ROWS && span % ROWS == 0 && N % span == 0; }
};

struct QJobs {
    int n;                                // jobs in this launch
    int wave;                             // snapshots per wave
    int span;                             // rows (row item) or columns (column item) per item
    int items;                            // items per snapshot and pass: N / span
    long long item0[kQMaxJobs + 1];       // first queue position of each job; item0[n] = total
    int snap0[kQMaxJobs + 1];             // first counter slot of each job
    float2* psi[kQMaxJobs];
    const float* V[kQMaxJobs];
    const float2* psi_in[kQMaxJobs];
    const float2* px[kQMaxJobs];
    const float2* py[kQMaxJobs];
    const int* kymax[kQMaxJobs];
    int n_t[kQMaxJobs], n_slices[kQMaxJobs];
    float sigma[kQMaxJobs];
    // per job: the exit waves as a 2-D array of 8-byte elements [n_t * N][N], boxes of
    // (ROWS columns) x (qbox rows) for the column tiles
    alignas(64) CUtensorMap cmap[kQMaxJobs];
};

struct QItem {
    int job, t, s, pass, tile;
};

// (The host keeps every job's item count below 2^31, so positions within a job
// are 32-bit.)
__device__ __forceinline__ QItem q_decode(const QJobs& jobs, long long it) {
    const int IT = jobs.items;
    QItem q;
    int j = 0;
    while (j + 1 < jobs.n && jobs.item0[j + 1] <= it) ++j;
    const int r = (int)(it - jobs.item0[j]);
    const int S = jobs.n_slices[j], T = jobs.n_t[j], Tw = jobs.wave;
    const int per_wave = S * 2 * IT * Tw;
    const int w = r / per_wave;
    const int first = w * Tw;
    const int nw = min(Tw, T - first);
    const int in_wave = r - w * per_wave;
    const int s = in_wave / (2 * nw * IT);
    int rem = in_wave - s * 2 * nw * IT;
    const int pass = rem >= nw * IT ? 1 : 0;
    if (pass) rem -= nw * IT;
    q.job = j;
    q.t = first + rem / IT;
    q.s = s;
    q.pass = pass;
    q.tile = rem % IT;
    return q;
}

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: waits until *ctr >= need, at most `polls` polls, leaving early when
// the call's abort word is set.  On giving up it sets the status flag and the
// abort word.  Returns whether the count was reached.
__device__ bool q_wait(const int* ctr, int need, int* abort_word, int* err, uint32_t polls) {
    for (uint32_t i = 0; i < polls; ++i) {
        if (ld_acquire_gpu(ctr) >= need) return true;
        if (*reinterpret_cast<volatile int*>(abort_word)) return false;
        __nanosleep(32);
    }
    atomicExch(err, 1);
    atomicExch(abort_word, 1);
    return false;
}

// A tile's stage: ROWS slots of PL float2 (row tile: the rows of psi at their
// natural positions, then the padded exchanges in place; column tile: the
// ROWS x N columns densely as [row][column], then the padded exchanges in
// place), followed by the tile's ROWS rows of v_s (row tiles).
template <int N>
struct QStage {
    static constexpr int PSI = QCfg<N>::ROWS * QCfg<N>::PL;             // float2
    static constexpr int F2 = PSI + QCfg<N>::ROWS * N / 2;              // float2 per stage
    static constexpr int NST = (2 * F2 + fft::TwSize<N>::value) * (int)sizeof(float2) <= 100 * 1024 ? 2 : 1;
};

// Rows of the column tiles' TMA boxes (at most 256 per box; N / qbox boxes per tile).
template <int N>
struct QBox {
    static constexpr int ROWS = N <= 256 ? N : (N % 256 == 0 ? 256 : N / 2);
    static constexpr int COUNT = N / ROWS;
    static_assert(ROWS <= 256 && N % ROWS == 0, "column-tile boxes");
};

// Thread 0: starts the asynchronous copies of tile ti of item q into a stage,
// completing on the stage's mbarrier: a row tile takes its rows of psi (the
// kept columns, from the second slice on; bulk copies of the two kept ranges of
// each row) and of v_s (one bulk copy), a column tile its ROWS columns (TMA
// boxes of the job's map); a tile the band limit drops arrives without bytes.
// The inputs were written by other blocks with ordinary stores and acquired
// through their counters, and the stage was last used by ordinary accesses:
// proxy fences order both before the copies.  16-byte aligned arrays.
template <int N>
__device__ __forceinline__ void q_issue(const QJobs& jobs, const QItem& q, int ti, float2* stage, uint64_t* bar) {
    using C = QCfg<N>;
    asm volatile("fence.proxy.async.global;" ::: "memory");
    fence_proxy_async_smem();
    const float2* snap = jobs.psi[q.job] + (size_t)q.t * N * N;
    const int K = __ldg(jobs.kymax[q.job] + N);
    if (q.pass == 0) {
        const int y0 = q.tile * jobs.span + ti * C::ROWS;
        int a = K + 1;                                   // kept columns [0, a) and [b, N), both ends even
        a += a & 1;
        if (a > N) a = N;
        int b = N - K;
        b -= b & 1;
        if (b < a) b = a;
        constexpr uint32_t V_BYTES = C::ROWS * N * (uint32_t)sizeof(float);
        const uint32_t psi_bytes = q.s > 0 ? (uint32_t)(C::ROWS * (a + N - b) * (int)sizeof(float2)) : 0u;
        tc::mbar_arrive_expect_tx(bar, psi_bytes + V_BYTES);
        if (q.s > 0) {
            const float2* rows = snap + (size_t)y0 * N;
            for (int r = 0; r < C::ROWS; ++r) {
                if (a > 0) bulk_copy_g2s(stage + r * C::PL, rows + (size_t)r * N, a * (uint32_t)sizeof(float2), bar);
                if (b < N)
                    bulk_copy_g2s(stage + r * C::PL + b, rows + (size_t)r * N + b, (N - b) * (uint32_t)sizeof(float2),
                                  bar);
            }
        }
        const float* Vs = jobs.V[q.job] + (((size_t)q.t * jobs.n_slices[q.job] + q.s) * N + y0) * N;
        bulk_copy_g2s(stage + QStage<N>::PSI, Vs, V_BYTES, bar);
    } else {
        const int kx0 = q.tile * jobs.span + ti * C::ROWS;
        if (kx0 > K && kx0 + C::ROWS - 1 < N - K) {
            tc::mbar_arrive(bar);
            return;
        }
        tc::mbar_arrive_expect_tx(bar, (uint32_t)(N * C::ROWS * (int)sizeof(float2)));
#pragma unroll
        for (int k = 0; k < QBox<N>::COUNT; ++k)
            tc::tma_load_2d(stage + k * QBox<N>::ROWS * C::ROWS, &jobs.cmap[q.job], bar, kx0,
                            q.t * N + k * QBox<N>::ROWS);
    }
}

// Row tile from its stage: ROWS rows of one snapshot (mode 0: the hybrid wave;
// 1: unit plane wave; 2: psi_in) transmitted by slice s and transformed back
// along x, kept columns written to the wave.
template <int N>
__device__ __forceinline__ void q_row_tile(float2* stage, float2* __restrict__ rowp, const float2* __restrict__ inrow,
                                           int mode, float sigma, int K, const float2* tw, int t, int row) {
    using namespace fft;
    using C = QCfg<N>;
    constexpr int E = C::E, TPT = C::TPT;
    const typename C::RowLay lay{row * C::PL};
    const auto sync = row_sync_of<TPT>(row);
    const float* vrow = reinterpret_cast<const float*>(stage + QStage<N>::PSI) + row * N;
    float2 v[E];
    if (mode == 0) {
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[m] = kept_column(t + TPT * m, N, K) ? stage[row * C::PL + t + TPT * m] : make_float2(0.f, 0.f);
        transform_plan<Plan<N>, N, true>(v, stage, stage, t, tw, lay, sync);
    } else if (mode == 1) {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = make_float2(1.f, 0.f);
    } else {
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = __ldg(inrow + t + TPT * m);
    }
    float x[E];
#pragma unroll
    for (int m = 0; m < E; ++m) x[m] = sigma * vrow[t + TPT * m];
    transmit<E>(v, x);
    transform_plan<Plan<N>, N, false>(v, stage, stage, t, tw, lay, sync);
#pragma unroll
    for (int m = 0; m < E; ++m)
        if (kept_column(t + TPT * m, N, K)) rowp[t + TPT * m] = v[m];
}

// Column tile from its stage: ROWS adjacent columns (Fy, times P BL / (nx ny),
// Fy^-1 unless `last`); a tile the band limit drops entirely only writes its
// zeros after the last slice.
template <int N>
__device__ __forceinline__ void q_col_tile(float2* stage, float2* __restrict__ snap, int kx0,
                                           const float2* __restrict__ px, const float2* __restrict__ py,
                                           const int* __restrict__ kymax, int K, int last, const float2* tw, int t,
                                           int c) {
    using namespace fft;
    using C = QCfg<N>;
    constexpr int E = C::E, TPT = C::TPT, W = C::ROWS;
    float2* col = snap + kx0 + c;
    if (kx0 > K && kx0 + W - 1 < N - K) {
        if (last) {
#pragma unroll
            for (int m = 0; m < E; ++m) col[(size_t)(t + TPT * m) * N] = make_float2(0.f, 0.f);
        }
        return;
    }
    const int kx = kx0 + c;
    // at 512 points (four columns) and for the 24-value plans (eight or sixteen columns) the first
    // exchange as p + p / 8, free of half-warp bank collisions, the others as p + p / 16
    using Lay = typename std::conditional<N == 512 || E == 24, fft::PadColLayout512<W>, fft::PadColLayout<W>>::type;
    static_assert(Lay::template slot<N>() * W <= QStage<N>::F2, "column tile fits its stage");
    const Lay lay{c};
    float2 v[E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = stage[(t + TPT * m) * W + c];
    transform_plan<Plan<N>, N, false>(v, stage, stage, t, tw, lay, BlockSync{});
    const float2 pxv = __ldg(px + kx);
    const int kmax = __ldg(kymax + kx);
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int ky = t + TPT * m;
        const int aky = ky < N / 2 ? ky : N - ky;
        v[m] = (aky <= kmax) ? cmul(v[m], cmul(pxv, __ldg(py + ky))) : make_float2(0.f, 0.f);
    }
    if (!last) transform_plan<Plan<N>, N, true>(v, stage, stage, t, tw, lay, BlockSync{});
#pragma unroll
    for (int m = 0; m < E; ++m) col[(size_t)(t + TPT * m) * N] = v[m];
}

__device__ __forceinline__ bool q_ready(const QJobs& jobs, const QItem& q, const int* row_done, const int* col_done) {
    const int u = jobs.snap0[q.job] + q.t;
    if (q.pass == 0) return q.s == 0 || ld_acquire_gpu(col_done + u) >= q.s * jobs.items;
    return ld_acquire_gpu(row_done + u) >= (q.s + 1) * jobs.items;
}

__device__ __forceinline__ bool q_wait_ready(const QJobs& jobs, const QItem& q, int* row_done, int* col_done,
                                             int* abort_word, int* err, uint32_t polls) {
    const int u = jobs.snap0[q.job] + q.t;
    if (q.pass == 0) return q.s == 0 || q_wait(col_done + u, q.s * jobs.items, abort_word, err, polls);
    return q_wait(row_done + u, (q.s + 1) * jobs.items, abort_word, err, polls);
}

// ctl (8-byte aligned): [0, 1] 64-bit queue head, [2] abort word, [3] unused;
// then row_done[U], col_done[U].  All zero before the launch.
// Each block walks its tiles through a ring of QStage<N>::NST stages, each
// with an mbarrier: while tile k is transformed, the copies of tile k + 1 (the
// next tile of the same item, or the first of the block's next item once that
// item's inputs are final) are in flight.  Thread 0 takes items from the
// queue, decodes them, plans the tile after next and issues the copies; every
// thread waits on the stage's mbarrier (bounded: a wait that gives up sets the
// status flag and the abort word, and the block drains its copies and leaves).
// Two barriers per tile: after the wait (a thread that gave up tells the
// others), and at the end of the tile's use of the stage (which also
// publishes the plan).  Lane 0 of warp 1 releases finished items, so that the
// release's fence does not hold up the next copies.
template <int N>
__global__ void __launch_bounds__(kQThreads, QCfg<N>::MIN_BLOCKS)
ms_queue_kernel(const __grid_constant__ QJobs jobs, const float2* __restrict__ tw_g, int* __restrict__ ctl,
                int* __restrict__ err, uint32_t polls) {
    using C = QCfg<N>;
    constexpr int NST = QStage<N>::NST;
    extern __shared__ __align__(128) float2 qsm[];
    float2* tw = qsm + NST * QStage<N>::F2;
    __shared__ __align__(8) uint64_t bars[2];
    // written by thread 0, read by all threads between two barriers: the first item; the plan of
    // the next tile (item, tile in item, 0 ready / 1 inputs not final yet / 2 none); the verdict of
    // a blocking wait
    __shared__ QItem s_first, s_next;
    __shared__ int s_first_ok, s_next_ti, s_next_flag, s_ok;
    unsigned long long* head = reinterpret_cast<unsigned long long*>(ctl);
    int* abort_word = ctl + 2;
    const int U = jobs.snap0[jobs.n];
    int* row_done = ctl + 4;
    int* col_done = ctl + 4 + U;
    const long long total = jobs.item0[jobs.n];
    const int tiles = jobs.span / C::ROWS;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
    }
    stage_twiddles<N>(tw, tw_g);
    const int tr = threadIdx.x % C::TPT, row = threadIdx.x / C::TPT;     // row tiles
    const int cc = threadIdx.x % C::ROWS, tc_ = threadIdx.x / C::ROWS;    // column tiles
    // thread 0: the block's next item, taken when the tile before the last of the current item is
    // planned (with the current item when items are one tile), so that few items are taken but
    // not started and the queue's latency hides behind a tile
    unsigned long long nxt = 0;
    bool have_nxt = false;
    auto plan = [&](const QItem& pq, int pti) {     // thread 0: the tile after (pq, pti)
        if (pti + 1 < tiles) {
            s_next = pq;
            s_next_ti = pti + 1;
            s_next_flag = 0;
            if (pti + 2 == tiles && !have_nxt) {
                nxt = atomicAdd(head, 1ull);
                have_nxt = true;
            }
            return;
        }
        if (!have_nxt) nxt = atomicAdd(head, 1ull);
        have_nxt = false;
        if ((long long)nxt >= total || *reinterpret_cast<volatile int*>(abort_word)) {
            s_next_flag = 2;
            return;
        }
        const QItem qd = q_decode(jobs, (long long)nxt);
        s_next = qd;
        s_next_ti = 0;
        s_next_flag = q_ready(jobs, qd, row_done, col_done) ? 0 : 1;
        if (tiles == 1) {
            nxt = atomicAdd(head, 1ull);
            have_nxt = true;
        }
    };
    if (threadIdx.x == 0) {
        const unsigned long long cur = atomicAdd(head, 1ull);
        s_first_ok = 0;
        if ((long long)cur < total) {
            s_first = q_decode(jobs, (long long)cur);
            s_first_ok = q_wait_ready(jobs, s_first, row_done, col_done, abort_word, err, polls);
        }
    }
    __syncthreads();
    if (!s_first_ok) return;
    QItem q = s_first;
    int ti = 0, st = 0;
    uint32_t uses[2] = {0u, 0u};                    // completed phases of each stage's mbarrier
    bool pending[2] = {true, false};                // a phase of the stage is in flight (thread 0 view)
    if (threadIdx.x == 0) {
        q_issue<N>(jobs, q, 0, qsm, &bars[0]);
        plan(q, 0);
    }
    __syncthreads();
    bool failed = false;
    for (;;) {
        const int flag = s_next_flag;
        const int nti = s_next_ti;
        const QItem qn = flag == 2 ? q : s_next;
        const int st_next = st ^ (NST - 1);
        float2* cur_stage = qsm + st * QStage<N>::F2;
        float2* nxt_stage = qsm + st_next * QStage<N>::F2;
        const bool early = NST == 2 && flag == 0;
        if (early && threadIdx.x == 0) {
            q_issue<N>(jobs, qn, nti, nxt_stage, &bars[st_next]);
            pending[st_next] = true;
        }
        const bool ok = tc::mbar_wait_quiet(&bars[st], uses[st] & 1u, polls);
        if (__syncthreads_or(!ok)) {                // this tile's copies never arrived
            if (threadIdx.x == 0) {
                atomicExch(err, 1);
                atomicExch(abort_word, 1);
            }
            failed = true;
            break;
        }
        ++uses[st];
        if (threadIdx.x == 0) pending[st] = false;
        const int S = jobs.n_slices[q.job];
        float2* snap = jobs.psi[q.job] + (size_t)q.t * N * N;
        const int K = __ldg(jobs.kymax[q.job] + N);
        if (q.pass == 0) {
            const int mode = q.s > 0 ? 0 : (jobs.psi_in[q.job] ? 2 : 1);
            const int y = q.tile * jobs.span + ti * C::ROWS + row;
            q_row_tile<N>(cur_stage, snap + (size_t)y * N,
                          mode == 2 ? jobs.psi_in[q.job] + (size_t)y * N : nullptr, mode, jobs.sigma[q.job], K,
                          tw, tr, row);
        } else {
            q_col_tile<N>(cur_stage, snap, q.tile * jobs.span + ti * C::ROWS, jobs.px[q.job], jobs.py[q.job],
                          jobs.kymax[q.job], K, q.s + 1 == S, tw, tc_, cc);
        }
        if (threadIdx.x == 0 && flag != 2) plan(qn, nti);
        __syncthreads();                            // the stage is free; the tile's stores are issued
        if (ti + 1 == tiles && threadIdx.x == 32) { // the item is done: warp 1 releases it while thread 0
            asm volatile("fence.proxy.async.global;" ::: "memory");   // goes on to the next copies
            __threadfence();
            atomicAdd((q.pass == 0 ? row_done : col_done) + jobs.snap0[q.job] + q.t, 1);
        }
        if (flag == 2) break;
        if (!early) {                               // inputs not final yet, or one stage: wait, then copy
            if (threadIdx.x == 0) {
                s_ok = flag == 0 || q_wait_ready(jobs, qn, row_done, col_done, abort_word, err, polls);
                if (s_ok) {
                    q_issue<N>(jobs, qn, nti, nxt_stage, &bars[st_next]);
                    pending[st_next] = true;
                }
            }
            __syncthreads();
            if (!s_ok) break;
        }
        q = qn;
        ti = nti;
        st = st_next;
    }
    if (failed && threadIdx.x == 0) {               // copies still in flight land before the block leaves
        for (int k = 0; k < 2; ++k)
            if (pending[k])
                for (int i = 0; i < 64 && !tc::mbar_wait_quiet(&bars[k], uses[k] & 1u, 1u << 20); ++i) {
                }
    }
}

}  // namespace

bool multislice_size_supported(int n) {
    return n == 64 || n == 128 || n == 256 || n == 384 || n == 512 || n == 768 || n == 1024;
}

struct MsTables {
    float2 *twx, *twy, *px, *py;
    int* kymax;
};

static MsTables carve_ms(Carver& cv, const tacaw_grid& g) {
    MsTables t;
    t.twx = cv.take<float2>(g.nx);
    t.twy = cv.take<float2>(g.ny);
    t.px = cv.take<float2>(g.nx);
    t.py = cv.take<float2>(g.ny);
    t.kymax = cv.take<int>(g.nx + 1);   // + K (see ms_setup_kernel)
    return t;
}

size_t multislice_ws_bytes(const tacaw_grid& g) {
    Carver cv(nullptr);
    carve_ms(cv, g);
    return cv.bytes();
}

// Default poll limit of the staged row pass's waits (about a second or more).
constexpr uint32_t kRowWaitPolls = 1u << 24;

int multislice_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                   float2* psi_q, double2* psi_sum, void* ws, cudaStream_t st, int flags) {
    const bool warp_rows = (flags & TACAW_MS_WARP_ROWS) != 0;
    const bool block_cols = (flags & TACAW_MS_BLOCK_COLS) != 0;
    Carver cv(ws);
    MsTables tb = carve_ms(cv, g);
    WaitCtl wc{nullptr, wait_polls(kRowWaitPolls)};
    int rc = timeout_flag(&wc.flag, "tacaw_multislice");
    if (rc) return rc;
    double lam = 0.0, sig = 0.0;
    beam_constants(g.kev, &lam, &sig);
    const double qmax = g.bandlimit * fmin((double)g.nx / (2.0 * g.lx), (double)g.ny / (2.0 * g.ly));
    const double qmax2 = qmax * qmax;
    const int nmax = g.nx > g.ny ? g.nx : g.ny;
    ms_setup_kernel<<<(nmax + 127) / 128, 128, 0, st>>>(tb.twx, tb.twy, tb.px, tb.py, tb.kymax,
                                                       g.nx, g.ny, g.lx, g.ly, lam * g.dz, qmax2);
    TACAW_LAUNCH_CHECK();
    const float sigma = (float)sig;
    for (int s = 0; s < g.n_slices; ++s) {
        const int mode = s > 0 ? 0 : (psi_in ? 2 : 1);
        TACAW_CUDA_CHECK(dispatch_row(g.nx, psi_q, V, psi_in, tb.twx, tb.kymax, g.ny, n_t, g.n_slices, s,
                                      sigma, mode, wc, st, warp_rows));
        TACAW_CUDA_CHECK(dispatch_col(g.ny, psi_q, tb.twy, tb.px, tb.py, tb.kymax, g.nx, n_t,
                                      s + 1 == g.n_slices, st, 0, block_cols ? WaitCtl{nullptr, 0} : wc));
    }
    if (psi_sum) {
        const size_t nq = (size_t)g.nx * g.ny;
        snapshot_sum_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>(psi_q, psi_sum, n_t, nq);
        TACAW_LAUNCH_CHECK();
    }
    return TACAW_OK;
}

// ------------------------------------------------------------------ batch
size_t multislice_batch_ws_bytes(const tacaw_job* jobs, int n_jobs) {
    Carver cv(nullptr);
    for (int j = 0; j < n_jobs; ++j) carve_ms(cv, jobs[j].grid);
    return cv.bytes();
}

// Uneven jobs in one call: per-job set-up tables, then for every slice index
// one row launch and one column launch per grid size covering all jobs of
// that size that still have slices left (in chunks of at most kMaxBatch jobs
// and 65535 snapshots), so small jobs share launches with large ones.
int multislice_batch_run(const tacaw_job* jobs, int n_jobs, void* ws, cudaStream_t st) {
    Carver cv(ws);
    std::vector<MsTables> tb(n_jobs);
    std::vector<float> sigma(n_jobs);
    int max_ns = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const tacaw_grid& g = jobs[j].grid;
        tb[j] = carve_ms(cv, g);
        double lam = 0.0, sig = 0.0;
        beam_constants(g.kev, &lam, &sig);
        sigma[j] = (float)sig;
        const double qmax = g.bandlimit * fmin((double)g.nx / (2.0 * g.lx), (double)g.ny / (2.0 * g.ly));
        const int nmax = g.nx > g.ny ? g.nx : g.ny;
        ms_setup_kernel<<<(nmax + 127) / 128, 128, 0, st>>>(tb[j].twx, tb[j].twy, tb[j].px, tb[j].py,
                                                           tb[j].kymax, g.nx, g.ny, g.lx, g.ly,
                                                           lam * g.dz, qmax * qmax);
        TACAW_LAUNCH_CHECK();
        if (jobs[j].n_t > 0) max_ns = max_ns > g.n_slices ? max_ns : g.n_slices;
    }
    std::vector<char> used(n_jobs);
    for (int s = 0; s < max_ns; ++s) {
        std::fill(used.begin(), used.end(), 0);
        for (int j0 = 0; j0 < n_jobs; ++j0) {
            const tacaw_job& a = jobs[j0];
            if (used[j0] || a.n_t <= 0 || s >= a.grid.n_slices) continue;
            // all remaining jobs of this grid size with slice s to do, in chunks
            std::vector<int> group;
            for (int j = j0; j < n_jobs; ++j) {
                const tacaw_job& b = jobs[j];
                if (!used[j] && b.n_t > 0 && s < b.grid.n_slices && b.grid.nx == a.grid.nx &&
                    b.grid.ny == a.grid.ny) {
                    group.push_back(j);
                    used[j] = 1;
                }
            }
            size_t gi = 0;
            while (gi < group.size()) {
                RowJobs rj;
                ColJobs cj;
                rj.n = cj.n = 0;
                int total = 0;
                while (gi < group.size() && rj.n < kMaxBatch && total + jobs[group[gi]].n_t <= 65535) {
                    const int j = group[gi++];
                    const tacaw_job& b = jobs[j];
                    const int k = rj.n++;
                    cj.n = rj.n;
                    rj.start[k] = cj.start[k] = total;
                    rj.psi[k] = cj.psi[k] = (float2*)b.psi_q;
                    rj.V[k] = b.V;
                    rj.psi_in[k] = (const float2*)b.psi_in;
                    rj.kymax[k] = tb[j].kymax;
                    rj.n_slices[k] = b.grid.n_slices;
                    rj.mode[k] = s > 0 ? 0 : (b.psi_in ? 2 : 1);
                    rj.sigma[k] = sigma[j];
                    cj.px[k] = tb[j].px;
                    cj.py[k] = tb[j].py;
                    cj.kymax[k] = tb[j].kymax;
                    cj.last[k] = (s + 1 == b.grid.n_slices) ? 1 : 0;
                    total += b.n_t;
                }
                rj.start[rj.n] = cj.start[cj.n] = total;
                const int first = group[0];
                TACAW_CUDA_CHECK(dispatch_row_batch(a.grid.nx, rj, tb[first].twx, a.grid.ny, total, s, st));
                TACAW_CUDA_CHECK(dispatch_col_batch(a.grid.ny, cj, tb[first].twy, a.grid.nx, total, st));
            }
        }
    }
    for (int j = 0; j < n_jobs; ++j) {
        if (!jobs[j].psi_sum || jobs[j].n_t <= 0) continue;
        const size_t nq = (size_t)jobs[j].grid.nx * jobs[j].grid.ny;
        snapshot_sum_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>((const float2*)jobs[j].psi_q,
                                                                         (double2*)jobs[j].psi_sum,
                                                                         jobs[j].n_t, nq);
        TACAW_LAUNCH_CHECK();
    }
    return TACAW_OK;
}

// ------------------------------------------------------------------ work queue (host)
namespace {

constexpr uint32_t kQueueWaitPolls = 1u << 22;   // a few seconds per dependency wait
constexpr double kQueueWaveBytes = 128.0 * 1024 * 1024;  // default wave: about 128 MiB of exit waves

// Columns of a column tile and rows of its TMA boxes, for grid size n.
void queue_tile_dims(int n, int* cols, int* box_rows) {
    switch (n) {
        case 64: *cols = QCfg<64>::ROWS; *box_rows = QBox<64>::ROWS; return;
        case 128: *cols = QCfg<128>::ROWS; *box_rows = QBox<128>::ROWS; return;
        case 256: *cols = QCfg<256>::ROWS; *box_rows = QBox<256>::ROWS; return;
        case 384: *cols = QCfg<384>::ROWS; *box_rows = QBox<384>::ROWS; return;
        case 512: *cols = QCfg<512>::ROWS; *box_rows = QBox<512>::ROWS; return;
        case 768: *cols = QCfg<768>::ROWS; *box_rows = QBox<768>::ROWS; return;
        case 1024: *cols = QCfg<1024>::ROWS; *box_rows = QBox<1024>::ROWS; return;
    }
    *cols = *box_rows = 0;
}

// The span for grid size n: the requested one where valid, else the default.
int queue_span(int n, int want) {
    switch (n) {
        case 64: return QCfg<64>::valid_span(want) ? want : QCfg<64>::SPAN;
        case 128: return QCfg<128>::valid_span(want) ? want : QCfg<128>::SPAN;
        case 256: return QCfg<256>::valid_span(want) ? want : QCfg<256>::SPAN;
        case 384: return QCfg<384>::valid_span(want) ? want : QCfg<384>::SPAN;
        case 512: return QCfg<512>::valid_span(want) ? want : QCfg<512>::SPAN;
        case 768: return QCfg<768>::valid_span(want) ? want : QCfg<768>::SPAN;
        case 1024: return QCfg<1024>::valid_span(want) ? want : QCfg<1024>::SPAN;
    }
    return 0;
}

template <int N>
cudaError_t launch_queue(const QJobs& jobs, const float2* tw, int* ctl, int* err, uint32_t polls, cudaStream_t st) {
    const size_t smem = (QStage<N>::NST * QStage<N>::F2 + fft::TwSize<N>::value) * sizeof(float2);
    cudaError_t e = ensure_smem((const void*)ms_queue_kernel<N>, (int)smem);
    if (e != cudaSuccess) return e;
    int resident = 0;
    e = resident_blocks((const void*)ms_queue_kernel<N>, kQThreads, (int)smem, &resident);
    if (e != cudaSuccess) return e;
    const long long total = jobs.item0[jobs.n];
    const int blocks = (long long)resident < total ? resident : (int)total;
    if (blocks <= 0) return cudaSuccess;
    ms_queue_kernel<N><<<blocks, kQThreads, smem, st>>>(jobs, tw, ctl, err, polls);
    return cudaGetLastError();
}

cudaError_t dispatch_queue(int n, const QJobs& jobs, const float2* tw, int* ctl, int* err, uint32_t polls,
                           cudaStream_t st) {
    TACAW_SIZE_SWITCH(n, return launch_queue<N_>(jobs, tw, ctl, err, polls, st));
    return cudaErrorInvalidValue;
}

}  // namespace

size_t multislice_queue_ws_bytes(const tacaw_job* jobs, int n_jobs) {
    Carver cv(nullptr);
    long long U = 0;
    for (int j = 0; j < n_jobs; ++j) {
        carve_ms(cv, jobs[j].grid);
        if (jobs[j].n_t > 0) U += jobs[j].n_t;
    }
    cv.take<int>((size_t)(4 + 2 * U));
    return cv.bytes();
}

// Jobs grouped by grid size (in order of first appearance, at most kQMaxJobs
// per launch): per group one persistent launch over the group's queue, after
// a reset of its counters; then the FP64 snapshot sums.
int multislice_queue_run(const tacaw_job* jobs, int n_jobs, int wave, int span, void* ws, cudaStream_t st) {
    Carver cv(ws);
    std::vector<MsTables> tb(n_jobs);
    std::vector<float> sigma(n_jobs);
    long long U = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const tacaw_grid& g = jobs[j].grid;
        tb[j] = carve_ms(cv, g);
        double lam = 0.0, sig = 0.0;
        beam_constants(g.kev, &lam, &sig);
        sigma[j] = (float)sig;
        const double qmax = g.bandlimit * fmin((double)g.nx / (2.0 * g.lx), (double)g.ny / (2.0 * g.ly));
        ms_setup_kernel<<<(g.nx + 127) / 128, 128, 0, st>>>(tb[j].twx, tb[j].twy, tb[j].px, tb[j].py,
                                                            tb[j].kymax, g.nx, g.ny, g.lx, g.ly, lam * g.dz,
                                                            qmax * qmax);
        TACAW_LAUNCH_CHECK();
        if (jobs[j].n_t > 0) U += jobs[j].n_t;
    }
    int* ctl_all = cv.take<int>((size_t)(4 + 2 * U));
    WaitCtl wc{nullptr, wait_polls(kQueueWaitPolls)};
    int rc = timeout_flag(&wc.flag, "tacaw_multislice_queue");
    if (rc) return rc;
    std::vector<char> used(n_jobs, 0);
    for (int j0 = 0; j0 < n_jobs; ++j0) {
        if (used[j0] || jobs[j0].n_t <= 0 || jobs[j0].grid.n_slices <= 0) continue;
        const int n = jobs[j0].grid.nx;
        const int sp = queue_span(n, span);
        int tile_cols = 0, box_rows = 0;
        queue_tile_dims(n, &tile_cols, &box_rows);
        const int items = n / sp;
        int wv = wave;
        if (wv <= 0) {
            const double per = 8.0 * n * n;
            wv = (int)(kQueueWaveBytes / per);
            wv = wv < 1 ? 1 : wv;
        }
        int j = j0;
        while (j < n_jobs) {
            QJobs q;
            q.n = 0;
            q.wave = wv;
            q.span = sp;
            q.items = items;
            long long item = 0;
            int snaps = 0;
            for (; j < n_jobs && q.n < kQMaxJobs; ++j) {
                const tacaw_job& b = jobs[j];
                if (used[j] || b.n_t <= 0 || b.grid.n_slices <= 0 || b.grid.nx != n) continue;
                used[j] = 1;
                const int k = q.n++;
                q.item0[k] = item;
                q.snap0[k] = snaps;
                q.psi[k] = (float2*)b.psi_q;
                q.V[k] = b.V;
                q.psi_in[k] = (const float2*)b.psi_in;
                q.px[k] = tb[j].px;
                q.py[k] = tb[j].py;
                q.kymax[k] = tb[j].kymax;
                q.n_t[k] = b.n_t;
                q.n_slices[k] = b.grid.n_slices;
                q.sigma[k] = sigma[j];
                TACAW_REQUIRE(encode_wave_map(&q.cmap[k], b.psi_q, n, (long long)b.n_t * n, tile_cols, box_rows),
                              TACAW_ECUDA, "tacaw_multislice_queue: job %d: tensor map of the exit waves not encoded",
                              j);
                const long long job_items = (long long)b.grid.n_slices * 2 * items * b.n_t;
                TACAW_REQUIRE(job_items < (1LL << 31), TACAW_EINVAL,
                              "tacaw_multislice_queue: job %d has %lld queue items (at most 2^31 - 1)", j, job_items);
                item += job_items;
                snaps += b.n_t;
            }
            if (q.n == 0) break;
            q.item0[q.n] = item;
            q.snap0[q.n] = snaps;
            TACAW_CUDA_CHECK(cudaMemsetAsync(ctl_all, 0, (size_t)(4 + 2 * snaps) * sizeof(int), st));
            TACAW_CUDA_CHECK(dispatch_queue(n, q, tb[j0].twx, ctl_all, wc.flag, wc.polls, st));
        }
    }
    for (int j = 0; j < n_jobs; ++j) {
        if (!jobs[j].psi_sum || jobs[j].n_t <= 0) continue;
        const size_t nq = (size_t)jobs[j].grid.nx * jobs[j].grid.ny;
        snapshot_sum_kernel<<<(unsigned)((nq + 255) / 256), 256, 0, st>>>((const float2*)jobs[j].psi_q,
                                                                         (double2*)jobs[j].psi_sum,
                                                                         jobs[j].n_t, nq);
        TACAW_LAUNCH_CHECK();
    }
    return TACAW_OK;
}

// ------------------------------------------------------------------ adjoint
// Workspace of the adjoint: the set-up tables, a working wave set W (forward
// recompute), the gradient wave set G, n_ck checkpoints and `every` segment
// states, each [T][ny][nx] complex64.
struct MsBackWs {
    MsTables tb;
    float2 *w, *g, *ck, *seg;
};

static MsBackWs carve_ms_back(Carver& cv, const tacaw_grid& g, int n_t, int every) {
    MsBackWs b;
    b.tb = carve_ms(cv, g);
    const size_t wave = (size_t)n_t * g.nx * g.ny;
    const int n_ck = (g.n_slices + every - 1) / every;
    b.w = cv.take<float2>(wave);
    b.g = cv.take<float2>(wave);
    b.ck = cv.take<float2>(wave * n_ck);
    b.seg = cv.take<float2>(wave * every);
    return b;
}

size_t multislice_backward_ws_bytes(const tacaw_grid& g, int n_t, int every) {
    Carver cv(nullptr);
    carve_ms_back(cv, g, n_t, every);
    return cv.bytes();
}

// dL/dV [T][n_slices][ny][nx] from dL/d(exit wave) [T][ny][nx] with checkpoints
// every `every` slices: forward to the checkpoints, then for each segment (last
// first) recompute its states and run the adjoint slice steps in reverse.
int multislice_backward_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                            const float2* g_exit, float* dV, int every, void* ws, cudaStream_t st) {
    Carver cv(ws);
    MsBackWs b = carve_ms_back(cv, g, n_t, every);
    const MsTables& tb = b.tb;
    WaitCtl wc{nullptr, wait_polls(kRowWaitPolls)};
    int rc = timeout_flag(&wc.flag, "tacaw_multislice_backward");
    if (rc) return rc;
    double lam = 0.0, sig = 0.0;
    beam_constants(g.kev, &lam, &sig);
    const double qmax = g.bandlimit * fmin((double)g.nx / (2.0 * g.lx), (double)g.ny / (2.0 * g.ly));
    const int nmax = g.nx > g.ny ? g.nx : g.ny;
    ms_setup_kernel<<<(nmax + 127) / 128, 128, 0, st>>>(tb.twx, tb.twy, tb.px, tb.py, tb.kymax,
                                                       g.nx, g.ny, g.lx, g.ly, lam * g.dz, qmax * qmax);
    TACAW_LAUNCH_CHECK();
    const float sigma = (float)sig;
    const size_t wave = (size_t)n_t * g.nx * g.ny;
    const size_t wave_bytes = wave * sizeof(float2);
    const int first_mode = psi_in ? 2 : 1;
    const int n_ck = (g.n_slices + every - 1) / every;

    // forward to the checkpoints: ck[c] = state entering slice c * every (c >= 1)
    for (int s = 0; s + 1 < (n_ck - 1) * every + 1 && s < g.n_slices; ++s) {
        if (s > 0 && s % every == 0)
            TACAW_CUDA_CHECK(cudaMemcpyAsync(b.ck + (size_t)(s / every) * wave, b.w, wave_bytes,
                                             cudaMemcpyDeviceToDevice, st));
        TACAW_CUDA_CHECK(dispatch_row(g.nx, b.w, V, psi_in, tb.twx, tb.kymax, g.ny, n_t, g.n_slices, s, sigma,
                                      s > 0 ? 0 : first_mode, wc, st));
        TACAW_CUDA_CHECK(dispatch_col(g.ny, b.w, tb.twy, tb.px, tb.py, tb.kymax, g.nx, n_t, 0, st));
    }
    if (n_ck > 1 && (n_ck - 1) * every < g.n_slices)
        TACAW_CUDA_CHECK(cudaMemcpyAsync(b.ck + (size_t)(n_ck - 1) * wave, b.w, wave_bytes,
                                         cudaMemcpyDeviceToDevice, st));

    TACAW_CUDA_CHECK(cudaMemcpyAsync(b.g, g_exit, wave_bytes, cudaMemcpyDeviceToDevice, st));
    bool first = true;
    for (int c = n_ck - 1; c >= 0; --c) {
        const int s0 = c * every, s1 = min(s0 + every, g.n_slices);
        // recompute the states entering slices s0 .. s1-1 (seg[j] for slice s0 + j, j >= 1;
        // slice s0 reads its checkpoint, slice 0 the incident wave)
        if (s1 - s0 > 1) {
            if (c > 0)
                TACAW_CUDA_CHECK(cudaMemcpyAsync(b.w, b.ck + (size_t)c * wave, wave_bytes,
                                                 cudaMemcpyDeviceToDevice, st));
            for (int s = s0; s + 1 < s1; ++s) {
                TACAW_CUDA_CHECK(dispatch_row(g.nx, b.w, V, psi_in, tb.twx, tb.kymax, g.ny, n_t, g.n_slices, s,
                                              sigma, s > 0 ? 0 : first_mode, wc, st));
                TACAW_CUDA_CHECK(dispatch_col(g.ny, b.w, tb.twy, tb.px, tb.py, tb.kymax, g.nx, n_t, 0, st));
                TACAW_CUDA_CHECK(cudaMemcpyAsync(b.seg + (size_t)(s + 1 - s0) * wave, b.w, wave_bytes,
                                                 cudaMemcpyDeviceToDevice, st));
            }
        }
        for (int s = s1 - 1; s >= s0; --s) {
            TACAW_CUDA_CHECK(dispatch_col(g.ny, b.g, tb.twy, tb.px, tb.py, tb.kymax, g.nx, n_t, 0, st,
                                          first ? 2 : 1));
            first = false;
            const float2* state = (s == s0) ? (c > 0 ? b.ck + (size_t)c * wave : nullptr)
                                            : b.seg + (size_t)(s - s0) * wave;
            TACAW_CUDA_CHECK(dispatch_row_back(g.nx, b.g, state, V, dV, psi_in, tb.twx, tb.kymax, g.ny, n_t,
                                               g.n_slices, s, sigma, s > 0 ? 0 : first_mode, s > 0 ? 1 : 0,
                                               st));
        }
    }
    return TACAW_OK;
}

}  // namespace tacaw
