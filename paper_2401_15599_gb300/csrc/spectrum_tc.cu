// Temporal transform on the 5th-generation tensor cores (tcgen05) in split
// BF16 with FP32 accumulation (Eq. (9): I(q, E) = |Phi(q, E)|^2 / T^2 with
// Phi = sum_n A(q, t_n) exp(-i E t_n / hbar), A = psi - time mean).
//
// The complex GEMM [nq x T] x [T x n_omega] is run as a real GEMM over
// K' = 2T: row q of A' is the centred series (re, im, re, im, ...), and the
// 256 columns of each N tile hold, for 128 energies, first the columns giving
// Re Phi (B'[2n] = Re e, B'[2n+1] = -Im e) and then those giving Im Phi
// (B'[2n] = Im e, B'[2n+1] = Re e), so the epilogue finds Re and Im of one
// energy 128 TMEM columns apart.  Every operand x is split as
// x = hi + lo (both BF16) and three products hi*hi + hi*lo + lo*hi are
// accumulated in FP32 (the lo*lo term, ~2^-16 relative, is dropped).
//
// Prologue kernels: the FP64 time mean and centring with the hi/lo split
// (written K-major, i.e. transposed from the time-major exit waves), and the
// split DFT matrix built in FP64.  Main kernel per 128 x 256 output tile:
// TMA (128-byte swizzle) into a 2-stage ring, one thread issues the MMAs,
// tcgen05.commit frees ring stages, four warps read the accumulator from
// TMEM and write |Phi|^2 / T^2 (times the Kubo factor).

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace tacaw {

// from spectrum.cu
int launch_time_sum(const float2* psi, size_t ld, double2* sum, int n_t, int nq, cudaStream_t st);
int launch_kubo(float* kubo, const double* omega, int n_t, int n_w, double dt, double beta,
                cudaStream_t st);
int launch_normalize(float* out, size_t n, double* i_el_user, const double* i_el, int nq,
                     double* partial, double* total, cudaStream_t st);
size_t normalize_ws_doubles();

namespace {

constexpr int TM = 128, TN = 256, TK = 64;     // tile; TK BF16 = 128 bytes per row
constexpr int STAGES = 2;
constexpr int A_BYTES = TM * TK * 2;
constexpr int B_BYTES = TN * TK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // 96 KiB
constexpr int TC_THREADS = 128;
constexpr int GROUP_N = 8;                               // N tiles sharing an L2 panel of B'
constexpr size_t TC_SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;

// CODATA 2018 Planck constant in meV*fs.

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// A'_hi / A'_lo [nq_pad][2 t_pad]: (q, 2n) = Re(psi(q, t_n) - m_q), (q, 2n+1) = Im(...);
// the subtraction is done in FP64, zero padding beyond nq / T.  One block moves a
// 32 (time) x 32 (q) tile through shared memory; also writes I_el = |m_q|^2.
__global__ void __launch_bounds__(256)
split_a_kernel(const float2* __restrict__ psi, size_t ld, const double2* __restrict__ sum, int n_t,
               int nq, int t_pad, __nv_bfloat16* __restrict__ ahi, __nv_bfloat16* __restrict__ alo,
               double* __restrict__ i_el) {
    __shared__ float2 tile[32][33];
    const int q0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
    const double inv_t = 1.0 / (double)n_t;
    {
        const int q = q0 + tx;
        double mr = 0.0, mi = 0.0;
        if (q < nq) {
            const double2 s = sum[q];
            mr = s.x * inv_t;
            mi = s.y * inv_t;
            if (blockIdx.y == 0 && ty == 0 && i_el) i_el[q] = mr * mr + mi * mi;
        }
        for (int r = ty; r < 32; r += 8) {
            const int t = t0 + r;
            float2 a = make_float2(0.f, 0.f);
            if (q < nq && t < n_t) {
                const float2 v = __ldg(psi + (size_t)t * ld + q);
                a = make_float2((float)((double)v.x - mr), (float)((double)v.y - mi));
            }
            tile[r][tx] = a;
        }
    }
    __syncthreads();
    const size_t k2 = 2 * (size_t)t_pad;
    for (int r = ty; r < 32; r += 8) {               // r: q within the tile, tx: time
        const int q = q0 + r, t = t0 + tx;
        const float2 a = tile[tx][r];
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(a.x, h0, l0);
        split_bf16(a.y, h1, l1);
        __nv_bfloat162 hh, ll;
        hh.x = h0; hh.y = h1;
        ll.x = l0; ll.y = l1;
        reinterpret_cast<__nv_bfloat162*>(ahi + (size_t)q * k2)[t] = hh;
        reinterpret_cast<__nv_bfloat162*>(alo + (size_t)q * k2)[t] = ll;
    }
}

// B'_hi / B'_lo [n_tiles * 256][2 t_pad], see the file comment; e = exp(-i E_k t_n / hbar)
// computed in FP64 (exact integer phase on the natural grid), zero beyond n_w / T.
__global__ void __launch_bounds__(128)
split_b_kernel(const double* __restrict__ omega, int n_t, int n_w, int t_pad, double dt,
               __nv_bfloat16* __restrict__ bhi, __nv_bfloat16* __restrict__ blo) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;   // time index
    const int j = blockIdx.y;                              // B' row
    if (n >= t_pad) return;
    const int tile = j / TN, c = j % TN;
    const int k = tile * (TN / 2) + (c & (TN / 2 - 1));
    const bool imag_row = c >= TN / 2;
    float er = 0.f, ei = 0.f;
    if (k < n_w && n < n_t) {
        double s, co;
        if (omega == nullptr) {
            const long long kk = (long long)k - n_t / 2;
            long long r = (kk * n) % n_t;
            if (r < 0) r += n_t;
            sincospi(-2.0 * (double)r / (double)n_t, &s, &co);
        } else {
            const double cyc = omega[k] * ((double)n * dt) / kPlanckMeVfs;
            sincospi(-2.0 * (cyc - rint(cyc)), &s, &co);
        }
        er = (float)co;
        ei = (float)s;
    }
    const float x0 = imag_row ? ei : er;
    const float x1 = imag_row ? er : -ei;
    __nv_bfloat16 h0, l0, h1, l1;
    split_bf16(x0, h0, l0);
    split_bf16(x1, h1, l1);
    __nv_bfloat162 hh, ll;
    hh.x = h0; hh.y = h1;
    ll.x = l0; ll.y = l1;
    const size_t k2 = 2 * (size_t)t_pad;
    reinterpret_cast<__nv_bfloat162*>(bhi + (size_t)j * k2)[n] = hh;
    reinterpret_cast<__nv_bfloat162*>(blo + (size_t)j * k2)[n] = ll;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
tc_power_kernel(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
                const __grid_constant__ CUtensorMap map_bhi, const __grid_constant__ CUtensorMap map_blo,
                const float* __restrict__ kubo, float* __restrict__ out, int nq, int n_w,
                int n_kblocks, int n_mtiles, int n_ntiles, float scale, int* __restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    int* consumed = reinterpret_cast<int*>(tmem_slot + 1);

    // tile order: groups of GROUP_N N tiles; inside a group, N fastest, then M
    const int b = blockIdx.x;
    const int gfull = GROUP_N * n_mtiles;
    const int g = b / gfull, rem = b % gfull;
    const int gw = min(GROUP_N, n_ntiles - g * GROUP_N);
    const int mt = rem / gw, nt = g * GROUP_N + rem % gw;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(accum, 1);
        *consumed = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TN);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == 0 && lane == 0) {
        // producer: TMA loads of the four operand tiles of each K block
        for (int kb = 0; kb < n_kblocks; ++kb) {
            const int s = kb % STAGES, u = kb / STAGES;
            if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, err)) break;
            uint8_t* st = base + s * STAGE_BYTES;
            tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
            tc::tma_load_2d(st, &map_ahi, &full[s], kb * TK, mt * TM);
            tc::tma_load_2d(st + A_BYTES, &map_alo, &full[s], kb * TK, mt * TM);
            tc::tma_load_2d(st + 2 * A_BYTES, &map_bhi, &full[s], kb * TK, nt * TN);
            tc::tma_load_2d(st + 2 * A_BYTES + B_BYTES, &map_blo, &full[s], kb * TK, nt * TN);
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16_f32(TM, TN);
        int kb = 0;
        for (; kb < n_kblocks; ++kb) {
            const int s = kb % STAGES, u = kb / STAGES;
            if (!tc::mbar_wait(&full[s], u & 1, err)) break;
            tc::fence_after_sync();
            const uint32_t sa = tc::smem_u32(base + s * STAGE_BYTES);
            const uint32_t ahi = sa, alo = sa + A_BYTES, bhi = sa + 2 * A_BYTES,
                           blo = sa + 2 * A_BYTES + B_BYTES;
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const uint32_t off = kk * 32;   // 16 BF16 along K inside the swizzled row
                const uint64_t dah = tc::desc_kmajor_sw128(ahi + off);
                const uint64_t dal = tc::desc_kmajor_sw128(alo + off);
                const uint64_t dbh = tc::desc_kmajor_sw128(bhi + off);
                const uint64_t dbl = tc::desc_kmajor_sw128(blo + off);
                tc::mma_bf16(tmem, dah, dbh, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                tc::mma_bf16(tmem, dah, dbl, idesc, 1u);
                tc::mma_bf16(tmem, dal, dbh, idesc, 1u);
            }
            tc::mma_commit(&empty[s]);
        }
        *consumed = kb;
        tc::mma_commit(accum);
    }
    __syncwarp();

    // epilogue: warp w owns TMEM lanes 32w .. 32w + 31 (rows of the tile)
    const bool ok = tc::mbar_wait(accum, 0, err);
    tc::fence_after_sync();
    if (ok && !*(volatile int*)err) {
        const int row = mt * TM + warp * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        float* orow = out + (size_t)row * n_w;
#pragma unroll 1
        for (int c0 = 0; c0 < TN / 2; c0 += 32) {
            float re[32], im[32];
            tc::tmem_ld_32cols(lane_addr + c0, re);
            tc::tmem_ld_32cols(lane_addr + TN / 2 + c0, im);
            if (row < nq) {
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const int k = nt * (TN / 2) + c0 + i;
                    if (k < n_w) {
                        float v = (re[i] * re[i] + im[i] * im[i]) * scale;
                        if (kubo) v *= __ldg(kubo + k);
                        orow[k] = v;
                    }
                }
            }
        }
    }
    // On a timeout, wait (bounded) for loads that were issued but never consumed
    // so no TMA write lands after the block has exited.
    __syncthreads();
    if (warp == 0 && lane == 0 && *(volatile int*)err) {
        for (int kb = *consumed; kb < issued; ++kb)
            tc::mbar_wait_quiet(&full[kb % STAGES], (kb / STAGES) & 1, 1u << 20);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 1) tc::tmem_dealloc(tmem, TN);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D BF16 tensor [rows][k2] (k2 contiguous), box 64 x box_rows, 128-byte swizzle.
int make_map(CUtensorMap* map, const void* ptr, size_t rows, size_t k2, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    TACAW_REQUIRE(fn != nullptr, TACAW_ECUDA, "tacaw_spectrum: cuTensorMapEncodeTiled unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)k2, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(k2 * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
                    estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    TACAW_REQUIRE(r == CUDA_SUCCESS, TACAW_ECUDA, "tacaw_spectrum: tensor map encoding failed (%d)", (int)r);
    return TACAW_OK;
}

struct TcGeom {
    int t_pad, nq_pad, n_mtiles, n_ntiles, n_kblocks;
    size_t k2;
};

TcGeom geom(int nq, int n_t, int n_w) {
    TcGeom g;
    g.t_pad = (n_t + TK / 2 - 1) / (TK / 2) * (TK / 2);     // 2 t_pad multiple of TK
    g.nq_pad = (nq + TM - 1) / TM * TM;
    g.n_mtiles = g.nq_pad / TM;
    g.n_ntiles = (n_w + TN / 2 - 1) / (TN / 2);
    g.k2 = 2 * (size_t)g.t_pad;
    g.n_kblocks = (int)(g.k2 / TK);
    return g;
}

struct TcWs {
    double2* sum;
    __nv_bfloat16 *ahi, *alo, *bhi, *blo;
    float* kubo;
    double* red;
    double* i_el;
    int* err;
};

TcWs carve_tc(Carver& cv, int nq, int n_t, int n_w, bool need_sum, bool need_iel) {
    const TcGeom g = geom(nq, n_t, n_w);
    TcWs w;
    w.sum = need_sum ? cv.take<double2>(nq) : nullptr;
    w.ahi = cv.take<__nv_bfloat16>((size_t)g.nq_pad * g.k2, 1024);
    w.alo = cv.take<__nv_bfloat16>((size_t)g.nq_pad * g.k2, 1024);
    w.bhi = cv.take<__nv_bfloat16>((size_t)g.n_ntiles * TN * g.k2, 1024);
    w.blo = cv.take<__nv_bfloat16>((size_t)g.n_ntiles * TN * g.k2, 1024);
    w.kubo = cv.take<float>(n_w);
    w.red = cv.take<double>(normalize_ws_doubles());
    w.i_el = need_iel ? cv.take<double>(nq) : nullptr;
    w.err = cv.take<int>(1);
    return w;
}

}  // namespace

size_t spectrum_tc_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel) {
    Carver cv(nullptr);
    carve_tc(cv, nq, n_t, n_w, !have_sum, !have_iel);
    return cv.bytes();
}

int spectrum_tc_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                    size_t ld, const double2* psi_sum, float* out, double* i_el, int flags,
                    double beta, void* ws, cudaStream_t st) {
    Carver cv(ws);
    TcWs w = carve_tc(cv, nq, n_t, n_w, psi_sum == nullptr, i_el == nullptr);
    const TcGeom g = geom(nq, n_t, n_w);
    TACAW_REQUIRE((size_t)g.n_mtiles * g.n_ntiles <= 0x7fffffffu, TACAW_EUNSUPPORTED,
                  "tacaw_spectrum: too many output tiles");
    const double2* sum = psi_sum;
    if (!sum) {
        int rc = launch_time_sum(psi, ld, w.sum, n_t, nq, st);
        if (rc) return rc;
        sum = w.sum;
    }
    double* iel = i_el ? i_el : w.i_el;
    TACAW_CUDA_CHECK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    {
        dim3 grid(g.nq_pad / 32, g.t_pad / 32);
        split_a_kernel<<<grid, 256, 0, st>>>(psi, ld, sum, n_t, nq, g.t_pad, w.ahi, w.alo, iel);
        TACAW_LAUNCH_CHECK();
    }
    {
        dim3 grid((g.t_pad + 127) / 128, g.n_ntiles * TN);
        split_b_kernel<<<grid, 128, 0, st>>>(omega, n_t, n_w, g.t_pad, dt_fs, w.bhi, w.blo);
        TACAW_LAUNCH_CHECK();
    }
    const bool kubo = (flags & TACAW_KUBO) != 0;
    if (kubo) {
        int rc = launch_kubo(w.kubo, omega, n_t, n_w, dt_fs, beta, st);
        if (rc) return rc;
    }
    CUtensorMap mah, mal, mbh, mbl;
    int rc = make_map(&mah, w.ahi, g.nq_pad, g.k2, TM);
    if (!rc) rc = make_map(&mal, w.alo, g.nq_pad, g.k2, TM);
    if (!rc) rc = make_map(&mbh, w.bhi, (size_t)g.n_ntiles * TN, g.k2, TN);
    if (!rc) rc = make_map(&mbl, w.blo, (size_t)g.n_ntiles * TN, g.k2, TN);
    if (rc) return rc;
    TACAW_CUDA_CHECK(ensure_smem((const void*)tc_power_kernel, (int)TC_SMEM));
    const float scale = (float)(1.0 / ((double)n_t * (double)n_t));
    const unsigned blocks = (unsigned)(g.n_mtiles * g.n_ntiles);
    tc_power_kernel<<<blocks, TC_THREADS, TC_SMEM, st>>>(mah, mal, mbh, mbl, kubo ? w.kubo : nullptr, out, nq,
                                                         n_w, g.n_kblocks, g.n_mtiles, g.n_ntiles, scale,
                                                         w.err);
    TACAW_LAUNCH_CHECK();
    if (flags & TACAW_NORMALIZE) {
        rc = launch_normalize(out, (size_t)nq * n_w, i_el, iel, nq, w.red, w.red + normalize_ws_doubles() - 1, st);
        if (rc) return rc;
    }
    return TACAW_OK;
}

}  // namespace tacaw
