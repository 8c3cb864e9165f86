// Temporal transform on the 5th-generation tensor cores (tcgen05) in split
// BF16 with FP32 accumulation (Eq. (9): I(q, E) = |Phi(q, E)|^2 / T^2 with
// Phi = sum_n A(q, t_n) exp(-i E t_n / hbar), A = psi - time mean).
//
// The complex GEMM [nq x T] x [T x n_omega] is run as a real GEMM over
// K' = 2T: row q of A' is the centred series (re, im, re, im, ...), and the
// 256 columns of each N tile hold, for 128 energies, first the columns giving
// Re Phi (B'[2n] = Re e, B'[2n+1] = -Im e) and then those giving Im Phi
// (B'[2n] = Im e, B'[2n+1] = Re e), so the epilogue finds Re and Im of one
// energy TN/2 TMEM columns apart.  Every operand x is split into BF16 terms:
//  * BF16X3: x = x0 + x1, products x0 y0 + x0 y1 + x1 y0 (the x1 y1 term and
//    the split residual, ~2^-16 relative, are dropped), three-stage ring;
//  * BF16X6: x = x0 + x1 + x2, products x0 y0 + x0 y1 + x1 y0 + x0 y2 + x1 y1 +
//    x2 y0 (dropped terms ~2^-24 relative), two-stage ring.
// The tensor cores' FP32 accumulation into TMEM does not round to nearest: its
// error is a bias that grows with the number of MMAs into one accumulator and
// with the accumulator's size (measured: -4.8e-5 relative on I at T = 4096 when
// one accumulator took the whole K).  So the leading product x0 y0 and the
// small products go to separate accumulators that restart every CHUNK K blocks
// (two TMEM buffers, double-buffered), and four epilogue warps add each chunk
// into FP32 registers with round-to-nearest adds.
//
// Prologue kernels: the FP64 time mean and centring with the hi/lo split
// (written K-major, i.e. transposed from the time-major exit waves), and the
// split DFT matrix built in FP64.  Main kernel per 128 x 256 output tile:
// TMA (128-byte swizzle) into a 2- or 3-stage ring (warp 4), one thread of
// warp 5 issues the MMAs, tcgen05.commit frees ring stages and hands finished
// chunks to warps 0-3, which accumulate them and finally write |Phi|^2 / T^2
// (times the Kubo factor).  N tiles are 128 wide: 64 energies, Re then Im.

#include <string.h>

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

constexpr int TM = 128, TN = 128, TK = 64;     // tile; TK BF16 = 128 bytes per row
constexpr int A_BYTES = TM * TK * 2;
constexpr int B_BYTES_ = TN * TK * 2;
constexpr int EPI_WARPS = 4;                   // warps 0-3: TMEM lanes 0-127, the epilogue
constexpr int LOAD_WARP = 4, MMA_WARP = 5;
constexpr int TC_THREADS = 6 * 32;
constexpr int GROUP_N = 8;                     // N tiles sharing an L2 panel of B'
constexpr int CHUNK = 8;                       // K blocks summed in TMEM before the FP32 drain
constexpr uint32_t TMEM_COLS = 4 * TN;         // two buffers x (big, small) accumulators

template <int NT>                              // BF16 terms per operand: 2 or 3
struct TcCfg {
    static constexpr int STAGES = NT == 2 ? 3 : 2;
    static constexpr int B_BYTES = B_BYTES_;
    static constexpr int STAGE_BYTES = NT * (A_BYTES + B_BYTES);   // 64 or 96 KiB
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
};

// x -> BF16 terms t0 + t1 (+ t2); every residual is exact in FP32
__device__ __forceinline__ void split_bf16(float x, int nt, __nv_bfloat16* t) {
    t[0] = __float2bfloat16_rn(x);
    const float r1 = x - __bfloat162float(t[0]);
    t[1] = __float2bfloat16_rn(r1);
    if (nt == 3) t[2] = __float2bfloat16_rn(r1 - __bfloat162float(t[1]));
}

// A'_hi / A'_lo [nq_pad][2 t_pad]: (q, 2n) = Re(psi(q, t_n) - m_q), (q, 2n+1) = Im(...);
// the subtraction is done in FP64, zero padding beyond nq / T.  One block moves a
// 32 (time) x 32 (q) tile through shared memory; also writes I_el = |m_q|^2.
__global__ void __launch_bounds__(256)
split_a_kernel(const float2* __restrict__ psi, size_t ld, const double2* __restrict__ sum, int n_t,
               int nq, int t_pad, __nv_bfloat16* __restrict__ a0, __nv_bfloat16* __restrict__ a1,
               __nv_bfloat16* __restrict__ a2, double* __restrict__ i_el, const double2* __restrict__ mean = nullptr) {
    __shared__ float2 tile[32][33];
    const int q0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of 32
    const double inv_t = 1.0 / (double)n_t;
    {
        const int q = q0 + tx;
        double mr = 0.0, mi = 0.0;
        if (q < nq && mean) {                        // a given reference mean (time-chunked spectra)
            mr = mean[q].x;
            mi = mean[q].y;
        } else if (q < nq) {
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
        const int nt = a2 ? 3 : 2;
        __nv_bfloat16 re[3], im[3];
        split_bf16(a.x, nt, re);
        split_bf16(a.y, nt, im);
        __nv_bfloat16* dst[3] = {a0, a1, a2};
        for (int i = 0; i < nt; ++i) {
            __nv_bfloat162 v;
            v.x = re[i];
            v.y = im[i];
            reinterpret_cast<__nv_bfloat162*>(dst[i] + (size_t)q * k2)[t] = v;
        }
    }
}

// B' terms [n_tiles * tn][2 t_pad], see the file comment; e = exp(-i E_k t_n / hbar)
// computed in FP64 (exact integer phase on the natural grid), zero beyond n_w / T.
__global__ void __launch_bounds__(128)
split_b_kernel(const double* __restrict__ omega, int n_t, int n_w, int t_pad, double dt, int tn,
               __nv_bfloat16* __restrict__ b0, __nv_bfloat16* __restrict__ b1, __nv_bfloat16* __restrict__ b2,
               int t0 = 0) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;   // time index
    const int j = blockIdx.y;                              // B' row
    if (n >= t_pad) return;
    const int tile = j / tn, c = j % tn;
    const int k = tile * (tn / 2) + (c & (tn / 2 - 1));
    const bool imag_row = c >= tn / 2;
    float er = 0.f, ei = 0.f;
    if (k < n_w && n < n_t) {
        double s, co;
        if (omega == nullptr) {
            const long long kk = (long long)k - n_t / 2;
            long long r = (kk * n) % n_t;
            if (r < 0) r += n_t;
            sincospi(-2.0 * (double)r / (double)n_t, &s, &co);
        } else {
            const double cyc = omega[k] * ((double)(t0 + n) * dt) / kPlanckMeVfs;
            sincospi(-2.0 * (cyc - rint(cyc)), &s, &co);
        }
        er = (float)co;
        ei = (float)s;
    }
    const float x0 = imag_row ? ei : er;
    const float x1 = imag_row ? er : -ei;
    const int nt = b2 ? 3 : 2;
    __nv_bfloat16 s0[3], s1[3];
    split_bf16(x0, nt, s0);
    split_bf16(x1, nt, s1);
    __nv_bfloat16* dst[3] = {b0, b1, b2};
    const size_t k2 = 2 * (size_t)t_pad;
    for (int i = 0; i < nt; ++i) {
        __nv_bfloat162 v;
        v.x = s0[i];
        v.y = s1[i];
        reinterpret_cast<__nv_bfloat162*>(dst[i] + (size_t)j * k2)[n] = v;
    }
}

// Operand tensor maps of one launch: A' and B' terms 0 .. NT-1.
struct TcMaps {
    CUtensorMap a[3], b[3];
};

template <int NT>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_power_kernel(const __grid_constant__ TcMaps maps, const float* __restrict__ kubo, float* __restrict__ out,
                int nq, int n_w, int n_kblocks, int n_mtiles, int n_ntiles, float scale, int* __restrict__ err,
                int* __restrict__ status, float2* __restrict__ phi_acc) {
    using Cfg = TcCfg<NT>;
    constexpr int STAGES = Cfg::STAGES;
    constexpr int B_BYTES = Cfg::B_BYTES;
    constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;     // [2]: a chunk's partial sums are complete in TMEM
    uint64_t* acc_empty = acc_full + 2;      // [2]: the epilogue warps have read them
    uint64_t* done = acc_empty + 2;          // every MMA of the block has completed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    int* consumed = reinterpret_cast<int*>(tmem_slot + 1);

    // tile order: groups of GROUP_N N tiles; inside a group, N fastest, then M
    const int b = blockIdx.x;
    const int gfull = GROUP_N * n_mtiles;
    const int g = b / gfull, rem = b % gfull;
    const int gw = min(GROUP_N, n_ntiles - g * GROUP_N);
    const int mt = rem / gw, nt = g * GROUP_N + rem % gw;
    const int n_chunks = (n_kblocks + CHUNK - 1) / CHUNK;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], EPI_WARPS);
        }
        tc::mbar_init(done, 1);
        *consumed = 0;
        tc::fence_mbar_init();
    }
    if (warp == MMA_WARP) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    int issued = 0;
    if (warp == LOAD_WARP && lane == 0) {
        // producer: TMA loads of the operand terms of each K block
        for (int kb = 0; kb < n_kblocks; ++kb) {
            const int s = kb % STAGES, u = kb / STAGES;
            if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, err)) break;
            uint8_t* st = base + s * STAGE_BYTES;
            tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                tc::tma_load_2d(st + i * A_BYTES, &maps.a[i], &full[s], kb * TK, mt * TM);
                tc::tma_load_2d(st + NT * A_BYTES + i * B_BYTES, &maps.b[i], &full[s], kb * TK, nt * TN);
            }
            issued = kb + 1;
        }
    } else if (warp == MMA_WARP && lane == 0) {
        // MMA issuer.  Chunk c (CHUNK K blocks) accumulates into TMEM buffer c & 1:
        // the leading product x0 y0 into its "big" half, every other product into
        // its "small" half, both starting from zero.
        constexpr uint32_t idesc = tc::idesc_bf16_f32(TM, TN);
        int kb = 0;
        bool ok = true;
        for (; kb < n_kblocks && ok; ++kb) {
            const int c = kb / CHUNK, buf = c & 1;
            const bool kfirst = (kb % CHUNK) == 0;
            if (kfirst && c >= 2 && !tc::mbar_wait(&acc_empty[buf], ((c >> 1) - 1) & 1, err)) break;
            const int s = kb % STAGES, u = kb / STAGES;
            if (!tc::mbar_wait(&full[s], u & 1, err)) break;
            tc::fence_after_sync();
            const uint32_t big = tmem + buf * 2 * TN, small = big + TN;
            const uint32_t sa = tc::smem_u32(base + s * STAGE_BYTES);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const uint32_t off = kk * 32;   // 16 BF16 along K inside the swizzled row
                uint64_t da[NT], db[NT];
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    da[i] = tc::desc_kmajor_sw128(sa + i * A_BYTES + off);
                    db[i] = tc::desc_kmajor_sw128(sa + NT * A_BYTES + i * B_BYTES + off);
                }
                const uint32_t acc = (kfirst && kk == 0) ? 0u : 1u;
                tc::mma_bf16(big, da[0], db[0], idesc, acc);
                tc::mma_bf16(small, da[0], db[1], idesc, acc);
                tc::mma_bf16(small, da[1], db[0], idesc, 1u);
                if constexpr (NT == 3) {
                    tc::mma_bf16(small, da[0], db[2], idesc, 1u);
                    tc::mma_bf16(small, da[1], db[1], idesc, 1u);
                    tc::mma_bf16(small, da[2], db[0], idesc, 1u);
                }
            }
            tc::mma_commit(&empty[s]);
            if ((kb % CHUNK) == CHUNK - 1 || kb == n_kblocks - 1) tc::mma_commit(&acc_full[buf]);
        }
        *consumed = kb;
        tc::mma_commit(done);
    } else if (warp < EPI_WARPS) {
        // epilogue warps: warp w owns TMEM lanes 32w .. 32w + 31 (rows of the tile) and
        // adds each chunk's partial sums into FP32 registers with round-to-nearest
        float acc[TN];
#pragma unroll
        for (int i = 0; i < TN; ++i) acc[i] = 0.f;
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        bool ok = true;
        for (int c = 0; c < n_chunks; ++c) {
            const int buf = c & 1;
            if (!tc::mbar_wait(&acc_full[buf], (c >> 1) & 1, err)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int c0 = 0; c0 < TN; c0 += 32) {
                float vb[32], vs[32];
                tc::tmem_ld_32cols(lane_addr + buf * 2 * TN + c0, vb);
                tc::tmem_ld_32cols(lane_addr + buf * 2 * TN + TN + c0, vs);
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[c0 + i] = __fadd_rn(__fadd_rn(acc[c0 + i], vb[i]), vs[i]);
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&acc_empty[buf]);
        }
        if (ok && !*(volatile int*)err && phi_acc) {   // time-chunked: add Phi itself
            const int row = mt * TM + warp * 32 + lane;
            if (row < nq) {
                float2* prow = phi_acc + (size_t)row * n_w;
#pragma unroll
                for (int i = 0; i < TN / 2; ++i) {
                    const int k = nt * (TN / 2) + i;
                    if (k < n_w) {
                        const float2 old = prow[k];
                        prow[k] = make_float2(old.x + acc[i], old.y + acc[TN / 2 + i]);
                    }
                }
            }
        } else if (ok && !*(volatile int*)err) {
            const int row = mt * TM + warp * 32 + lane;
            if (row < nq) {
                float* orow = out + (size_t)row * n_w;
#pragma unroll
                for (int i = 0; i < TN / 2; ++i) {
                    const int k = nt * (TN / 2) + i;
                    if (k < n_w) {
                        float v = (acc[i] * acc[i] + acc[TN / 2 + i] * acc[TN / 2 + i]) * scale;
                        if (kubo) v *= __ldg(kubo + k);
                        orow[k] = v;
                    }
                }
            }
        }
    }
    __syncwarp();
    // Before TMEM is freed: every MMA has completed (bounded wait), and after a
    // timeout the loads that were issued but never consumed have landed.
    __syncthreads();
    if (warp == LOAD_WARP && lane == 0) {
        tc::mbar_wait_quiet(done, 0, 1u << 22);
        if (*(volatile int*)err)
            for (int kb = *consumed; kb < issued; ++kb)
                tc::mbar_wait_quiet(&full[kb % STAGES], (kb / STAGES) & 1, 1u << 20);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == MMA_WARP) tc::tmem_dealloc(tmem, TMEM_COLS);
    // a role gave up: the launch's flag coordinated the roles; the sticky
    // status flag reports it to the host (tacaw_status)
    if (threadIdx.x == 0 && *(volatile int*)err) atomicExch(status, 1);
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
    int nt, tn, t_pad, nq_pad, n_mtiles, n_ntiles, n_kblocks;
    size_t k2;
};

TcGeom geom(int nq, int n_t, int n_w, int nt) {
    TcGeom g;
    g.nt = nt;
    g.tn = TN;
    g.t_pad = (n_t + TK / 2 - 1) / (TK / 2) * (TK / 2);     // 2 t_pad multiple of TK
    g.nq_pad = (nq + TM - 1) / TM * TM;
    g.n_mtiles = g.nq_pad / TM;
    g.n_ntiles = (n_w + g.tn / 2 - 1) / (g.tn / 2);
    g.k2 = 2 * (size_t)g.t_pad;
    g.n_kblocks = (int)(g.k2 / TK);
    return g;
}

struct TcWs {
    double2* sum;
    __nv_bfloat16 *a[3], *b[3];
    float* kubo;
    double* red;
    double* i_el;
    int* err;
};

TcWs carve_tc(Carver& cv, int nq, int n_t, int n_w, bool need_sum, bool need_iel, int nt) {
    const TcGeom g = geom(nq, n_t, n_w, nt);
    TcWs w;
    w.sum = need_sum ? cv.take<double2>(nq) : nullptr;
    for (int i = 0; i < 3; ++i) {
        w.a[i] = i < nt ? cv.take<__nv_bfloat16>((size_t)g.nq_pad * g.k2, 1024) : nullptr;
        w.b[i] = i < nt ? cv.take<__nv_bfloat16>((size_t)g.n_ntiles * g.tn * g.k2, 1024) : nullptr;
    }
    w.kubo = cv.take<float>(n_w);
    w.red = cv.take<double>(normalize_ws_doubles());
    w.i_el = need_iel ? cv.take<double>(nq) : nullptr;
    w.err = cv.take<int>(1);
    return w;
}

}  // namespace

size_t spectrum_tc_ws_bytes(int nq, int n_t, int n_w, bool have_sum, bool have_iel, int terms) {
    Carver cv(nullptr);
    carve_tc(cv, nq, n_t, n_w, !have_sum, !have_iel, terms);
    return cv.bytes();
}

// terms = 2 (BF16X3) or 3 (BF16X6)
int spectrum_tc_run(int nq, int n_t, double dt_fs, int n_w, const double* omega, const float2* psi,
                    size_t ld, const double2* psi_sum, float* out, double* i_el, int flags,
                    double beta, int terms, void* ws, cudaStream_t st) {
    Carver cv(ws);
    TcWs w = carve_tc(cv, nq, n_t, n_w, psi_sum == nullptr, i_el == nullptr, terms);
    const TcGeom g = geom(nq, n_t, n_w, terms);
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
        split_a_kernel<<<grid, 256, 0, st>>>(psi, ld, sum, n_t, nq, g.t_pad, w.a[0], w.a[1], w.a[2], iel);
        TACAW_LAUNCH_CHECK();
    }
    {
        dim3 grid((g.t_pad + 127) / 128, g.n_ntiles * g.tn);
        split_b_kernel<<<grid, 128, 0, st>>>(omega, n_t, n_w, g.t_pad, dt_fs, g.tn, w.b[0], w.b[1], w.b[2]);
        TACAW_LAUNCH_CHECK();
    }
    const bool kubo = (flags & TACAW_KUBO) != 0;
    if (kubo) {
        int rc = launch_kubo(w.kubo, omega, n_t, n_w, dt_fs, beta, st);
        if (rc) return rc;
    }
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    int rc = TACAW_OK;
    for (int i = 0; i < terms && !rc; ++i) {
        rc = make_map(&maps.a[i], w.a[i], g.nq_pad, g.k2, TM);
        if (!rc) rc = make_map(&maps.b[i], w.b[i], (size_t)g.n_ntiles * g.tn, g.k2, g.tn);
    }
    if (rc) return rc;
    const float scale = (float)(1.0 / ((double)n_t * (double)n_t));
    const unsigned blocks = (unsigned)(g.n_mtiles * g.n_ntiles);
    int* status = nullptr;
    rc = timeout_flag(&status, "tacaw_spectrum");
    if (rc) return rc;
    if (terms == 2) {
        TACAW_CUDA_CHECK(ensure_smem((const void*)tc_power_kernel<2>, (int)TcCfg<2>::SMEM));
        tc_power_kernel<2><<<blocks, TC_THREADS, TcCfg<2>::SMEM, st>>>(maps, kubo ? w.kubo : nullptr, out, nq, n_w,
                                                                      g.n_kblocks, g.n_mtiles, g.n_ntiles, scale,
                                                                      w.err, status, nullptr);
    } else {
        TACAW_CUDA_CHECK(ensure_smem((const void*)tc_power_kernel<3>, (int)TcCfg<3>::SMEM));
        tc_power_kernel<3><<<blocks, TC_THREADS, TcCfg<3>::SMEM, st>>>(maps, kubo ? w.kubo : nullptr, out, nq, n_w,
                                                                      g.n_kblocks, g.n_mtiles, g.n_ntiles, scale,
                                                                      w.err, status, nullptr);
    }
    TACAW_LAUNCH_CHECK();
    if (flags & TACAW_NORMALIZE) {
        rc = launch_normalize(out, (size_t)nq * n_w, i_el, iel, nq, w.red, w.red + normalize_ws_doubles() - 1, st);
        if (rc) return rc;
    }
    return TACAW_OK;
}

// ------------------------------------------------------------------ time-chunked spectra
// phi[q][k] += sum_{j < n_chunk} (psi[j][q] - m_ref[q]) exp(-i E_k (t0 + j) dt / hbar),
// the same split-BF16 GEMM with the FP32 drains, Phi added in the epilogue.
size_t spectrum_tc_accumulate_ws_bytes(int nq, int n_t, int n_w, int terms) {
    Carver cv(nullptr);
    carve_tc(cv, nq, n_t, n_w, false, false, terms);
    return cv.bytes();
}

int spectrum_tc_accumulate_run(int nq, int t0, int n_chunk, double dt_fs, int n_w, const double* omega,
                               const float2* psi, size_t ld, const double2* m_ref, float2* phi, int terms,
                               void* ws, cudaStream_t st) {
    Carver cv(ws);
    TcWs w = carve_tc(cv, nq, n_chunk, n_w, false, false, terms);
    const TcGeom g = geom(nq, n_chunk, n_w, terms);
    TACAW_REQUIRE((size_t)g.n_mtiles * g.n_ntiles <= 0x7fffffffu, TACAW_EUNSUPPORTED,
                  "tacaw_spectrum_accumulate: too many output tiles");
    TACAW_CUDA_CHECK(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    split_a_kernel<<<dim3(g.nq_pad / 32, g.t_pad / 32), 256, 0, st>>>(psi, ld, nullptr, n_chunk, nq, g.t_pad, w.a[0],
                                                                      w.a[1], w.a[2], nullptr, m_ref);
    TACAW_LAUNCH_CHECK();
    split_b_kernel<<<dim3((g.t_pad + 127) / 128, g.n_ntiles * g.tn), 128, 0, st>>>(omega, n_chunk, n_w, g.t_pad, dt_fs,
                                                                                 g.tn, w.b[0], w.b[1], w.b[2], t0);
    TACAW_LAUNCH_CHECK();
    TcMaps maps;
    memset(&maps, 0, sizeof(maps));
    int rc = TACAW_OK;
    for (int i = 0; i < terms && !rc; ++i) {
        rc = make_map(&maps.a[i], w.a[i], g.nq_pad, g.k2, TM);
        if (!rc) rc = make_map(&maps.b[i], w.b[i], (size_t)g.n_ntiles * g.tn, g.k2, g.tn);
    }
    if (rc) return rc;
    int* status = nullptr;
    rc = timeout_flag(&status, "tacaw_spectrum_accumulate");
    if (rc) return rc;
    const unsigned blocks = (unsigned)(g.n_mtiles * g.n_ntiles);
    if (terms == 2) {
        TACAW_CUDA_CHECK(ensure_smem((const void*)tc_power_kernel<2>, (int)TcCfg<2>::SMEM));
        tc_power_kernel<2><<<blocks, TC_THREADS, TcCfg<2>::SMEM, st>>>(maps, nullptr, nullptr, nq, n_w, g.n_kblocks,
                                                                      g.n_mtiles, g.n_ntiles, 1.f, w.err, status, phi);
    } else {
        TACAW_CUDA_CHECK(ensure_smem((const void*)tc_power_kernel<3>, (int)TcCfg<3>::SMEM));
        tc_power_kernel<3><<<blocks, TC_THREADS, TcCfg<3>::SMEM, st>>>(maps, nullptr, nullptr, nq, n_w, g.n_kblocks,
                                                                      g.n_mtiles, g.n_ntiles, 1.f, w.err, status, phi);
    }
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace tacaw
