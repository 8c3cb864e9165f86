// Slice-potential builder: Gaussian atoms projected onto the grid and split
// over slices (the scattering potential of a configuration that the
// multislice step of the paper's procedure propagates through).
//
//   v_s(r) = sum_a amp_a exp(-|r - R_a|^2 / (2 s_a^2)) w_s(z_a)
//   w_s(z) = (erf((z_{s+1} - z)/(sqrt2 s)) - erf((z_s - z)/(sqrt2 s))) / 2
//
// Laterally the Gaussian is cut to the square |dx|, |dy| <= 6 s (minimum
// periodic image), which keeps it separable in x and y;
// slices that do not meet [z - 6 s, z + 6 s] get weight 0; the first slice
// extends to -inf and the last to +inf.
//
// Two kernels per call:
//  1. bin_kernel (one block per snapshot): counting sort of the atoms into
//     bins (slab of the atom centre) x (band of kBandRows grid rows).
//  2. potential_kernel (one block per band, slice and snapshot): the block
//     owns kBandRows x nx pixels in shared memory and adds the contributions
//     of the atoms of the neighbouring bins.  Sums are kept in 64-bit fixed
//     point (2^-32 V*A), so the result does not depend on the order in which
//     atoms arrive: identical configurations give bit-identical potentials.

#include <math.h>

#include "common.cuh"

namespace tacaw {

namespace {

constexpr int kBandRows = 8;
constexpr int kBinThreads = 1024;
constexpr int kPotThreads = 256;
// Fixed point: each contribution is rounded to a multiple of 2^-20 V*A as a
// 32-bit integer (so one contribution must stay below 2048 V*A; the host
// checks the amplitudes) and summed exactly into a 64-bit accumulator.
// 64-bit float<->int conversions are avoided on purpose: on this GPU they
// run on the FP64 pipe.
constexpr float kFixScale = 1048576.0f;              // 2^20
constexpr float kFixInv = 9.5367431640625e-07f;      // 2^-20
constexpr float kMaxAmp = 2000.0f;

struct PotParams {
    int nx, ny, n_slices, n_atoms, n_species;
    int n_bands, n_bins, slab_reach, band_reach;
    float lx, ly, dx, dy, inv_dx, inv_lx, inv_ly, z0, dz, inv_dz, inv_band_h;
    double dx_d, dy_d, inv_dx_d, inv_dy_d;
    float amp[TACAW_MAX_SPECIES], sigma[TACAW_MAX_SPECIES];
};

// An atom's position is split once, in FP64, into the pixel (ic, jc) that
// holds it and a small offset (fx, fy) from that pixel, so that later
// pixel-atom distances k*d - f carry no rounding from large coordinates.
// Its band is the exact integer row band of jc; its slab comes from z with
// explicit round-to-nearest operations (the bin is computed twice per atom,
// count then scatter, and both passes must agree).
struct Split {
    int ic, jc;
    float fx, fy;
    bool ok;
};

__device__ __forceinline__ Split split_position(float x, float y, const PotParams& p) {
    Split r;
    const double fxd = (double)x * p.inv_dx_d, fyd = (double)y * p.inv_dy_d;
    r.ok = fabs(fxd) < 1e9 && fabs(fyd) < 1e9;
    const double icd = r.ok ? floor(fxd) : 0.0, jcd = r.ok ? floor(fyd) : 0.0;
    r.ic = (int)icd;
    r.jc = (int)jcd;
    r.fx = (float)((fxd - icd) * p.dx_d);
    r.fy = (float)((fyd - jcd) * p.dy_d);
    return r;
}

__device__ __forceinline__ int atom_bin(int jc, float z, const PotParams& p) {
    int jw = jc % p.ny;
    if (jw < 0) jw += p.ny;
    const int band = jw / kBandRows;
    int slab = (int)floorf(__fmul_rn(__fsub_rn(z, p.z0), p.inv_dz));
    slab = min(max(slab, 0), p.n_slices - 1);
    return slab * p.n_bands + band;
}

__global__ void __launch_bounds__(kBinThreads)
bin_kernel(const float* __restrict__ pos, const int* __restrict__ species, PotParams p,
           int* __restrict__ bin_off, float4* __restrict__ binned, int2* __restrict__ binned_px) {
    extern __shared__ int cnt[];
    __shared__ int warp_off[kBinThreads / 32];
    const size_t t = blockIdx.x;
    const float* P = pos + t * (size_t)p.n_atoms * 3;
    for (int b = threadIdx.x; b < p.n_bins; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < p.n_atoms; a += blockDim.x) {
        const Split sp = split_position(P[3 * a], P[3 * a + 1], p);
        atomicAdd(&cnt[atom_bin(sp.jc, P[3 * a + 2], p)], 1);
    }
    __syncthreads();

    // exclusive scan of the counts; thread i owns a contiguous chunk of bins
    const int chunk = (p.n_bins + blockDim.x - 1) / blockDim.x;
    const int c0 = min((int)threadIdx.x * chunk, p.n_bins), c1 = min(c0 + chunk, p.n_bins);
    int local = 0;
    for (int b = c0; b < c1; ++b) local += cnt[b];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_off[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x / 32;
        const int mine = lane < nw ? warp_off[lane] : 0;
        int wi = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        if (lane < nw) warp_off[lane] = wi - mine;
    }
    __syncthreads();
    int run = warp_off[wid] + incl - local;
    int* off = bin_off + t * (size_t)(p.n_bins + 1);
    for (int b = c0; b < c1; ++b) {
        const int c = cnt[b];
        cnt[b] = run;
        off[b] = run;
        run += c;
    }
    if (threadIdx.x == 0) off[p.n_bins] = p.n_atoms;
    __syncthreads();

    float4* out = binned + t * (size_t)p.n_atoms;
    int2* out_px = binned_px + t * (size_t)p.n_atoms;
    for (int a = threadIdx.x; a < p.n_atoms; a += blockDim.x) {
        const float z = P[3 * a + 2];
        const Split sp = split_position(P[3 * a], P[3 * a + 1], p);
        const int slot = atomicAdd(&cnt[atom_bin(sp.jc, z, p)], 1);
        // a species of -1 marks an atom that is skipped (non-finite or absurd position)
        const int spc = (sp.ok && fabsf(z) < 1e9f) ? __ldg(species + a) : -1;
        out[slot] = make_float4(sp.fx, sp.fy, z, __int_as_float(spc));
        out_px[slot] = make_int2(sp.ic, sp.jc);
    }
}

// Candidate atoms of one block, gathered per chunk of source atoms.
constexpr int kChunk = kPotThreads;      // source atoms examined per chunk
constexpr int kSegs = kPotThreads / 32;  // one column segment per warp
constexpr int kMaxNbBins = 64;           // neighbouring bins scanned per block

struct CandSmem {
    int ic[kChunk], jc[kChunk];                 // pixel index of the atom (wrapped into the box)
    float fx[kChunk], fy[kChunk];               // offset of the atom from that pixel, A
    float aw[kChunk], inv2s2[kChunk], rc2[kChunk];
    int sp[kChunk];
    float w[kChunk], dw[kChunk];                // slice weight and d(weight)/d(sigma)
    float gy[kChunk][kBandRows];
    float dy2[kChunk][kBandRows];
    unsigned short seg_list[kSegs][kChunk];
    int seg_cnt[kSegs];
    int n_cand;
    int bin_start[kMaxNbBins], bin_cum[kMaxNbBins + 1];
    int n_nb;
};

struct Tile {
    int band, s, r0, nrows, seg_w;
    size_t t;
    bool first, lastsl;
    float lo, hi, band_span;
};

__device__ __forceinline__ Tile make_tile(const PotParams& p) {
    Tile tl;
    tl.band = blockIdx.x;
    tl.s = blockIdx.y;
    tl.t = blockIdx.z;
    tl.r0 = tl.band * kBandRows;
    tl.nrows = min(kBandRows, p.ny - tl.r0);
    tl.seg_w = (p.nx + kSegs - 1) / kSegs;
    tl.first = (tl.s == 0);
    tl.lastsl = (tl.s == p.n_slices - 1);
    tl.lo = tl.first ? -INFINITY : p.z0 + (float)tl.s * p.dz;
    tl.hi = tl.lastsl ? INFINITY : p.z0 + (float)(tl.s + 1) * p.dz;
    tl.band_span = (float)(tl.nrows - 1) * p.dy;
    return tl;
}

// Neighbouring bins (slabs s +- slab_reach, bands +- band_reach) as one flat
// list: warp 0 loads the ranges and scans the counts.  Returns the number of
// source atoms (after a block barrier).
__device__ int load_neighbour_bins(CandSmem& sm, const PotParams& p, const int* __restrict__ off,
                                   const Tile& tl) {
    const int lane = threadIdx.x & 31;
    const int slab0 = max(0, tl.s - p.slab_reach), slab1 = min(p.n_slices - 1, tl.s + p.slab_reach);
    const bool all_bands = 2 * p.band_reach + 1 >= p.n_bands;
    const int nb = all_bands ? p.n_bands : 2 * p.band_reach + 1;
    const int n_nb = nb * (slab1 - slab0 + 1);
    if (threadIdx.x < 32) {
        int carry = 0;
        for (int base = 0; base < n_nb; base += 32) {
            const int i = base + lane;
            int cnt = 0, start = 0;
            if (i < n_nb) {
                const int slab = slab0 + i / nb, k = i % nb;
                int b = all_bands ? k : tl.band - p.band_reach + k;
                b = ((b % p.n_bands) + p.n_bands) % p.n_bands;
                const int bin = slab * p.n_bands + b;
                start = __ldg(off + bin);
                cnt = __ldg(off + bin + 1) - start;
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (i < n_nb) {
                sm.bin_start[i] = start;
                sm.bin_cum[i] = carry + incl - cnt;
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) {
            sm.bin_cum[n_nb] = carry;
            sm.n_nb = n_nb;
        }
    }
    __syncthreads();
    return sm.bin_cum[sm.n_nb];
}

// Candidates of one chunk of source atoms: the atoms that reach this slice
// and band, listed in every column segment their window touches, with their
// per-row Gaussian factors.  Ends with a block barrier.
__device__ void gather_chunk(CandSmem& sm, const PotParams& p, const float4* __restrict__ atoms,
                             const int2* __restrict__ atoms_px, const Tile& tl, int c0, int n_src) {
    if (threadIdx.x < kSegs) sm.seg_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) sm.n_cand = 0;
    __syncthreads();
    const int src = c0 + threadIdx.x;
    if (src < n_src) {
        int bi = 0;
        while (sm.bin_cum[bi + 1] <= src) ++bi;
        const int ai = sm.bin_start[bi] + (src - sm.bin_cum[bi]);
        const float4 at = atoms[ai];               // (fx, fy, z, species)
        const int2 px = atoms_px[ai];              // (ic, jc)
        const int sp = __float_as_int(at.w);
        bool ok = sp >= 0 && sp < p.n_species;
        const float sg = ok ? p.sigma[sp] : 1.f;
        const float rc = 6.0f * sg;
        ok = ok && (tl.hi > at.z - rc) && (tl.lo < at.z + rc);
        const int ic = px.x, jc = px.y;
        int k0 = (tl.r0 - jc) % p.ny;              // wrapped pixel distance of the band's first row
        if (k0 < 0) k0 += p.ny;
        if (k0 >= (p.ny + 1) / 2) k0 -= p.ny;
        const float d0 = (float)k0 * p.dy - at.y;
        ok = ok && (d0 <= rc) && (d0 + tl.band_span >= -rc);
        if (ok) {
            const float kz = 0.70710678118654752f / sg;
            const float uh = (tl.hi - at.z) * kz, ul = (tl.lo - at.z) * kz;
            const float fh = tl.lastsl ? 0.5f : 0.5f * erff(uh);
            const float fl = tl.first ? -0.5f : 0.5f * erff(ul);
            // d/dsigma of erf(u)/2 with u = (edge - z)/(sqrt2 sigma): -(u/sigma) exp(-u^2)/sqrt(pi)
            const float dh = tl.lastsl ? 0.f : -(uh / sg) * expf(-uh * uh) * 0.56418958354775628f;
            const float dl = tl.first ? 0.f : -(ul / sg) * expf(-ul * ul) * 0.56418958354775628f;
            const int c = atomicAdd(&sm.n_cand, 1);
            int icw = ic % p.nx, jcw = jc % p.ny;   // pixel indices wrapped into the box
            if (icw < 0) icw += p.nx;
            if (jcw < 0) jcw += p.ny;
            sm.ic[c] = icw;
            sm.jc[c] = jcw;
            sm.fx[c] = at.x;
            sm.fy[c] = at.y;
            sm.sp[c] = sp;
            sm.w[c] = fh - fl;
            sm.dw[c] = dh - dl;
            sm.aw[c] = p.amp[sp] * (fh - fl);
            sm.inv2s2[c] = 0.5f / (sg * sg);
            sm.rc2[c] = rc * rc;
            // columns within the cut-off lie in [i0, i0 + wx) (one spare column each side)
            const int reach = (int)ceilf(rc * p.inv_dx);
            const int i0 = ic - reach - 1;
            const int wx = 2 * reach + 3;
            unsigned mask = 0;
            if (wx >= p.nx) {
                mask = (1u << kSegs) - 1u;
            } else {
                int a = i0 % p.nx;
                if (a < 0) a += p.nx;
                const int b = a + wx - 1;
                for (int col = a; col <= b; col += tl.seg_w) mask |= 1u << ((col % p.nx) / tl.seg_w);
                mask |= 1u << ((b % p.nx) / tl.seg_w);
            }
            while (mask) {
                const int si = __ffs(mask) - 1;
                mask &= mask - 1;
                const int slot = atomicAdd(&sm.seg_cnt[si], 1);
                sm.seg_list[si][slot] = (unsigned short)c;
            }
        }
    }
    __syncthreads();
    const int nc = sm.n_cand;
    for (int e = threadIdx.x; e < nc * kBandRows; e += blockDim.x) {
        const int c = e / kBandRows, r = e % kBandRows;
        int k = tl.r0 + r - sm.jc[c];              // in (-ny, ny): wrap to the nearest image
        if (k >= (p.ny + 1) / 2) k -= p.ny;
        if (k < -(p.ny / 2)) k += p.ny;
        const float ddy = (float)k * p.dy - sm.fy[c];
        const float d2 = ddy * ddy;
        const bool in = r < tl.nrows && d2 <= sm.rc2[c];
        sm.dy2[c][r] = in ? d2 : INFINITY;
        sm.gy[c][r] = in ? expf(-d2 * sm.inv2s2[c]) : 0.f;
    }
    __syncthreads();
}

// Squared distance from column `col` to candidate c (nearest image), wrapped
// integer pixel distance times dx minus the atom's offset in its pixel.
__device__ __forceinline__ float col_dist2(const CandSmem& sm, const PotParams& p, int c, int col) {
    int kx = col - sm.ic[c];                        // in (-nx, nx): wrap to the nearest image
    if (kx >= (p.nx + 1) / 2) kx -= p.nx;
    if (kx < -(p.nx / 2)) kx += p.nx;
    const float ddx = (float)kx * p.dx - sm.fx[c];
    return ddx * ddx;
}

// One block per (band of kBandRows rows, slice, snapshot).  Warp w owns the
// column segment [w * seg_w, (w + 1) * seg_w) (CPL columns per lane) and keeps
// the band's sums for those columns in 64-bit fixed-point registers: no
// atomics on pixels, the Gaussian is evaluated separably (one row factor per
// candidate and row, one column factor per candidate and column), and the
// result does not depend on the order in which candidates arrive.
template <int CPL>
__global__ void __launch_bounds__(kPotThreads)
potential_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                 const int2* __restrict__ binned_px, PotParams p, float* __restrict__ V) {
    __shared__ CandSmem sm;
    const Tile tl = make_tile(p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* atoms = binned + tl.t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + tl.t * (size_t)p.n_atoms;
    const int n_src = load_neighbour_bins(sm, p, bin_off + tl.t * (size_t)(p.n_bins + 1), tl);

    long long acc[CPL][kBandRows];
#pragma unroll
    for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int r = 0; r < kBandRows; ++r) acc[k][r] = 0;
    const int col0 = warp * tl.seg_w;
    const int col1 = min(col0 + tl.seg_w, p.nx);

    for (int c0 = 0; c0 < n_src; c0 += kChunk) {
        gather_chunk(sm, p, atoms, atoms_px, tl, c0, n_src);
        const int cnt = sm.seg_cnt[warp];
        for (int j = 0; j < cnt; ++j) {
            const int c = sm.seg_list[warp][j];
            const float aw = sm.aw[c], inv2s2 = sm.inv2s2[c], rc2 = sm.rc2[c];
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int col = col0 + lane + 32 * k;
                if (col >= col1) continue;
                const float dx2 = col_dist2(sm, p, c, col);
                if (dx2 > rc2) continue;
                const float gx = aw * expf(-dx2 * inv2s2);
#pragma unroll
                for (int r = 0; r < kBandRows; ++r)   // square cut-off: |dx|, |dy| <= 6 s
                    if (sm.dy2[c][r] <= rc2) acc[k][r] += __float2int_rn(gx * sm.gy[c][r] * kFixScale);
            }
        }
        __syncthreads();
    }
    // write the band (lanes on consecutive columns)
    float* out = V + ((tl.t * p.n_slices + tl.s) * (size_t)p.ny + tl.r0) * p.nx;
#pragma unroll
    for (int k = 0; k < CPL; ++k) {
        const int col = col0 + lane + 32 * k;
        if (col >= col1) continue;
#pragma unroll
        for (int r = 0; r < kBandRows; ++r)
            if (r < tl.nrows) {
                // sums below 2048 V*A fit in 32 bits: convert those without the FP64 pipe
                const long long a = acc[k][r];
                const float f = (a == (long long)(int)a) ? (float)(int)a : (float)a;
                out[(size_t)r * p.nx + col] = f * kFixInv;
            }
    }
}

// Adjoint of the potential for the per-species Gaussian parameters: with
// P = exp(-rho^2 / 2 s^2) inside the cut-off and g = dL/dv,
//   dL/d amp += g P w,   dL/d s += g amp P (rho^2 / s^3 w + dw/ds).
// Each lane sums its contributions per candidate, the warp reduces them and
// adds to per-species FP64 block totals; every block writes its totals to
// `partial` [block][n_species][2] for a fixed-order final reduction.
template <int CPL>
__global__ void __launch_bounds__(kPotThreads)
potential_backward_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                          const int2* __restrict__ binned_px, PotParams p, const float* __restrict__ dV,
                          double* __restrict__ partial) {
    __shared__ CandSmem sm;
    __shared__ double tot[TACAW_MAX_SPECIES][2];
    extern __shared__ float gtile[];                // [kBandRows][nx]: dL/dv of the band
    const Tile tl = make_tile(p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* atoms = binned + tl.t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + tl.t * (size_t)p.n_atoms;
    if (threadIdx.x < 2 * TACAW_MAX_SPECIES) tot[threadIdx.x / 2][threadIdx.x % 2] = 0.0;
    const float* grow = dV + ((tl.t * p.n_slices + tl.s) * (size_t)p.ny + tl.r0) * p.nx;
    for (int i = threadIdx.x; i < tl.nrows * p.nx; i += blockDim.x)
        gtile[i] = __ldg(grow + i);
    const int n_src = load_neighbour_bins(sm, p, bin_off + tl.t * (size_t)(p.n_bins + 1), tl);
    const int col0 = warp * tl.seg_w;
    const int col1 = min(col0 + tl.seg_w, p.nx);

    for (int c0 = 0; c0 < n_src; c0 += kChunk) {
        gather_chunk(sm, p, atoms, atoms_px, tl, c0, n_src);
        const int cnt = sm.seg_cnt[warp];
        for (int j = 0; j < cnt; ++j) {
            const int c = sm.seg_list[warp][j];
            const int sp = sm.sp[c];
            const float inv2s2 = sm.inv2s2[c], rc2 = sm.rc2[c];
            const float sg = p.sigma[sp];
            const float inv_s3 = 1.0f / (sg * sg * sg);
            const float w = sm.w[c], dw = sm.dw[c];
            float ga = 0.f, gs = 0.f;
#pragma unroll
            for (int k = 0; k < CPL; ++k) {
                const int col = col0 + lane + 32 * k;
                if (col >= col1) continue;
                const float dx2 = col_dist2(sm, p, c, col);
                if (dx2 > rc2) continue;
                const float gx = expf(-dx2 * inv2s2);
#pragma unroll
                for (int r = 0; r < kBandRows; ++r) {
                    const float r2 = dx2 + sm.dy2[c][r];
                    if (sm.dy2[c][r] <= rc2) {             // square cut-off: |dx|, |dy| <= 6 s
                        const float gp = gtile[r * p.nx + col] * gx * sm.gy[c][r];
                        ga += gp;
                        gs += gp * r2;
                    }
                }
            }
            // ga = sum g P, gs = sum g P rho^2  ->  (w ga, amp (gs w / s^3 + ga dw))
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ga += __shfl_xor_sync(0xffffffffu, ga, o);
                gs += __shfl_xor_sync(0xffffffffu, gs, o);
            }
            if (lane == 0) {
                atomicAdd(&tot[sp][0], (double)ga * (double)w);
                atomicAdd(&tot[sp][1], (double)p.amp[sp] * ((double)gs * (double)w * (double)inv_s3 +
                                                            (double)ga * (double)dw));
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (threadIdx.x < 2 * p.n_species)
        partial[blk * 2 * p.n_species + threadIdx.x] = tot[threadIdx.x / 2][threadIdx.x % 2];
}

// out[i] = sum over blocks of partial[block][i], fixed order (one block per i).
__global__ void __launch_bounds__(256)
reduce_partials_kernel(const double* __restrict__ partial, size_t n_blocks, int n_vals,
                       double* __restrict__ out) {
    __shared__ double sh[256];
    const int i = blockIdx.x;
    double acc = 0.0;
    for (size_t b = threadIdx.x; b < n_blocks; b += blockDim.x) acc += partial[b * n_vals + i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
}

struct PotWs {
    int* bin_off;
    float4* binned;
    int2* binned_px;
};

PotWs carve_pot(Carver& cv, int n_t, int n_atoms, int n_bins) {
    PotWs w;
    w.bin_off = cv.take<int>((size_t)n_t * (n_bins + 1));
    w.binned = cv.take<float4>((size_t)n_t * n_atoms);
    w.binned_px = cv.take<int2>((size_t)n_t * n_atoms);
    return w;
}

int make_params(const tacaw_grid& g, int n_atoms, int n_species, const float* amp_sigma,
                PotParams* p) {
    float smax = 0.f;
    for (int i = 0; i < n_species; ++i) {
        TACAW_REQUIRE(amp_sigma[2 * i + 1] > 0.f && isfinite(amp_sigma[2 * i + 1]) &&
                          fabsf(amp_sigma[2 * i]) <= kMaxAmp,
                      TACAW_EINVAL,
                      "tacaw_potential: species %d needs a width > 0 and |amplitude| <= %g V*A", i,
                      (double)kMaxAmp);
        p->amp[i] = amp_sigma[2 * i];
        p->sigma[i] = amp_sigma[2 * i + 1];
        smax = fmaxf(smax, amp_sigma[2 * i + 1]);
    }
    for (int i = n_species; i < TACAW_MAX_SPECIES; ++i) p->amp[i] = p->sigma[i] = 0.f;
    const double rc = 6.0 * smax;
    TACAW_REQUIRE(2.0 * rc < g.lx && 2.0 * rc < g.ly, TACAW_EINVAL,
                  "tacaw_potential: cut-off 6 sigma = %g A must be below half the box", rc);
    p->nx = g.nx;
    p->ny = g.ny;
    p->n_slices = g.n_slices;
    p->n_atoms = n_atoms;
    p->n_species = n_species;
    p->n_bands = (g.ny + kBandRows - 1) / kBandRows;
    p->n_bins = g.n_slices * p->n_bands;
    const double dy = g.ly / g.ny;
    // an atom in pixel row jc reaches rows jc - ceil(rc/dy) .. jc + 1 + ceil(rc/dy); the
    // slab is assigned in float, so its reach gets a little slack
    p->band_reach = (int)ceil((ceil(rc / dy) + 1.0) / kBandRows);
    p->slab_reach = (int)ceil((rc + 1e-4 * g.dz) / g.dz);
    p->lx = (float)g.lx;
    p->ly = (float)g.ly;
    p->dx = (float)(g.lx / g.nx);
    p->dy = (float)dy;
    p->inv_dx = (float)(g.nx / g.lx);
    p->inv_lx = (float)(1.0 / g.lx);
    p->dx_d = g.lx / g.nx;
    p->dy_d = g.ly / g.ny;
    p->inv_dx_d = g.nx / g.lx;
    p->inv_dy_d = g.ny / g.ly;
    p->inv_ly = (float)(1.0 / g.ly);
    p->z0 = (float)g.z0;
    p->dz = (float)g.dz;
    p->inv_dz = (float)(1.0 / g.dz);
    p->inv_band_h = (float)(1.0 / (kBandRows * dy));
    return TACAW_OK;
}

}  // namespace

static size_t pot_backward_blocks(const tacaw_grid& g, int n_t) {
    return (size_t)((g.ny + kBandRows - 1) / kBandRows) * g.n_slices * n_t;
}

int potential_backward_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, int n_species, size_t* bytes) {
    const int n_bins = g.n_slices * ((g.ny + kBandRows - 1) / kBandRows);
    Carver cv(nullptr);
    carve_pot(cv, n_t, n_atoms, n_bins);
    cv.take<double>(pot_backward_blocks(g, n_t) * 2 * n_species);
    *bytes = cv.bytes();
    return TACAW_OK;
}

int potential_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, size_t* bytes) {
    const int n_bins = g.n_slices * ((g.ny + kBandRows - 1) / kBandRows);
    Carver cv(nullptr);
    carve_pot(cv, n_t, n_atoms, n_bins);
    *bytes = cv.bytes();
    return TACAW_OK;
}

static int check_tables(const tacaw_grid& g, const PotParams& p) {
    const size_t bin_smem = (size_t)p.n_bins * sizeof(int);
    TACAW_REQUIRE(bin_smem <= 200 * 1024, TACAW_EUNSUPPORTED,
                  "tacaw_potential: %d bins exceed the shared-memory histogram", p.n_bins);
    TACAW_REQUIRE(g.nx <= 4 * 32 * kSegs, TACAW_EUNSUPPORTED,
                  "tacaw_potential: nx = %d above the supported %d", g.nx, 4 * 32 * kSegs);
    const int nb = (2 * p.band_reach + 1 >= p.n_bands) ? p.n_bands : 2 * p.band_reach + 1;
    const int n_nb = nb * (min(g.n_slices - 1, 2 * p.slab_reach) + 1);
    TACAW_REQUIRE(n_nb <= kMaxNbBins, TACAW_EUNSUPPORTED,
                  "tacaw_potential: %d neighbouring bins per tile exceed %d (widths too large for "
                  "the slice thickness or pixel size)", n_nb, kMaxNbBins);
    return TACAW_OK;
}

static int run_binning(const PotParams& p, int n_t, const float* pos, const int* species, PotWs& w,
                       cudaStream_t st) {
    const size_t bin_smem = (size_t)p.n_bins * sizeof(int);
    TACAW_CUDA_CHECK(ensure_smem((const void*)bin_kernel, (int)bin_smem));
    bin_kernel<<<n_t, kBinThreads, bin_smem, st>>>(pos, species, p, w.bin_off, w.binned, w.binned_px);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int potential_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos, const int* species,
                  int n_species, const float* amp_sigma, float* V, void* ws, cudaStream_t st) {
    PotParams p;
    int rc = make_params(g, n_atoms, n_species, amp_sigma, &p);
    if (rc == TACAW_OK) rc = check_tables(g, p);
    if (rc != TACAW_OK) return rc;
    Carver cv(ws);
    PotWs w = carve_pot(cv, n_t, n_atoms, p.n_bins);
    rc = run_binning(p, n_t, pos, species, w, st);
    if (rc != TACAW_OK) return rc;
    dim3 grid(p.n_bands, g.n_slices, n_t);
    const int cpl = ((g.nx + kSegs - 1) / kSegs + 31) / 32;
    if (cpl <= 1)
        potential_kernel<1><<<grid, kPotThreads, 0, st>>>(w.bin_off, w.binned, w.binned_px, p, V);
    else if (cpl == 2)
        potential_kernel<2><<<grid, kPotThreads, 0, st>>>(w.bin_off, w.binned, w.binned_px, p, V);
    else
        potential_kernel<4><<<grid, kPotThreads, 0, st>>>(w.bin_off, w.binned, w.binned_px, p, V);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int potential_backward_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos,
                           const int* species, int n_species, const float* amp_sigma, const float* dV,
                           double* grad, void* ws, cudaStream_t st) {
    PotParams p;
    int rc = make_params(g, n_atoms, n_species, amp_sigma, &p);
    if (rc == TACAW_OK) rc = check_tables(g, p);
    if (rc != TACAW_OK) return rc;
    Carver cv(ws);
    PotWs w = carve_pot(cv, n_t, n_atoms, p.n_bins);
    const size_t n_blocks = pot_backward_blocks(g, n_t);
    double* partial = cv.take<double>(n_blocks * 2 * n_species);
    rc = run_binning(p, n_t, pos, species, w, st);
    if (rc != TACAW_OK) return rc;
    dim3 grid(p.n_bands, g.n_slices, n_t);
    const int cpl = ((g.nx + kSegs - 1) / kSegs + 31) / 32;
    const int dsm = (int)(kBandRows * g.nx * sizeof(float));
    if (cpl <= 1) {
        TACAW_CUDA_CHECK(ensure_smem((const void*)potential_backward_kernel<1>, dsm));
        potential_backward_kernel<1><<<grid, kPotThreads, dsm, st>>>(w.bin_off, w.binned, w.binned_px, p, dV, partial);
    } else if (cpl == 2) {
        TACAW_CUDA_CHECK(ensure_smem((const void*)potential_backward_kernel<2>, dsm));
        potential_backward_kernel<2><<<grid, kPotThreads, dsm, st>>>(w.bin_off, w.binned, w.binned_px, p, dV, partial);
    } else {
        TACAW_CUDA_CHECK(ensure_smem((const void*)potential_backward_kernel<4>, dsm));
        potential_backward_kernel<4><<<grid, kPotThreads, dsm, st>>>(w.bin_off, w.binned, w.binned_px, p, dV, partial);
    }
    TACAW_LAUNCH_CHECK();
    reduce_partials_kernel<<<2 * n_species, 256, 0, st>>>(partial, n_blocks, 2 * n_species, grad);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace tacaw
