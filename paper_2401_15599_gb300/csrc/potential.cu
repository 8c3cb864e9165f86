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
//     bins (slab of the atom centre) x (band of rows) x (tile of columns); each
//     bin is sorted back into input order, so the bins of identical
//     configurations are identical.
//  2. potential_tile_kernel (one block per 32 x 64 pixel tile, slice and
//     snapshot): the separable Gaussian makes the tile a sum of outer products,
//     V_tile = sum_a gy_a (x) gx_a, accumulated in FP32 registers over the
//     candidate atoms in bin order (a fixed order: identical configurations give
//     bit-identical potentials).
//     When 6 s <= dz for every species, potential_slab_kernel takes its place:
//     one block per tile and snapshot walks the slabs, tabulating each slab's
//     candidates once and accumulating them into the three slices they reach.
// The adjoint (potential_backward_kernel) keeps one block per band of 8 rows.

#include <math.h>
#include <algorithm>
#include <stdint.h>

#include "common.cuh"

namespace tacaw {

namespace {

constexpr int kBandRows = 8;             // rows per band of the adjoint kernel
constexpr int kBinThreads = 1024;
constexpr int kPotThreads = 256;
constexpr int kMaxBinInts = 48 * 1024;   // bins per snapshot held by the histogram (192 KiB)
constexpr float kMaxAmp = 2000.0f;

struct PotParams {
    int nx, ny, n_slices, n_atoms, n_species;
    // bins: (slab, band of band_h rows, tile of ctile_w columns)
    int n_bands, n_ctiles, n_bins, band_h, ctile_w;
    int slab_reach;                            // neighbouring slabs that can reach a slice
    int nb_max, nc_max;                        // most bands / column tiles any tile needs
    int reach_x, reach_y;                      // ceil(6 s_max / d): pixels an atom reaches
    float lx, ly, dx, dy, inv_dx, z0, dz, inv_dz;
    double dx_d, dy_d, inv_dx_d, inv_dy_d;
    float amp[TACAW_MAX_SPECIES], sigma[TACAW_MAX_SPECIES];
    // per species: log2(e) / (2 s^2), 6 s and 1 / (sqrt2 s), rounded once on the host
    float c2[TACAW_MAX_SPECIES], rc[TACAW_MAX_SPECIES], kz[TACAW_MAX_SPECIES];
};

// An atom's position is split once, in FP64, into the pixel (ic, jc) that
// holds it and a small offset (fx, fy) from that pixel, so that later
// pixel-atom distances k*d - f carry no rounding from large coordinates.
// The binned copy keeps (ic, jc) wrapped into the box.
// Its slab comes from z with explicit round-to-nearest operations (the bin is
// computed twice per atom, count then scatter, and both passes must agree).
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

__device__ __forceinline__ int wrap(int k, int n) {
    k %= n;
    return k < 0 ? k + n : k;
}

// Bins along one periodic axis (bands of w rows or column tiles of w columns,
// the last one shorter when w does not divide n) holding a pixel within R of
// bin `bin`'s pixels, through the wrap: `count` bins from `first` on, modulo
// n_axis.  Counted from pixel intervals, not from whole bins, because across a
// short last bin a pixel R away can lie two or more bins over.
struct AxisRange {
    int first, count;
};

__host__ __device__ __forceinline__ AxisRange axis_range(int bin, int w, int n, int n_axis, int R) {
    const int t0 = bin * w, len = (n - t0 < w) ? n - t0 : w;
    AxisRange a;
    a.first = 0;
    a.count = n_axis;
    if (len + 2 * R >= n) return a;                  // the interval covers the axis
    const int lo = t0 - R, hi = t0 + len - 1 + R;   // -n < lo, hi < 2n
    const int bf = (lo < 0 ? lo + n : lo) / w, bl = (hi >= n ? hi - n : hi) / w;
    if (lo >= 0 && hi < n) {
        a.first = bf;
        a.count = bl - bf + 1;
    } else if (bl < bf) {                            // wraps without meeting itself
        a.first = bf;
        a.count = n_axis - bf + bl + 1;
    }
    return a;
}

__device__ __forceinline__ int atom_bin(const Split& sp, float z, const PotParams& p) {
    const int band = wrap(sp.jc, p.ny) / p.band_h;
    const int ct = wrap(sp.ic, p.nx) / p.ctile_w;
    int slab = (int)floorf(__fmul_rn(__fsub_rn(z, p.z0), p.inv_dz));
    slab = min(max(slab, 0), p.n_slices - 1);
    return (slab * p.n_bands + band) * p.n_ctiles + ct;
}

// Shell sort (Knuth's gaps) of one bin's records by atom index (key.x): bins
// hold a handful of atoms, so this is an insertion sort in practice, and any
// crowded bin still ends in input order.
__device__ void sort_bin_by_index(float4* __restrict__ rec, int2* __restrict__ key, int n) {
    int h = 1;
    while (h < n / 3) h = 3 * h + 1;
    for (; h >= 1; h /= 3) {
        for (int i = h; i < n; ++i) {
            const int2 kk = key[i];
            const float4 rr = rec[i];
            int j = i;
            while (j >= h && key[j - h].x > kk.x) {
                key[j] = key[j - h];
                rec[j] = rec[j - h];
                j -= h;
            }
            key[j] = kk;
            rec[j] = rr;
        }
    }
}

// One block per snapshot.  Counts per bin (shared-memory histogram), an
// exclusive scan into bin_off, a scatter whose slots come from shared-memory
// atomics (any order; the atom index and the packed pixel ride along in the
// pixel array), then every bin sorted back into input order and its pixels
// unpacked, so every bin lists its atoms in input order.
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
        atomicAdd(&cnt[atom_bin(sp, P[3 * a + 2], p)], 1);
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
        const int slot = atomicAdd(&cnt[atom_bin(sp, z, p)], 1);
        // a species of -1 marks an atom that is skipped (non-finite or absurd position)
        const int spc = (sp.ok && fabsf(z) < 1e9f) ? __ldg(species + a) : -1;
        out[slot] = make_float4(sp.fx, sp.fy, z, __int_as_float(spc));
        out_px[slot] = make_int2(a, (int)((unsigned)wrap(sp.ic, p.nx) | ((unsigned)wrap(sp.jc, p.ny) << 16)));
    }
    __syncthreads();                               // cnt[b] is now the end of bin b
    for (int b = threadIdx.x; b < p.n_bins; b += blockDim.x) {
        const int s0 = b ? cnt[b - 1] : 0, s1 = cnt[b];
        sort_bin_by_index(out + s0, out_px + s0, s1 - s0);
        for (int i = s0; i < s1; ++i) {
            const unsigned pk = (unsigned)out_px[i].y;
            out_px[i] = make_int2((int)(pk & 0xffffu), (int)(pk >> 16));
        }
    }
}

// Neighbouring bins of a tile (slabs slab0 .. slab1; the bands and column
// tiles holding a pixel within reach + 1 of the tile, from axis_range) as one
// flat list: warp 0 loads the ranges and scans the counts into bin_start /
// bin_cum.  Returns the number of source atoms (after a block barrier).
constexpr int kMaxNbBins = 128;

__device__ int load_bins_slabs(int* bin_start, int* bin_cum, const PotParams& p, const int* __restrict__ off,
                               int slab0, int slab1, int band, int ctile, int* n_nb_out) {
    const int lane = threadIdx.x & 31;
    const AxisRange rb = axis_range(band, p.band_h, p.ny, p.n_bands, p.reach_y + 1);
    const AxisRange rx = axis_range(ctile, p.ctile_w, p.nx, p.n_ctiles, p.reach_x + 1);
    const int nb = rb.count, nc = rx.count;
    const int n_nb = nb * nc * (slab1 - slab0 + 1);
    if (threadIdx.x < 32) {
        int carry = 0;
        for (int base = 0; base < n_nb; base += 32) {
            const int i = base + lane;
            int cnt = 0, start = 0;
            if (i < n_nb) {
                const int slab = slab0 + i / (nb * nc);
                const int kb = (i / nc) % nb, kc = i % nc;
                const int b = (rb.first + kb) % p.n_bands;
                const int c = (rx.first + kc) % p.n_ctiles;
                const int bin = (slab * p.n_bands + b) * p.n_ctiles + c;
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
                bin_start[i] = start;
                bin_cum[i] = carry + incl - cnt;
            }
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) bin_cum[n_nb] = carry;
    }
    __syncthreads();
    *n_nb_out = n_nb;
    return bin_cum[n_nb];
}

__device__ int load_bins(int* bin_start, int* bin_cum, const PotParams& p, const int* __restrict__ off,
                         int s, int band, int ctile, int* n_nb_out) {
    return load_bins_slabs(bin_start, bin_cum, p, off, max(0, s - p.slab_reach),
                           min(p.n_slices - 1, s + p.slab_reach), band, ctile, n_nb_out);
}

// Source index -> atom index through the scanned bin list: the last bin whose
// running count is <= src (never an empty bin) holds it.
__device__ __forceinline__ int source_atom(const int* bin_start, const int* bin_cum, int n_nb, int src) {
    int lo = 0, hi = n_nb - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (bin_cum[mid] <= src) lo = mid; else hi = mid - 1;
    }
    return bin_start[lo] + (src - bin_cum[lo]);
}

// Slice weight of an atom at height z with width sg in slice [lo, hi):
// (erf((hi - z)/(sqrt2 sg)) - erf((lo - z)/(sqrt2 sg))) / 2, open at the first
// and last slice; `dw` receives d(weight)/d(sigma).
__device__ __forceinline__ float slice_weight(float z, float sg, float lo, float hi, bool first,
                                              bool lastsl, float* dw) {
    const float kz = 0.70710678118654752f / sg;
    const float uh = (hi - z) * kz, ul = (lo - z) * kz;
    const float fh = lastsl ? 0.5f : 0.5f * erff(uh);
    const float fl = first ? -0.5f : 0.5f * erff(ul);
    if (dw) {
        // d/dsigma of erf(u)/2 with u = (edge - z)/(sqrt2 sigma): -(u/sigma) exp(-u^2)/sqrt(pi)
        const float dh = lastsl ? 0.f : -(uh / sg) * expf(-uh * uh) * 0.56418958354775628f;
        const float dl = first ? 0.f : -(ul / sg) * expf(-ul * ul) * 0.56418958354775628f;
        *dw = dh - dl;
    }
    return fh - fl;
}

// Nearest periodic image of a pixel offset k in (-n, n).
__device__ __forceinline__ int nearest_image(int k, int n) {
    if (k >= (n + 1) / 2) k -= n;
    if (k < -(n / 2)) k += n;
    return k;
}

// Smallest distance |k d - f| (nearest images) from an atom in pixel c, at
// offset f, to the pixels [a, a + len), with c and a in [0, n): 0 when the
// atom's pixel is in the range, else the nearer end of the range (the offsets
// k run monotonically away from the atom between the ends).
__device__ __forceinline__ float range_gap(int c, float f, int a, int len, int n, float d) {
    int u = c - a;
    if (u < 0) u += n;
    if (u < len) return 0.f;
    const float d0 = fabsf((float)nearest_image(a - c, n) * d - f);
    const float d1 = fabsf((float)nearest_image(a + len - 1 - c, n) * d - f);
    return fminf(d0, d1);
}

// ------------------------------------------------------------------ forward
// One block per (tile of kTR rows x kTC columns, slice, snapshot).  Lane l of
// every warp owns tile row l; warp w owns the 8 columns [8w, 8w + 8), so each
// thread accumulates 8 pixels in registers.  The block
//  1. examines the sources of the neighbouring bins, one per thread, and keeps
//     those that reach this slice and tile as candidates (compacted in source
//     order);
//  2. per group of kTCand candidates tabulates the row factors
//     gy[r] = exp(-dy^2 / 2 s^2) over the tile rows and the column factors
//     gx[c] = amp w_s exp(-dx^2 / 2 s^2) over the tile columns (0 outside
//     |d| <= 6 s), one warp per candidate, with a mask of the 8-column groups
//     the candidate touches;
//  3. lets every warp run over the candidates that touch its columns, in order:
//     acc += gy[lane] * gx[8w .. 8w + 7].
constexpr int kTR = 32;
constexpr int kTC = 64;
constexpr int kTCand = 64;               // candidates tabulated at a time
constexpr int kTWarps = kPotThreads / 32;
static_assert(kTC == 8 * kTWarps && kTR == 32, "tile = 32 rows x 8 columns per warp");

struct TileSmem {
    float gy[kTCand][kTR];
    float4 gx[kTCand][kTC / 4];
    int wmask[kTCand];
    unsigned char wlist[kTWarps][kTCand];
    // candidates of one pass over the sources: nearest-image pixel offsets of the
    // tile's first row / column from the atom, the atom's offset in its pixel,
    // amp * w_s, log2(e) / (2 s^2) and the cut-off 6 s
    int k0y[kPotThreads], k0x[kPotThreads];
    float fx[kPotThreads], fy[kPotThreads], aw[kPotThreads], c2[kPotThreads], rc[kPotThreads];
    int warp_cnt[kTWarps];
    int bin_start[kMaxNbBins], bin_cum[kMaxNbBins + 1];
};

// Exact float of a small integer (|k| < 2^22) without a conversion instruction.
__device__ __forceinline__ float small_int_to_float(int k) {
    return __int_as_float(0x4B400000 + k) - 12582912.0f;
}

__global__ void __launch_bounds__(kPotThreads, 6)
potential_tile_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                      const int2* __restrict__ binned_px, PotParams p, int n_tx, int vec_out,
                      float* __restrict__ V) {
    extern __shared__ __align__(16) unsigned char tile_smem_raw[];
    TileSmem& sm = *reinterpret_cast<TileSmem*>(tile_smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int r0 = (blockIdx.x / n_tx) * kTR, c0 = (blockIdx.x % n_tx) * kTC;
    const int s = blockIdx.y;
    const size_t t = blockIdx.z;
    const int nrows = min(kTR, p.ny - r0), ncols = min(kTC, p.nx - c0);
    const int half_x = (p.nx + 1) / 2, half_y = (p.ny + 1) / 2;
    const bool first = (s == 0), lastsl = (s == p.n_slices - 1);
    const float lo = first ? -INFINITY : p.z0 + (float)s * p.dz;
    const float hi = lastsl ? INFINITY : p.z0 + (float)(s + 1) * p.dz;
    const float4* atoms = binned + t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + t * (size_t)p.n_atoms;
    int n_nb;
    const int n_src = load_bins(sm.bin_start, sm.bin_cum, p, bin_off + t * (size_t)(p.n_bins + 1), s,
                                r0 / p.band_h, c0 / p.ctile_w, &n_nb);

    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = 0.f;

    for (int sb = 0; sb < n_src; sb += kPotThreads) {
        // 1. candidates among the sources [sb, sb + kPotThreads), in source order
        bool ok = false;
        float4 at = make_float4(0.f, 0.f, 0.f, 0.f);
        int icw = 0, jcw = 0, sp = 0;
        float rc = 0.f;
        if (sb + (int)threadIdx.x < n_src) {
            const int ai = source_atom(sm.bin_start, sm.bin_cum, n_nb, sb + threadIdx.x);
            at = atoms[ai];                              // (fx, fy, z, species)
            const int2 px = atoms_px[ai];                // (ic, jc), wrapped
            sp = __float_as_int(at.w);
            ok = sp >= 0 && sp < p.n_species;
            rc = 6.0f * (ok ? p.sigma[sp] : 1.f);
            ok = ok && (hi > at.z - rc) && (lo < at.z + rc);
            icw = px.x;
            jcw = px.y;
            ok = ok && range_gap(jcw, at.y, r0, nrows, p.ny, p.dy) <= rc &&
                 range_gap(icw, at.x, c0, ncols, p.nx, p.dx) <= rc;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) sm.warp_cnt[warp] = __popc(bal);
        __syncthreads();
        int n_cand = 0, my_off = 0;
#pragma unroll
        for (int w = 0; w < kTWarps; ++w) {
            const int c = sm.warp_cnt[w];
            if (w < warp) my_off += c;
            n_cand += c;
        }
        if (ok) {
            const int c = my_off + __popc(bal & lt);
            const float sg = p.sigma[sp];
            sm.k0y[c] = nearest_image(r0 - jcw, p.ny);
            sm.k0x[c] = nearest_image(c0 - icw, p.nx);
            sm.fx[c] = at.x;
            sm.fy[c] = at.y;
            sm.aw[c] = p.amp[sp] * slice_weight(at.z, sg, lo, hi, first, lastsl, nullptr);
            sm.c2[c] = 1.4426950408889634f * (0.5f / (sg * sg));
            sm.rc[c] = rc;
        }
        __syncthreads();

        for (int cb = 0; cb < n_cand; cb += kTCand) {
            const int nc = min(kTCand, n_cand - cb);
            // 2. factors (square cut-off |dx|, |dy| <= 6 s): lane l gives row l and
            //    columns l, l + 32; offsets from the atom's pixel by nearest image
            for (int c = warp; c < nc; c += kTWarps) {
                const int cc = cb + c;
                const int k0y = sm.k0y[cc], k0x = sm.k0x[cc];
                const float fx = sm.fx[cc], fy = sm.fy[cc], aw = sm.aw[cc], c2 = sm.c2[cc], rcc = sm.rc[cc];
                float gyv = 0.f, g0 = 0.f, g1 = 0.f;
                int ky = k0y + lane;
                if (ky >= half_y) ky -= p.ny;
                int kx0 = k0x + lane;
                if (kx0 >= half_x) kx0 -= p.nx;
                int kx1 = k0x + lane + 32;
                if (kx1 >= half_x) kx1 -= p.nx;
                const float dy_ = small_int_to_float(ky) * p.dy - fy;
                const float dx0 = small_int_to_float(kx0) * p.dx - fx;
                const float dx1 = small_int_to_float(kx1) * p.dx - fx;
                if (lane < nrows && fabsf(dy_) <= rcc) gyv = exp2f(-(dy_ * dy_) * c2);
                if (lane < ncols && fabsf(dx0) <= rcc) g0 = aw * exp2f(-(dx0 * dx0) * c2);
                if (lane + 32 < ncols && fabsf(dx1) <= rcc) g1 = aw * exp2f(-(dx1 * dx1) * c2);
                sm.gy[c][lane] = gyv;
                float* gxr = reinterpret_cast<float*>(sm.gx[c]);
                gxr[lane] = g0;
                gxr[lane + 32] = g1;
                const unsigned b0 = __ballot_sync(0xffffffffu, g0 != 0.f);
                const unsigned b1 = __ballot_sync(0xffffffffu, g1 != 0.f);
                const int q = lane & 7;                  // lane q < 8 reports column group q
                const unsigned grp = (q < 4 ? b0 >> (8 * q) : b1 >> (8 * (q - 4))) & 0xffu;
                const unsigned wm = __ballot_sync(0xffffffffu, lane < 8 && grp != 0u);
                if (lane == 0) sm.wmask[c] = (int)wm;
            }
            __syncthreads();

            // 3. this warp's candidates, in order, then the outer-product updates
            int cnt = 0;
            for (int base = 0; base < nc; base += 32) {
                const int c = base + lane;
                const bool has = c < nc && ((sm.wmask[c] >> warp) & 1);
                const unsigned b = __ballot_sync(0xffffffffu, has);
                if (has) sm.wlist[warp][cnt + __popc(b & lt)] = (unsigned char)c;
                cnt += __popc(b);
            }
            __syncwarp();
#pragma unroll 2
            for (int j = 0; j < cnt; ++j) {
                const int c = sm.wlist[warp][j];
                const float gyv = sm.gy[c][lane];
                const float4 a = sm.gx[c][2 * warp], b = sm.gx[c][2 * warp + 1];
                acc[0] = fmaf(gyv, a.x, acc[0]);
                acc[1] = fmaf(gyv, a.y, acc[1]);
                acc[2] = fmaf(gyv, a.z, acc[2]);
                acc[3] = fmaf(gyv, a.w, acc[3]);
                acc[4] = fmaf(gyv, b.x, acc[4]);
                acc[5] = fmaf(gyv, b.y, acc[5]);
                acc[6] = fmaf(gyv, b.z, acc[6]);
                acc[7] = fmaf(gyv, b.w, acc[7]);
            }
            __syncthreads();
        }
        __syncthreads();                                 // the next pass rewrites the candidates
    }

    if (lane < nrows) {
        const int cw = 8 * warp;
        float* out = V + ((t * p.n_slices + s) * (size_t)p.ny + r0 + lane) * p.nx + c0 + cw;
        if (vec_out && cw + 8 <= ncols) {
            reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (cw + k < ncols) out[k] = acc[k];
        }
    }
}

// ------------------------------------------------------------------ forward, slab walk
// One block per (tile, snapshot) walks the slabs in order.  When 6 s <= dz an
// atom of slab k reaches only slices k-1, k and k+1, so each candidate of slab
// k is selected, tabulated and accumulated once, into three running slices
// held in registers (acc_m, acc_c, acc_p for slices k-1, k, k+1); slice k-1
// is complete after slab k and is written then.  The weights amp w_s(z) of
// the three slices come from the erf at the four slice boundaries around the
// slab.  Per slice the sum runs over slabs s-1, s, s+1, each in source order,
// as in the tile kernel: fixed by the configuration.
// Global-memory latency is taken off the slab-to-slab path: the tile's bin
// ranges of up to kTabInts / (2 n_nb + 1) slabs are loaded at once into a
// table, and while slab k is tabulated and accumulated the atom records of
// slab k+1 (its first kPotThreads sources) are copied into shared memory with
// cp.async.
constexpr int kSCand = 32;                // candidates tabulated at a time
constexpr int kSBins = 32;                // bins per slab neighbourhood (one warp scans them)
constexpr int kTabInts = 4096;            // bin table: per slab n_nb starts, n_nb + 1 running counts

struct SlabSmem {
    float gy[kSCand][kTR];
    float4 gx[kSCand][kTC / 4];
    float4 w[kSCand];                     // amp w_{k-1}, amp w_k, amp w_{k+1}, 0
    float4 st_at[2][kPotThreads];         // staged atom records of the next slab, by source index
    int2 st_px[2][kPotThreads];
    int wmask[kSCand];
    // candidates of one pass over the sources (see TileSmem)
    int k0y[kPotThreads], k0x[kPotThreads], spc[kPotThreads];
    float fx[kPotThreads], fy[kPotThreads], z[kPotThreads];
    int tab[kTabInts];
    int warp_cnt[kTWarps];
    unsigned char wlist[kTWarps][kSCand];
};

__device__ __forceinline__ void cp_async_16(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Bin table of slabs [k0, k0 + n_k): for slab k0 + j at tab + j (2 n_nb + 1):
// n_nb bin starts, then the n_nb + 1 running counts (the last = the slab's
// sources).  All threads load, one warp per slab scans; ends with a barrier.
__device__ void load_bin_table(int* tab, const PotParams& p, const int* __restrict__ off, int k0, int n_k,
                               AxisRange rb, AxisRange rx) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nc = rx.count, n_nb = rb.count * rx.count, stride = 2 * n_nb + 1;
    for (int e = threadIdx.x; e < n_k * n_nb; e += kPotThreads) {
        const int j = e / n_nb, i = e - j * n_nb;
        const int kb = i / nc, kc = i - kb * nc;
        const int b = (rb.first + kb) % p.n_bands, c = (rx.first + kc) % p.n_ctiles;
        const int bin = ((k0 + j) * p.n_bands + b) * p.n_ctiles + c;
        const int s0 = __ldg(off + bin);
        tab[j * stride + i] = s0;
        tab[j * stride + n_nb + i] = __ldg(off + bin + 1) - s0;
    }
    __syncthreads();
    for (int j = warp; j < n_k; j += kTWarps) {
        int* cum = tab + j * stride + n_nb;
        const int cnt = lane < n_nb ? cum[lane] : 0;
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane < n_nb) cum[lane] = incl - cnt;
        if (lane == 31) cum[n_nb] = incl;
    }
    __syncthreads();
}

// Height of slice boundary j: the first slice is open below, the last above.
__device__ __forceinline__ float slice_boundary(const PotParams& p, int j) {
    return j <= 0 ? -INFINITY : (j >= p.n_slices ? INFINITY : p.z0 + (float)j * p.dz);
}

__device__ __forceinline__ void store_tile_row(const PotParams& p, float* __restrict__ V, size_t t, int s, int r0,
                                               int c0, int nrows, int ncols, int vec_out, const float (&acc)[8]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < nrows) {
        const int cw = 8 * warp;
        float* out = V + ((t * p.n_slices + s) * (size_t)p.ny + r0 + lane) * p.nx + c0 + cw;
        if (vec_out && cw + 8 <= ncols) {
            reinterpret_cast<float4*>(out)[0] = make_float4(acc[0], acc[1], acc[2], acc[3]);
            reinterpret_cast<float4*>(out)[1] = make_float4(acc[4], acc[5], acc[6], acc[7]);
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (cw + k < ncols) out[k] = acc[k];
        }
    }
}

__global__ void __launch_bounds__(kPotThreads, 4)
potential_slab_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                      const int2* __restrict__ binned_px, PotParams p, int n_tx, int vec_out,
                      float* __restrict__ V) {
    static_assert(kSCand == 32 && kSBins <= 32, "one list lane per tabulated candidate, one scan lane per bin");
    extern __shared__ __align__(16) unsigned char slab_smem_raw[];
    SlabSmem& sm = *reinterpret_cast<SlabSmem*>(slab_smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int r0 = (blockIdx.x / n_tx) * kTR, c0 = (blockIdx.x % n_tx) * kTC;
    const int nrows = min(kTR, p.ny - r0), ncols = min(kTC, p.nx - c0);
    const int half_x = (p.nx + 1) / 2, half_y = (p.ny + 1) / 2;
    const size_t t = blockIdx.y;
    const float4* atoms = binned + t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + t * (size_t)p.n_atoms;
    const int* off = bin_off + t * (size_t)(p.n_bins + 1);
    const AxisRange rb = axis_range(r0 / p.band_h, p.band_h, p.ny, p.n_bands, p.reach_y + 1);
    const AxisRange rx = axis_range(c0 / p.ctile_w, p.ctile_w, p.nx, p.n_ctiles, p.reach_x + 1);
    const int n_nb = rb.count * rx.count, stride = 2 * n_nb + 1;
    const int chunk = kTabInts / stride;         // slabs per table load (>= 49 with n_nb <= 32)

    float acc_m[8], acc_c[8], acc_p[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc_m[i] = acc_c[i] = acc_p[i] = 0.f;

    int k0 = 0, n_staged = 0;                    // first slab of the table; sources staged for slab k
    for (int k = 0; k < p.n_slices; ++k) {
        if (k == 0 || k == k0 + chunk) {
            if (k > 0) k0 = k;
            load_bin_table(sm.tab, p, off, k0, min(chunk, p.n_slices - k0), rb, rx);
            n_staged = 0;                        // the first slab of a table is read directly
        }
        const int* bstart = sm.tab + (k - k0) * stride;
        const int* bcum = bstart + n_nb;
        const int n_src = bcum[n_nb];
        const int buf = k & 1;
        const float bm = slice_boundary(p, k - 1), b0 = slice_boundary(p, k), b1 = slice_boundary(p, k + 1),
                    b2 = slice_boundary(p, k + 2);
        const bool has_m = k >= 1, has_p = k + 1 < p.n_slices;

        for (int sb = 0; sb < n_src; sb += kPotThreads) {
            // 1. candidates among the sources [sb, sb + kPotThreads), in source order
            const int src = sb + (int)threadIdx.x;
            bool ok = false;
            float4 at = make_float4(0.f, 0.f, 0.f, 0.f);
            int2 px = make_int2(0, 0);
            int sp = 0;
            if (src < n_src) {
                if (src < n_staged) {
                    at = sm.st_at[buf][src];
                    px = sm.st_px[buf][src];
                } else {
                    const int ai = source_atom(bstart, bcum, n_nb, src);
                    at = atoms[ai];                      // (fx, fy, z, species)
                    px = atoms_px[ai];                   // (ic, jc), wrapped
                }
                sp = __float_as_int(at.w);
                ok = sp >= 0 && sp < p.n_species;
                const float rc = 6.0f * (ok ? p.sigma[sp] : 1.f);
                ok = ok && range_gap(px.y, at.y, r0, nrows, p.ny, p.dy) <= rc &&
                     range_gap(px.x, at.x, c0, ncols, p.nx, p.dx) <= rc;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (lane == 0) sm.warp_cnt[warp] = __popc(bal);
            __syncthreads();
            int n_cand = 0, my_off = 0;
#pragma unroll
            for (int w = 0; w < kTWarps; ++w) {
                const int c = sm.warp_cnt[w];
                if (w < warp) my_off += c;
                n_cand += c;
            }
            if (ok) {
                const int c = my_off + __popc(bal & lt);
                sm.k0y[c] = nearest_image(r0 - px.y, p.ny);
                sm.k0x[c] = nearest_image(c0 - px.x, p.nx);
                sm.fx[c] = at.x;
                sm.fy[c] = at.y;
                sm.z[c] = at.z;
                sm.spc[c] = sp;
            }
            if (sb == 0 && k + 1 < p.n_slices && k + 1 < k0 + chunk) {
                // stage the next slab's first sources while this one is worked on
                // (the other buffer was last read before this slab's first barrier)
                const int* nstart = bstart + stride;
                const int n1 = nstart[2 * n_nb];
                if ((int)threadIdx.x < n1) {
                    const int ai = source_atom(nstart, nstart + n_nb, n_nb, threadIdx.x);
                    cp_async_16(&sm.st_at[buf ^ 1][threadIdx.x], atoms + ai);
                    cp_async_8(&sm.st_px[buf ^ 1][threadIdx.x], atoms_px + ai);
                }
                cp_async_commit();
            }
            __syncthreads();

            for (int cb = 0; cb < n_cand; cb += kSCand) {
                const int nc = min(kSCand, n_cand - cb);
                // 2. factors, in tasks of 8 values: task (c, g) for g < 4 tabulates rows
                //    8g .. 8g + 7 of gy and erf/2 at slice boundary k - 1 + g; task (c, g)
                //    for g < 8 of the column tasks tabulates columns 8g .. 8g + 7 of gx (the
                //    columns of warp g).  Square cut-off |dx|, |dy| <= 6 s; rows and columns
                //    outside the tile are 0.  Row tasks of a candidate are 4 aligned lanes,
                //    column tasks 8 aligned lanes (column tasks start at a multiple of 8).
                const int n_rt = 4 * nc, col0 = (n_rt + 7) & ~7, n_task = col0 + 8 * nc;
                for (int ib = 0; ib < n_task; ib += kPotThreads) {
                    const int i = ib + (int)threadIdx.x;
                    const bool row_task = i < n_rt, col_task = i >= col0 && i < n_task;
                    const int c = row_task ? (i >> 2) : (col_task ? (i - col0) >> 3 : 0);
                    const int g = row_task ? (i & 3) : (i & 7);
                    const int cc = cb + c;
                    const int csp = sm.spc[cc];
                    const float c2 = p.c2[csp], rcc = p.rc[csp];
                    bool nz = false;
                    if (row_task || col_task) {
                        // rows: offsets k0y + r from the atom's pixel, limit nrows; columns alike
                        const int k0 = row_task ? sm.k0y[cc] : sm.k0x[cc];
                        const float f = row_task ? sm.fy[cc] : sm.fx[cc];
                        const int n = row_task ? p.ny : p.nx, half = row_task ? half_y : half_x;
                        const int lim = row_task ? nrows : ncols;
                        const float dd = row_task ? p.dy : p.dx;
                        float4* dst = row_task ? reinterpret_cast<float4*>(&sm.gy[c][8 * g]) : &sm.gx[c][2 * g];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            float v[4];
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const int o = 8 * g + 4 * h + r;
                                int kk = k0 + o;
                                if (kk >= half) kk -= n;
                                const float d = small_int_to_float(kk) * dd - f;
                                v[r] = (o < lim && fabsf(d) <= rcc) ? exp2f(-(d * d) * c2) : 0.f;
                                nz = nz || v[r] != 0.f;
                            }
                            dst[h] = make_float4(v[0], v[1], v[2], v[3]);
                        }
                    }
                    // erf(.)/2 at boundary k - 1 + g (open ends -1/2, +1/2), gathered per row
                    // group; only warps that hold row tasks (resp. column tasks) take part
                    const int wi0 = ib + 32 * warp;      // this warp's first task index
                    if (wi0 < n_rt) {
                        const float bj = slice_boundary(p, k - 1 + g);
                        const float zc = sm.z[cc];
                        const float e = bj == -INFINITY ? -0.5f
                                        : (bj == INFINITY ? 0.5f : 0.5f * erff((bj - zc) * p.kz[csp]));
                        const int l4 = lane & ~3;
                        const float e0 = __shfl_sync(0xffffffffu, e, l4), e1 = __shfl_sync(0xffffffffu, e, l4 + 1);
                        const float e2 = __shfl_sync(0xffffffffu, e, l4 + 2), e3 = __shfl_sync(0xffffffffu, e, l4 + 3);
                        if (row_task && g == 0) {
                            const float amp = p.amp[csp];
                            const float lo_z = zc - rcc, hi_z = zc + rcc;
                            const float wm_ = (has_m && b0 > lo_z && bm < hi_z) ? amp * (e1 - e0) : 0.f;
                            const float wc_ = (b1 > lo_z && b0 < hi_z) ? amp * (e2 - e1) : 0.f;
                            const float wp_ = (has_p && b2 > lo_z && b1 < hi_z) ? amp * (e3 - e2) : 0.f;
                            sm.w[c] = make_float4(wm_, wc_, wp_, 0.f);
                        }
                    }
                    if (wi0 + 31 >= col0 && wi0 < n_task) {
                        const unsigned nzb = __ballot_sync(0xffffffffu, col_task && nz);
                        if (col_task && g == 0) sm.wmask[c] = (int)((nzb >> (lane & 24)) & 0xffu);
                    }
                }
                __syncthreads();

                // 3. this warp's candidates, in order, then the outer-product updates of
                //    the three running slices
                bool has = lane < nc && ((sm.wmask[lane] >> warp) & 1);
                if (has) {
                    const float4 wv = sm.w[lane];
                    has = wv.x != 0.f || wv.y != 0.f || wv.z != 0.f;
                }
                const unsigned hb = __ballot_sync(0xffffffffu, has);
                if (has) sm.wlist[warp][__popc(hb & lt)] = (unsigned char)lane;
                __syncwarp();
                const int cnt = __popc(hb);
                for (int j = 0; j < cnt; ++j) {
                    const int c = sm.wlist[warp][j];
                    const float gyv = sm.gy[c][lane];
                    const float4 wv = sm.w[c];
                    const float ym = gyv * wv.x, yc = gyv * wv.y, yp = gyv * wv.z;
                    const float4 a = sm.gx[c][2 * warp], b = sm.gx[c][2 * warp + 1];
                    const float g[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        acc_m[i] = fmaf(ym, g[i], acc_m[i]);
                        acc_c[i] = fmaf(yc, g[i], acc_c[i]);
                        acc_p[i] = fmaf(yp, g[i], acc_p[i]);
                    }
                }
                // the next chunk rewrites the table; after a slab's last chunk the
                // end-of-slab barrier comes first (the next writes follow the next
                // slab's selection barriers)
                if (cb + kSCand < n_cand || sb + kPotThreads < n_src) __syncthreads();
            }
        }
        // slice k-1 has all its slabs (k-2 .. k): write it, then move the window up
        if (has_m) store_tile_row(p, V, t, k - 1, r0, c0, nrows, ncols, vec_out, acc_m);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            acc_m[i] = acc_c[i];
            acc_c[i] = acc_p[i];
            acc_p[i] = 0.f;
        }
        const bool staged_next = n_src > 0 && k + 1 < p.n_slices && k + 1 < k0 + chunk;
        if (staged_next) {
            cp_async_wait_all();
            n_staged = min(bcum[n_nb + stride], kPotThreads);
        } else {
            n_staged = 0;
        }
        __syncthreads();                                 // staged records visible; candidates reusable
    }
    store_tile_row(p, V, t, p.n_slices - 1, r0, c0, nrows, ncols, vec_out, acc_m);
}

// ------------------------------------------------------------------ forward, band walk
// Band-walking potential (6 s <= dz: an atom of slab k reaches only slices
// k-1, k and k+1).  For every (snapshot, slab, band of kBR rows) a list holds
// the slab's atoms whose window reaches the band -- per atom its row factors
// gy over the band's rows, its weights amp w_{k-1}, amp w_k, amp w_{k+1}
// (computed once per atom and snapshot by atom_weights_kernel), and its column
// and offset in the pixel -- sorted by the atom's pixel column (periodic
// images of atoms near the left and right edges as entries of their own), with
// a table of the first entry that can reach each group of 8 columns.  One block
// per (band, snapshot) then walks the slabs in order, a thread owning kB2Cols
// adjacent columns of the band running over exactly the entries whose window
// can reach them:
//   v_s(x, y) = sum over slabs k = s-1, s, s+1 (in this order), over list
//               entries in list order, of gy(y) * amp w_s * exp(-dx^2 / 2 s^2).
// List order is (column, position of the atom in the slab's bins), and the
// bins hold atoms in input order, so the order -- and so the FP32 sum -- is
// fixed by the configuration.  A slab whose list would not fit a slot is
// built in chunks of sources by the accumulating block itself.
constexpr int kBR = kBandRows;           // rows per band (the Bands bin layout)
constexpr int kB2Threads = 128;
constexpr int kB2Cols = 4;               // adjacent columns per thread
constexpr int kB2Cap = 96;               // list entries per slot
constexpr int kB2Group = 2;              // slabs built per round
constexpr int kB2Ring = kB2Group + 2;    // slots for slabs s-1 .. s+kB2Group
constexpr int kB2Chunk = kB2Ring;        // the slot for chunks of an over-full slab
constexpr int kB2Slots = kB2Ring + 1;
constexpr int kB2ChunkSrc = kB2Cap / 3;  // sources per chunk (each gives at most 3 entries)
constexpr int kBGroups = 129;            // 8-column groups for nx <= 1024, plus one
constexpr int kBFirst = 144;             // bytes of a first[] table (kBGroups rounded up to 16)
constexpr int kBMaxBins = 32;            // bands within reach of a band (one warp scans them)
constexpr int kBMaxNx = 1024;
static_assert(kB2Cap <= 255, "first[] holds list positions in a byte");
static_assert(kB2Threads * 3 <= 512, "positions in a slab's build order fit the low 9 bits of a sort key");

struct BandSmem {
    float4 hd[kB2Slots][kB2Cap];         // (column key as int bits, fx, log2(e) / (2 s^2), 6 s)
    float4 g[kB2Slots][kB2Cap][2];       // gy over the band's rows (0 outside |dy| <= 6 s)
    float4 w[kB2Slots][kB2Cap];          // amp w_{k-1}, amp w_k, amp w_{k+1}, q = exp2(-2 d^2 c2)
    __align__(16) unsigned char first[kB2Slots][kBFirst];
    int n[kB2Slots];                     // entries of the slot, or -1: slab processed in chunks
    // per slab of a round: unique sort keys (column key * 512 + position in the slab's build
    // order), padded with INT_MAX to a multiple of 4 so the ranking reads four at a time
    __align__(16) int ckey[kB2Group][kB2Threads * 3 + 4];
    int bin_start[kB2Group][kBMaxBins], bin_cum[kB2Group][kBMaxBins + 1];
    int nsrc[kB2Group];                  // sources of each slab of the round
    int lstart[kB2Group + 1];            // build positions where each slab's entries start
    int warp_tot[kB2Threads / 32];
};

// Slice weights amp w_{k-1}, amp w_k, amp w_{k+1} of every binned atom, k its
// slab (the same rounded expression as the binning), 0 for slices outside the
// stack or the 6 s window and for skipped atoms.
__global__ void atom_weights_kernel(const float4* __restrict__ binned, float4* __restrict__ wts, PotParams p,
                                    size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 at = binned[i];
    const int sp = __float_as_int(at.w);
    float w[3] = {0.f, 0.f, 0.f};
    if (sp >= 0 && sp < p.n_species) {
        int k = (int)floorf(__fmul_rn(__fsub_rn(at.z, p.z0), p.inv_dz));
        k = min(max(k, 0), p.n_slices - 1);
        const float sg = p.sigma[sp], rc = p.rc[sp], amp = p.amp[sp];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int s = k - 1 + j;
            const float lo = slice_boundary(p, s), hi = slice_boundary(p, s + 1);
            if (s >= 0 && s < p.n_slices && hi > at.z - rc && lo < at.z + rc)
                w[j] = amp * slice_weight(at.z, sg, lo, hi, s == 0, s == p.n_slices - 1, nullptr);
        }
    }
    wts[i] = make_float4(w[0], w[1], w[2], 0.f);
}

// Exclusive prefix sum of v over the block; *total receives the sum.  Ends
// with a barrier.
__device__ __forceinline__ int block_excl_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = 0, all = 0;
    for (int w = 0; w < nw; ++w) {
        const int c = warp_tot[w];
        if (w < warp) before += c;
        all += c;
    }
    *total = all;
    __syncthreads();
    return before + incl - v;
}

// Sources of slabs k0 .. k0 + nk - 1 near band `band`: warp j loads the starts
// and counts of the rb.count bins (k0 + j, band') with band' within reach and
// scans them into bin_start[j] / bin_cum[j], nsrc[j].  Ends with a barrier.
__device__ void band_bins(BandSmem& sm, const PotParams& p, const int* __restrict__ off, int k0, int nk,
                          AxisRange rb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = warp; j < nk; j += kB2Threads / 32) {
        int cnt = 0, start = 0;
        if (lane < rb.count) {
            const int bin = (k0 + j) * p.n_bands + (rb.first + lane) % p.n_bands;   // one column tile
            start = __ldg(off + bin);
            cnt = __ldg(off + bin + 1) - start;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        if (lane < rb.count) {
            sm.bin_start[j][lane] = start;
            sm.bin_cum[j][lane] = incl - cnt;
        }
        if (lane == 31) sm.nsrc[j] = incl;
    }
    __syncthreads();
}

// Lists of nk consecutive slabs k0 .. in one round (the accumulating kernel's
// chunks of an over-full slab): slab j's sources
// [src0_j, src1_j) (bin tables loaded by band_bins; the sources of all slabs
// together at most blockDim.x) into slot slot_j, each sorted by (column key,
// build position).  slot_j < 0 skips a slab.  Every slab's entry count goes to
// sm.n[slot_j], or -1 when it exceeds kB2Cap.  Ends with a barrier.
__device__ void band_build(BandSmem& sm, const PotParams& p, const float4* __restrict__ atoms,
                           const int2* __restrict__ atoms_px, const float4* __restrict__ wts, int nk,
                           const int* src0, const int* src1, const int* slot, int nbins, int r0, int nrows,
                           int kofs, int ngroups) {
    // this thread's source: slab j, source index src
    int j = -1, src = 0, before = 0;
    for (int q = 0; q < nk; ++q) {
        const int cnt = slot[q] >= 0 ? src1[q] - src0[q] : 0;
        if (j < 0 && (int)threadIdx.x < before + cnt) {
            j = q;
            src = src0[q] + ((int)threadIdx.x - before);
        }
        before += cnt;
    }
    int nkeys = 0, key[3] = {0, 0, 0};
    float fx = 0.f, c2 = 0.f, rc = 0.f, g[kBR];
    float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int r = 0; r < kBR; ++r) g[r] = 0.f;
    if (j >= 0) {
        int lo = 0, hi = nbins - 1;                      // the last bin starting at or before src
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.bin_cum[j][mid] <= src) lo = mid; else hi = mid - 1;
        }
        const int ai = sm.bin_start[j][lo] + (src - sm.bin_cum[j][lo]);
        const float4 at = atoms[ai];                     // (fx, fy, z, species)
        const int2 px = atoms_px[ai];                    // (ic, jc), wrapped
        const int sp = __float_as_int(at.w);
        bool ok = sp >= 0 && sp < p.n_species;
        if (ok) {
            rc = p.rc[sp];
            c2 = p.c2[sp];
            ok = range_gap(px.y, at.y, r0, nrows, p.ny, p.dy) <= rc;
        }
        if (ok) {
            wv = wts[ai];
            wv.w = exp2f(-2.f * (p.dx * p.dx) * c2);    // ratio of ratios of consecutive column factors
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                const int ky = nearest_image(r0 + r - px.y, p.ny);
                const float d = small_int_to_float(ky) * p.dy - at.y;
                g[r] = (r < nrows && fabsf(d) <= rc) ? exp2f(-(d * d) * c2) : 0.f;
            }
            fx = at.x;
            key[nkeys++] = px.x + kofs;
            if (px.x <= p.reach_x + 1) key[nkeys++] = px.x + p.nx + kofs;          // image to the right
            if (px.x >= p.nx - p.reach_x - 2) key[nkeys++] = px.x - p.nx + kofs;   // image to the left
        }
    }
    int total = 0;
    const int base = block_excl_scan(nkeys, sm.warp_tot, &total);
    // sources are ordered by slab, so each slab's entries are contiguous in build order
    if (j >= 0 && src == src0[j]) sm.lstart[j] = base;
    for (int q = threadIdx.x; q < nk; q += blockDim.x)
        if (slot[q] < 0 || src1[q] == src0[q]) sm.lstart[q] = -1;
    __syncthreads();
    if (threadIdx.x == 0) {                              // empty or skipped slabs start where the next one does
        int next = total;
        for (int q = nk - 1; q >= 0; --q) {
            if (sm.lstart[q] < 0) sm.lstart[q] = next;
            next = sm.lstart[q];
        }
        sm.lstart[nk] = total;
    }
    __syncthreads();
    int l0 = 0, l1 = 0;
    if (j >= 0) {
        l0 = sm.lstart[j];
        l1 = sm.lstart[j + 1];
        for (int m = 0; m < nkeys; ++m) sm.ckey[j][base + m - l0] = key[m] * 512 + (base + m - l0);
    }
    for (int t = threadIdx.x; t < 4 * nk; t += blockDim.x) {   // INT_MAX padding to a multiple of 4
        const int q = t >> 2, n = sm.lstart[q + 1] - sm.lstart[q];
        const int pos = n + (t & 3);
        if (pos < ((n + 3) & ~3)) sm.ckey[q][pos] = 0x7fffffff;
    }
    __syncthreads();
    if (j >= 0 && l1 - l0 <= kB2Cap) {
        float4* hd = sm.hd[slot[j]];
        float4 (*gs)[2] = sm.g[slot[j]];
        float4* ws = sm.w[slot[j]];
        const int4* ck4 = reinterpret_cast<const int4*>(sm.ckey[j]);
        const int n4 = (l1 - l0 + 3) >> 2;
        for (int m = 0; m < nkeys; ++m) {
            const int ck = key[m] * 512 + (base + m - l0);
            int rank = 0;
#pragma unroll 4
            for (int q = 0; q < n4; ++q) {
                const int4 v = ck4[q];
                rank += (v.x < ck) + (v.y < ck) + (v.z < ck) + (v.w < ck);
            }
            hd[rank] = make_float4(__int_as_float(key[m]), fx, c2, rc);
            gs[rank][0] = make_float4(g[0], g[1], g[2], g[3]);
            gs[rank][1] = make_float4(g[4], g[5], g[6], g[7]);
            ws[rank] = wv;
        }
    }
    __syncthreads();
    // first[c]: the first entry whose key is >= the lowest key that can reach column group c
    for (int t = threadIdx.x; t < nk * ngroups; t += blockDim.x) {
        const int q = t / ngroups, c = t - q * ngroups;
        if (slot[q] < 0) continue;
        const int n = sm.lstart[q + 1] - sm.lstart[q];
        if (n > kB2Cap) continue;
        const int want = 8 * c - p.reach_x - 1 + kofs;
        const float4* hd = sm.hd[slot[q]];
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (__float_as_int(hd[mid].x) < want) lo = mid + 1; else hi = mid;
        }
        sm.first[slot[q]][c] = (unsigned char)lo;
    }
    for (int q = threadIdx.x; q < nk; q += blockDim.x)
        if (slot[q] >= 0) {
            const int n = sm.lstart[q + 1] - sm.lstart[q];
            sm.n[slot[q]] = n <= kB2Cap ? n : -1;
        }
    __syncthreads();
}

// ------------------------------------------------------------ slab lists
// Two kernels per chunk of snapshots: potential_lists_kernel builds every
// list of the chunk at once, one warp per (snapshot, slab, band), into global
// memory (no block barriers, every warp busy), and potential_accum_kernel only
// accumulates, streaming each slab's list into its shared-memory ring two
// slabs ahead.  A list is the one band_build makes from the same sources
// (same entries, order and first[] table).
constexpr int kLWarps = 4;                     // lists per block of the list kernel
constexpr int kLFirst = 144;                   // bytes of a list's first[] table (kBGroups, padded)
static_assert(kBFirst == kLFirst && kBGroups <= kLFirst && kLFirst % 16 == 0, "first[] table size");
// one list in global memory: first[] table, then hd[], g[][2], w[] of kB2Cap entries
constexpr int kLHd = kLFirst;
constexpr int kLG = kLHd + 16 * kB2Cap;
constexpr int kLW = kLG + 32 * kB2Cap;
constexpr int kLBytes = kLW + 16 * kB2Cap;
static_assert(kLBytes % 16 == 0, "lists are 16-byte aligned");

__device__ __forceinline__ void cp_async_cg16_pot(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait_pot() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

// Source `src` of a list: the atom index, or -1.  excl/start: per-lane
// exclusive source counts and first atoms of the list's bins (lane j: bin j).
__device__ __forceinline__ int list_source_atom(int src, int nsrc, int count, int excl, int start) {
    int j = 0;
    for (int q = 1; q < count; ++q) {
        const int e = __shfl_sync(0xffffffffu, excl, q);
        if (e <= src) j = q;
    }
    const int s0 = __shfl_sync(0xffffffffu, start, j);
    const int e0 = __shfl_sync(0xffffffffu, excl, j);
    return src < nsrc ? s0 + (src - e0) : -1;
}

// The keys of source atom ai for band rows [r0, r0 + nrows): none when the
// atom is skipped or reaches none of the rows; else its column (+ kofs) and
// the images within reach of the other edge.
__device__ __forceinline__ int list_keys(const PotParams& p, const float4& at, const int2& px, int r0, int nrows,
                                         int kofs, int (&key)[3]) {
    const int sp = __float_as_int(at.w);
    if (sp < 0 || sp >= p.n_species) return 0;
    if (range_gap(px.y, at.y, r0, nrows, p.ny, p.dy) > p.rc[sp]) return 0;
    int n = 0;
    key[n++] = px.x + kofs;
    if (px.x <= p.reach_x + 1) key[n++] = px.x + p.nx + kofs;
    if (px.x >= p.nx - p.reach_x - 2) key[n++] = px.x - p.nx + kofs;
    return n;
}

// One warp per (snapshot t0 + blockIdx.z, slab blockIdx.y, band): the sources
// of the bins within reach, in bin order, each with its keys (build order);
// entries ranked by (key, build position) and written at their rank, then
// the first[] table and the entry count (n_list; -1 for a list over kB2Cap
// entries, which the accumulating kernel builds in chunks itself).
__global__ void __launch_bounds__(32 * kLWarps)
potential_lists_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                       const int2* __restrict__ binned_px, const float4* __restrict__ binned_w, PotParams p, int t0,
                       unsigned char* __restrict__ lists, int* __restrict__ n_list) {
    __shared__ __align__(16) int ckey[kLWarps][kB2Cap + 4];
    __shared__ int skey[kLWarps][kB2Cap];
    __shared__ __align__(4) unsigned char first_b[kLWarps][kLFirst];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int band = blockIdx.x * kLWarps + warp;
    if (band >= p.n_bands) return;                    // whole warps only: no block barrier below
    const int k = blockIdx.y;
    const size_t tl = blockIdx.z, t = t0 + tl;
    const float4* atoms = binned + t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + t * (size_t)p.n_atoms;
    const float4* wts = binned_w + t * (size_t)p.n_atoms;
    const int* off = bin_off + t * (size_t)(p.n_bins + 1);
    const AxisRange rb = axis_range(band, kBR, p.ny, p.n_bands, p.reach_y + 1);
    const int r0 = band * kBR, nrows = min(kBR, p.ny - r0);
    const int kofs = p.reach_x + 2;
    unsigned char* L = lists + ((tl * p.n_slices + k) * (size_t)p.n_bands + band) * kLBytes;
    int* nl = n_list + (tl * p.n_bands + band) * (size_t)p.n_slices + k;
    int start = 0, cnt = 0;
    if (lane < rb.count) {
        const int bin = k * p.n_bands + (rb.first + lane) % p.n_bands;
        start = __ldg(off + bin);
        cnt = __ldg(off + bin + 1) - start;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
    }
    const int excl = incl - cnt;
    const int nsrc = __shfl_sync(0xffffffffu, incl, 31);
    // pass 1: composite keys (key * 512 + build position) of every entry
    int total = 0;
    for (int c0 = 0; c0 < nsrc; c0 += 32) {
        const int ai = list_source_atom(c0 + lane, nsrc, rb.count, excl, start);
        int key[3], nk = 0;
        if (ai >= 0) nk = list_keys(p, __ldg(atoms + ai), __ldg(atoms_px + ai), r0, nrows, kofs, key);
        int base = nk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, base, o);
            if (lane >= o) base += u;
        }
        const int chunk = __shfl_sync(0xffffffffu, base, 31);
        base += total - nk;
        if (total + chunk <= kB2Cap)
            for (int m = 0; m < nk; ++m) ckey[warp][base + m] = key[m] * 512 + (base + m);
        total += chunk;
    }
    if (total > kB2Cap) {
        if (lane == 0) *nl = -1;
        return;
    }
    if (lane < 4 && total + lane < ((total + 3) & ~3)) ckey[warp][total + lane] = 0x7fffffff;
    __syncwarp();
    // pass 2: each entry at its rank
    float4* hd = reinterpret_cast<float4*>(L + kLHd);
    float4* gs = reinterpret_cast<float4*>(L + kLG);
    float4* ws = reinterpret_cast<float4*>(L + kLW);
    const int4* ck4 = reinterpret_cast<const int4*>(ckey[warp]);
    const int n4 = (total + 3) >> 2;
    int done = 0;
    for (int c0 = 0; c0 < nsrc; c0 += 32) {
        const int ai = list_source_atom(c0 + lane, nsrc, rb.count, excl, start);
        int key[3], nk = 0;
        float4 at = make_float4(0.f, 0.f, 0.f, 0.f);
        int2 px = make_int2(0, 0);
        if (ai >= 0) {
            at = __ldg(atoms + ai);
            px = __ldg(atoms_px + ai);
            nk = list_keys(p, at, px, r0, nrows, kofs, key);
        }
        int base = nk;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, base, o);
            if (lane >= o) base += u;
        }
        const int chunk = __shfl_sync(0xffffffffu, base, 31);
        base += done - nk;
        done += chunk;
        if (nk == 0) continue;
        const int sp = __float_as_int(at.w);
        const float c2 = p.c2[sp], rc = p.rc[sp];
        float4 wv = __ldg(wts + ai);
        wv.w = exp2f(-2.f * (p.dx * p.dx) * c2);
        float g[kBR];
#pragma unroll
        for (int r = 0; r < kBR; ++r) {
            const int ky = nearest_image(r0 + r - px.y, p.ny);
            const float d = small_int_to_float(ky) * p.dy - at.y;
            g[r] = (r < nrows && fabsf(d) <= rc) ? exp2f(-(d * d) * c2) : 0.f;
        }
        for (int m = 0; m < nk; ++m) {
            const int ck = key[m] * 512 + (base + m);
            int rank = 0;
#pragma unroll 4
            for (int q = 0; q < n4; ++q) {
                const int4 v = ck4[q];
                rank += (v.x < ck) + (v.y < ck) + (v.z < ck) + (v.w < ck);
            }
            hd[rank] = make_float4(__int_as_float(key[m]), at.x, c2, rc);
            gs[2 * rank] = make_float4(g[0], g[1], g[2], g[3]);
            gs[2 * rank + 1] = make_float4(g[4], g[5], g[6], g[7]);
            ws[rank] = wv;
            skey[warp][rank] = key[m];
        }
    }
    __syncwarp();
    // first[c]: the first entry whose key is >= want(c) = 8 c - reach_x - 1 + kofs, the lowest
    // key that can reach column group c; four groups per 32-bit word.  The keys are sorted, so
    // first[c] = i exactly for the groups with key[i - 1] < want(c) <= key[i] (key[-1] = -inf,
    // key[total] = +inf): each entry writes the groups of its gap.
    const int ngroups = (p.nx + 7) / 8;
    const int nwords = (ngroups + 3) / 4;
    const int c_last = 4 * nwords - 1;
    const int c0k = kofs - p.reach_x - 1;          // want(c) = 8 c + c0k
    unsigned char* fb = first_b[warp];
    for (int i = lane; i <= total; i += 32) {
        const int lo_key = i == 0 ? -(1 << 29) : skey[warp][i - 1];
        const int hi_key = i == total ? (1 << 29) : skey[warp][i];
        const int ca = max(((lo_key - c0k) >> 3) + 1, 0);     // want(c) > lo_key
        const int cb = min((hi_key - c0k) >> 3, c_last);      // want(c) <= hi_key
        for (int c = ca; c <= cb; ++c) fb[c] = (unsigned char)i;
    }
    __syncwarp();
    uint32_t* fw = reinterpret_cast<uint32_t*>(L);
    for (int w4 = lane; w4 < nwords; w4 += 32)
        fw[w4] = (uint32_t)fb[4 * w4] | ((uint32_t)fb[4 * w4 + 1] << 8) | ((uint32_t)fb[4 * w4 + 2] << 16) |
                 ((uint32_t)fb[4 * w4 + 3] << 24);
    if (lane == 0) *nl = total;
}

// Adds slab list `slot` to the three slices it reaches, for columns x0 ..
// x0 + kB2Cols - 1 of the band: acc_m (slice k - 1, weight w_{k-1}), acc_0
// (slice k), acc_p (slice k + 1).  Each entry's column factors
// g_m = exp2(-dx_m^2 c2) are formed once for the three slices and scaled by
// each slice's weight.  RECUR: the factors by the exact recurrence
// g_{m+1} = g_m r_m, r_{m+1} = r_m q with r_0 = exp2(-(2 dx_0 d + d^2) c2) and
// q = exp2(-2 d^2 c2) (two exponentials per entry instead of kB2Cols, a few
// ulp of rounding), used when no factor within reach underflows (the host
// checks); otherwise one exponential per factor.
template <bool RECUR>
__device__ __forceinline__ void slab_accumulate(const BandSmem& sm, int slot, int x0, int reach, int kofs, float d,
                                                float (&acc_m)[kBR][kB2Cols], float (&acc_0)[kBR][kB2Cols],
                                                float (&acc_p)[kBR][kB2Cols]) {
    const int lo = x0 - reach - 1 + kofs, hi = x0 + kB2Cols - 1 + reach + 2 + kofs;
    const int n = sm.n[slot];
    for (int i = sm.first[slot][x0 >> 3]; i < n; ++i) {
        const float4 h = sm.hd[slot][i];
        const int key = __float_as_int(h.x);
        if (key > hi) break;
        if (key < lo) continue;
        const float4 w = sm.w[slot][i];
        const int k0 = x0 + kofs - key;
        float gx[kB2Cols];
        if constexpr (RECUR) {
            const float dx0 = small_int_to_float(k0) * d - h.y;
            float g = exp2f(-(dx0 * dx0) * h.z);
            float r = exp2f(-fmaf(2.f * dx0, d, d * d) * h.z);
#pragma unroll
            for (int m = 0; m < kB2Cols; ++m) {
                const float dx = fmaf((float)m, d, dx0);
                gx[m] = fabsf(dx) <= h.w ? g : 0.f;
                g *= r;
                r *= w.w;
            }
        } else {
#pragma unroll
            for (int m = 0; m < kB2Cols; ++m) {
                const float dx = small_int_to_float(k0 + m) * d - h.y;
                gx[m] = fabsf(dx) <= h.w ? exp2f(-(dx * dx) * h.z) : 0.f;
            }
        }
        const float4 ga = sm.g[slot][i][0], gb = sm.g[slot][i][1];
        const float gy[kBR] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w};
#pragma unroll
        for (int m = 0; m < kB2Cols; ++m) {
            const float a = gx[m] * w.x, b = gx[m] * w.y, c = gx[m] * w.z;
#pragma unroll
            for (int r = 0; r < kBR; ++r) {
                acc_m[r][m] = fmaf(gy[r], a, acc_m[r][m]);
                acc_0[r][m] = fmaf(gy[r], b, acc_0[r][m]);
                acc_p[r][m] = fmaf(gy[r], c, acc_p[r][m]);
            }
        }
    }
}

// The three slices' accumulators of a thread (k - 1, k, k + 1) in memory, for
// the out-of-line path below.
struct SlabAcc { float a[3][kBR][kB2Cols]; };

// An over-full slab list (more entries than a ring slot holds): built here in
// chunks of sources by the accumulating block itself and added chunk by chunk.
// Rare, and kept out of line so that the common path's accumulators stay in
// registers; every thread of the block calls it (it has block barriers).
template <bool RECUR>
__device__ __noinline__ void slab_overfull(BandSmem& sm, const PotParams& p, const int* __restrict__ off, int k,
                                           AxisRange rb, const float4* __restrict__ atoms,
                                           const int2* __restrict__ atoms_px, const float4* __restrict__ wts,
                                           int r0, int nrows, int kofs, int ngroups, bool active, int x0,
                                           SlabAcc* acc) {
    band_bins(sm, p, off, k, 1, rb);
    const int nsrc = sm.nsrc[0];
    for (int c0 = 0; c0 < nsrc; c0 += kB2ChunkSrc) {
        const int a0 = c0, a1 = min(nsrc, c0 + kB2ChunkSrc), sl = kB2Chunk;
        band_build(sm, p, atoms, atoms_px, wts, 1, &a0, &a1, &sl, rb.count, r0, nrows, kofs, ngroups);
        if (active) slab_accumulate<RECUR>(sm, kB2Chunk, x0, p.reach_x, kofs, p.dx, acc->a[0], acc->a[1], acc->a[2]);
        __syncthreads();                             // the chunk slot is rebuilt next
    }
}

// Accumulates the band's potential slab by slab from the lists of
// potential_lists_kernel (snapshot t0 + blockIdx.y; its lists are those of
// the chunk's snapshot blockIdx.y): each thread holds its columns of three
// slices (k - 1, k, k + 1), every list entry is read once, and after slab k
// slice k - 1 is complete and stored.  Ring of kB2Ring slots, the list of slab
// k + 2 copied (cp.async, 16-byte pieces) while slab k accumulates; an
// over-full list is built in chunks here, as the band kernel does.  Dynamic
// shared memory: BandSmem, then the entry counts of the band's lists.
template <bool RECUR>
__global__ void __launch_bounds__(kB2Threads, 4)
potential_accum_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                       const int2* __restrict__ binned_px, const float4* __restrict__ binned_w, PotParams p,
                       int vec4, float* __restrict__ V, const unsigned char* __restrict__ lists,
                       const int* __restrict__ n_list, int t0) {
    extern __shared__ __align__(16) unsigned char band_smem_raw[];
    BandSmem& sm = *reinterpret_cast<BandSmem*>(band_smem_raw);
    int* n_all = reinterpret_cast<int*>(band_smem_raw + sizeof(BandSmem));
    const int band = blockIdx.x;
    const size_t tl = blockIdx.y, t = t0 + tl;
    const int r0 = band * kBR, nrows = min(kBR, p.ny - r0);
    const float4* atoms = binned + t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + t * (size_t)p.n_atoms;
    const float4* wts = binned_w + t * (size_t)p.n_atoms;
    const int* off = bin_off + t * (size_t)(p.n_bins + 1);
    const AxisRange rb = axis_range(band, kBR, p.ny, p.n_bands, p.reach_y + 1);
    const int kofs = p.reach_x + 2;
    const int ngroups = (p.nx + 7) / 8;
    constexpr int span = kB2Cols * kB2Threads;
    const int passes = (p.nx + span - 1) / span;
    const int S = p.n_slices;
    for (int k = threadIdx.x; k < S; k += blockDim.x) n_all[k] = __ldg(n_list + (tl * p.n_bands + band) * S + k);
    __syncthreads();
    // copies of slab k's list into ring slot k % kB2Ring (one commit group per call, possibly empty)
    auto fetch = [&](int k) {
        const int slot = k % kB2Ring;
        if (k < S) {
            const int n = n_all[k];
            if (threadIdx.x == 0) sm.n[slot] = n;
            if (n >= 0) {
                const unsigned char* L = lists + ((tl * S + k) * (size_t)p.n_bands + band) * kLBytes;
                const int pieces = kLFirst / 16 + 4 * n;     // first[], then hd, g (two each), w per entry
                for (int i = threadIdx.x; i < pieces; i += blockDim.x) {
                    if (i < kLFirst / 16) {
                        cp_async_cg16_pot(&sm.first[slot][16 * i], L + 16 * i);
                    } else {
                        const int e = i - kLFirst / 16;
                        if (e < n) cp_async_cg16_pot(&sm.hd[slot][e], L + kLHd + 16 * e);
                        else if (e < 3 * n) cp_async_cg16_pot(reinterpret_cast<float4*>(sm.g[slot]) + (e - n),
                                                               L + kLG + 16 * (e - n));
                        else cp_async_cg16_pot(&sm.w[slot][e - 3 * n], L + kLW + 16 * (e - 3 * n));
                    }
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    auto store = [&](int si, int x0, const float (&acc)[kBR][kB2Cols]) {
        float* out = V + ((t * S + si) * (size_t)p.ny + r0) * p.nx + x0;
#pragma unroll
        for (int r = 0; r < kBR; ++r) {
            if (r < nrows) {
                float* o = out + (size_t)r * p.nx;
                if (vec4) {
                    *reinterpret_cast<float4*>(o) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
                } else {
#pragma unroll
                    for (int m = 0; m < kB2Cols; ++m)
                        if (x0 + m < p.nx) o[m] = acc[r][m];
                }
            }
        }
    };
    for (int pass = 0; pass < passes; ++pass) {
        const int x0 = kB2Cols * ((int)threadIdx.x + pass * kB2Threads);
        const bool active = x0 < p.nx;
        // slice s accumulates in acc[s % 3]: slab k adds to acc[(k + 2) % 3] (slice k - 1),
        // acc[k % 3] (slice k) and acc[(k + 1) % 3] (slice k + 1); after slab k slice k - 1 is
        // stored and its array restarts as slice k + 2.  The slab loop is unrolled by three so
        // that the arrays' roles rotate without copies.
        float acc0[kBR][kB2Cols], acc1[kBR][kB2Cols], acc2[kBR][kB2Cols];
#pragma unroll
        for (int r = 0; r < kBR; ++r)
#pragma unroll
            for (int m = 0; m < kB2Cols; ++m) acc0[r][m] = acc1[r][m] = acc2[r][m] = 0.f;
        fetch(0);
        fetch(1);
        auto slab = [&](int k, float (&acc_m)[kBR][kB2Cols], float (&acc_0)[kBR][kB2Cols],
                        float (&acc_p)[kBR][kB2Cols]) {
            fetch(k + 2);
            cp_async_wait_pot<2>();                      // slab k has landed
            __syncthreads();
            const int slot = k % kB2Ring;
            if (sm.n[slot] >= 0) {
                if (active) slab_accumulate<RECUR>(sm, slot, x0, p.reach_x, kofs, p.dx, acc_m, acc_0, acc_p);
            } else {
                SlabAcc t;
#pragma unroll
                for (int r = 0; r < kBR; ++r)
#pragma unroll
                    for (int m = 0; m < kB2Cols; ++m) {
                        t.a[0][r][m] = acc_m[r][m];
                        t.a[1][r][m] = acc_0[r][m];
                        t.a[2][r][m] = acc_p[r][m];
                    }
                slab_overfull<RECUR>(sm, p, off, k, rb, atoms, atoms_px, wts, r0, nrows, kofs, ngroups, active, x0,
                                     &t);
#pragma unroll
                for (int r = 0; r < kBR; ++r)
#pragma unroll
                    for (int m = 0; m < kB2Cols; ++m) {
                        acc_m[r][m] = t.a[0][r][m];
                        acc_0[r][m] = t.a[1][r][m];
                        acc_p[r][m] = t.a[2][r][m];
                    }
            }
            if (active && k > 0) store(k - 1, x0, acc_m);     // slice k - 1 has all its slabs
#pragma unroll
            for (int r = 0; r < kBR; ++r)
#pragma unroll
                for (int m = 0; m < kB2Cols; ++m) acc_m[r][m] = 0.f;
        };
        for (int k = 0; k < S; k += 3) {
            slab(k, acc2, acc0, acc1);
            if (k + 1 < S) slab(k + 1, acc0, acc1, acc2);
            if (k + 2 < S) slab(k + 2, acc1, acc2, acc0);
        }
        if (active) {                                    // slice S - 1: its slabs S - 2 and S - 1 added
            const int last = (S - 1) % 3;
            if (last == 0) store(S - 1, x0, acc0);
            else if (last == 1) store(S - 1, x0, acc1);
            else store(S - 1, x0, acc2);
        }
        cp_async_wait_pot<0>();
        __syncthreads();                                 // the ring is refilled by the next pass
    }
}

// ------------------------------------------------------------------ adjoint
// Candidate atoms of one block of the adjoint kernel, gathered per chunk of
// source atoms.
constexpr int kChunk = kPotThreads;      // source atoms examined per chunk
constexpr int kSegs = kPotThreads / 32;  // one column segment per warp

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

// Candidates of one chunk of source atoms: the atoms that reach this slice
// and band, listed in every column segment their window touches, with their
// per-row Gaussian factors.  Ends with a block barrier.
__device__ void gather_chunk(CandSmem& sm, const PotParams& p, const float4* __restrict__ atoms,
                             const int2* __restrict__ atoms_px, const Tile& tl, int c0, int n_src, int n_nb) {
    if (threadIdx.x < kSegs) sm.seg_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) sm.n_cand = 0;
    __syncthreads();
    const int src = c0 + threadIdx.x;
    if (src < n_src) {
        const int ai = source_atom(sm.bin_start, sm.bin_cum, n_nb, src);
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
            float dw_ds;
            const float w = slice_weight(at.z, sg, tl.lo, tl.hi, tl.first, tl.lastsl, &dw_ds);
            const int c = atomicAdd(&sm.n_cand, 1);
            const int icw = ic, jcw = jc;           // binned pixel indices are wrapped into the box
            sm.ic[c] = icw;
            sm.jc[c] = jcw;
            sm.fx[c] = at.x;
            sm.fy[c] = at.y;
            sm.sp[c] = sp;
            sm.w[c] = w;
            sm.dw[c] = dw_ds;
            sm.aw[c] = p.amp[sp] * w;
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

// Adjoint of the potential for the per-species Gaussian parameters: with
// P = exp(-rho^2 / 2 s^2) inside the cut-off and g = dL/dv,
//   dL/d amp += g P w,   dL/d s += g amp P (rho^2 / s^3 w + dw/ds).
// Each lane sums its contributions per candidate, the warp reduces them, and
// lane 0 adds the candidate's two terms (FP32 products, amp applied at the
// end) into its warp's per-species sums in shared memory, compensated
// (Kahan) so that they carry FP32 rounding per term only, not per addition.
// At the end the block adds its warps' sums in FP64 in warp order and writes
// its totals to `partial` [block][n_species][2] for a fixed-order final
// reduction.
template <int CPL>
__global__ void __launch_bounds__(kPotThreads)
potential_backward_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned,
                          const int2* __restrict__ binned_px, PotParams p, const float* __restrict__ dV,
                          double* __restrict__ partial) {
    __shared__ CandSmem sm;
    __shared__ float wsum[kPotThreads / 32][TACAW_MAX_SPECIES][2][2];   // per warp: (sum, compensation)
    extern __shared__ float gtile[];                // [kBandRows][nx]: dL/dv of the band
    const Tile tl = make_tile(p);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float4* atoms = binned + tl.t * (size_t)p.n_atoms;
    const int2* atoms_px = binned_px + tl.t * (size_t)p.n_atoms;
    for (int i = threadIdx.x; i < (kPotThreads / 32) * TACAW_MAX_SPECIES * 4; i += blockDim.x)
        (&wsum[0][0][0][0])[i] = 0.f;
    const float* grow = dV + ((tl.t * p.n_slices + tl.s) * (size_t)p.ny + tl.r0) * p.nx;
    for (int i = threadIdx.x; i < tl.nrows * p.nx; i += blockDim.x)
        gtile[i] = __ldg(grow + i);
    int n_nb;
    const int n_src = load_bins(sm.bin_start, sm.bin_cum, p, bin_off + tl.t * (size_t)(p.n_bins + 1), tl.s,
                                tl.band, 0, &n_nb);
    const int col0 = warp * tl.seg_w;
    const int col1 = min(col0 + tl.seg_w, p.nx);

    for (int c0 = 0; c0 < n_src; c0 += kChunk) {
        gather_chunk(sm, p, atoms, atoms_px, tl, c0, n_src, n_nb);
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
                const float term[2] = {ga * w, fmaf(gs * w, inv_s3, ga * dw)};
#pragma unroll
                for (int q = 0; q < 2; ++q) {           // compensated running sums
                    float* acc = wsum[warp][sp][q];
                    const float y = term[q] - acc[1];
                    const float tsum = acc[0] + y;
                    acc[1] = (tsum - acc[0]) - y;
                    acc[0] = tsum;
                }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const size_t blk = ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    if (threadIdx.x < 2 * p.n_species) {
        const int sp = threadIdx.x / 2, q = threadIdx.x % 2;
        double total = 0.0;
        for (int wi = 0; wi < kPotThreads / 32; ++wi)
            total += (double)wsum[wi][sp][q][0] - (double)wsum[wi][sp][q][1];
        partial[blk * 2 * p.n_species + threadIdx.x] = q == 0 ? total : (double)p.amp[sp] * total;
    }
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

// Bin shapes: the forward kernel bins by (slab, 32-row band, 64-column tile),
// coarsened along x, then y, while the histogram would exceed kMaxBinInts;
// the adjoint bins by (slab, 8-row band).
enum class BinLayout { Tiles, Bands };

struct BinShape {
    int band_h, ctile_w, n_bands, n_ctiles;
    long long n_bins;
};

BinShape bin_shape(const tacaw_grid& g, BinLayout lay) {
    BinShape b;
    b.band_h = lay == BinLayout::Tiles ? kTR : kBandRows;
    b.ctile_w = lay == BinLayout::Tiles ? kTC : g.nx;
    for (;;) {
        b.n_bands = (g.ny + b.band_h - 1) / b.band_h;
        b.n_ctiles = (g.nx + b.ctile_w - 1) / b.ctile_w;
        b.n_bins = (long long)g.n_slices * b.n_bands * b.n_ctiles;
        if (b.n_bins <= kMaxBinInts || lay == BinLayout::Bands) break;
        if (b.ctile_w < g.nx) b.ctile_w *= 2;
        else if (b.band_h < g.ny) b.band_h *= 2;
        else break;
    }
    return b;
}

int make_params(const tacaw_grid& g, int n_atoms, int n_species, const float* amp_sigma, BinLayout lay,
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
        const float sg = p->sigma[i];
        p->c2[i] = 1.4426950408889634f * (0.5f / (sg * sg));
        p->rc[i] = 6.0f * sg;
        p->kz[i] = 0.70710678118654752f / sg;
        smax = fmaxf(smax, amp_sigma[2 * i + 1]);
    }
    for (int i = n_species; i < TACAW_MAX_SPECIES; ++i) p->amp[i] = p->sigma[i] = p->c2[i] = p->rc[i] = p->kz[i] = 0.f;
    TACAW_REQUIRE(g.nx <= 65535 && g.ny <= 65535, TACAW_EUNSUPPORTED,
                  "tacaw_potential: nx and ny must be at most 65535");
    const double rc = 6.0 * smax;
    TACAW_REQUIRE(2.0 * rc < g.lx && 2.0 * rc < g.ly, TACAW_EINVAL,
                  "tacaw_potential: cut-off 6 sigma = %g A must be below half the box", rc);
    const BinShape b = bin_shape(g, lay);
    TACAW_REQUIRE(b.n_bins <= kMaxBinInts, TACAW_EUNSUPPORTED,
                  "tacaw_potential: %lld bins exceed the shared-memory histogram (too many slices)",
                  b.n_bins);
    p->nx = g.nx;
    p->ny = g.ny;
    p->n_slices = g.n_slices;
    p->n_atoms = n_atoms;
    p->n_species = n_species;
    p->band_h = b.band_h;
    p->ctile_w = b.ctile_w;
    p->n_bands = b.n_bands;
    p->n_ctiles = b.n_ctiles;
    p->n_bins = (int)b.n_bins;
    const double dx = g.lx / g.nx, dy = g.ly / g.ny;
    // an atom in pixel (ic, jc) reaches columns ic - reach_x - 1 .. ic + reach_x + 1 (rows
    // alike); the slab is assigned in float, so its reach gets a little slack
    p->reach_x = (int)ceil(rc / dx);
    p->reach_y = (int)ceil(rc / dy);
    p->nb_max = p->nc_max = 0;
    for (int b = 0; b < p->n_bands; ++b) {
        const int c = axis_range(b, p->band_h, g.ny, p->n_bands, p->reach_y + 1).count;
        p->nb_max = c > p->nb_max ? c : p->nb_max;
    }
    for (int b = 0; b < p->n_ctiles; ++b) {
        const int c = axis_range(b, p->ctile_w, g.nx, p->n_ctiles, p->reach_x + 1).count;
        p->nc_max = c > p->nc_max ? c : p->nc_max;
    }
    p->slab_reach = (int)ceil((rc + 1e-4 * g.dz) / g.dz);
    p->lx = (float)g.lx;
    p->ly = (float)g.ly;
    p->dx = (float)dx;
    p->inv_dx = (float)(g.nx / g.lx);
    p->dy = (float)dy;
    p->dx_d = dx;
    p->dy_d = dy;
    p->inv_dx_d = g.nx / g.lx;
    p->inv_dy_d = g.ny / g.ly;
    p->z0 = (float)g.z0;
    p->dz = (float)g.dz;
    p->inv_dz = (float)(1.0 / g.dz);
    const int n_nb = p->nb_max * p->nc_max * (min(g.n_slices - 1, 2 * p->slab_reach) + 1);
    TACAW_REQUIRE(n_nb <= kMaxNbBins, TACAW_EUNSUPPORTED,
                  "tacaw_potential: %d neighbouring bins per tile exceed %d (widths too large for "
                  "the slice thickness or pixel size)", n_nb, kMaxNbBins);
    return TACAW_OK;
}

}  // namespace

static size_t pot_backward_blocks(const tacaw_grid& g, int n_t) {
    return (size_t)((g.ny + kBandRows - 1) / kBandRows) * g.n_slices * n_t;
}

static long long clamp_bins(long long n) { return n < kMaxBinInts ? n : kMaxBinInts; }

int potential_backward_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, int n_species, size_t* bytes) {
    Carver cv(nullptr);
    carve_pot(cv, n_t, n_atoms, (int)clamp_bins(bin_shape(g, BinLayout::Bands).n_bins));
    cv.take<double>(pot_backward_blocks(g, n_t) * 2 * n_species);
    *bytes = cv.bytes();
    return TACAW_OK;
}

// Snapshots whose slab lists are built at once: lists of about kListChunkBytes.
constexpr double kListChunkBytes = 2.5e9;

static int list_chunk(const tacaw_grid& g, int n_t) {
    const double per = (double)g.n_slices * ((g.ny + kBR - 1) / kBR) * (kLBytes + sizeof(int));
    const double c = floor(kListChunkBytes / per);
    const int chunk = c < 1.0 ? 1 : (c > n_t ? n_t : (int)c);
    return chunk < 1 ? 1 : chunk;
}

int potential_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, size_t* bytes) {
    Carver cv(nullptr);
    const long long bins = std::max(clamp_bins(bin_shape(g, BinLayout::Tiles).n_bins),
                                    clamp_bins(bin_shape(g, BinLayout::Bands).n_bins));
    carve_pot(cv, n_t, n_atoms, (int)bins);
    cv.take<float4>((size_t)n_t * n_atoms);              // per-atom slice weights (band-walking kernels)
    const size_t lists = (size_t)list_chunk(g, n_t) * g.n_slices * ((g.ny + kBR - 1) / kBR);
    cv.take<unsigned char>(lists * kLBytes);             // slab lists of one chunk of snapshots
    cv.take<int>(lists);                                 // their entry counts
    *bytes = cv.bytes();
    return TACAW_OK;
}

// Parameters of the band-walking kernel, if it applies: every species has
// 6 s <= dz (atoms reach only the neighbouring slices), the bands within
// reach of a band fit one warp's scan, and nx <= kBMaxNx.
static bool band_params(const tacaw_grid& g, int n_atoms, int n_species, const float* amp_sigma, PotParams* p) {
    if (g.nx > kBMaxNx) return false;
    if (make_params(g, n_atoms, n_species, amp_sigma, BinLayout::Bands, p) != TACAW_OK) {
        clear_error();
        return false;
    }
    return p->slab_reach <= 1 && p->n_ctiles == 1 && p->band_h == kBR && p->nb_max <= kBMaxBins;
}

static int run_binning(const PotParams& p, int n_t, const float* pos, const int* species, PotWs& w,
                       cudaStream_t st) {
    const size_t bin_smem = (size_t)p.n_bins * sizeof(int);
    TACAW_CUDA_CHECK(ensure_smem((const void*)bin_kernel, (int)bin_smem));
    bin_kernel<<<n_t, kBinThreads, bin_smem, st>>>(pos, species, p, w.bin_off, w.binned, w.binned_px);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

static int check_launch_dims(const tacaw_grid& g, int n_t) {
    TACAW_REQUIRE(g.n_slices <= 65535 && n_t <= 65535, TACAW_EUNSUPPORTED,
                  "tacaw_potential: at most 65535 slices and 65535 snapshots per call");
    return TACAW_OK;
}

int potential_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos, const int* species,
                  int n_species, const float* amp_sigma, float* V, void* ws, cudaStream_t st) {
    PotParams p;
    int rc = make_params(g, n_atoms, n_species, amp_sigma, BinLayout::Tiles, &p);
    if (rc == TACAW_OK) rc = check_launch_dims(g, n_t);
    if (rc != TACAW_OK) return rc;
    PotParams pb;
    if (band_params(g, n_atoms, n_species, amp_sigma, &pb)) {
        // atoms reach at most the neighbouring slices: walk the slices once per band of rows
        Carver cv(ws);
        PotWs w = carve_pot(cv, n_t, n_atoms, pb.n_bins);
        float4* wts = cv.take<float4>((size_t)n_t * n_atoms);
        rc = run_binning(pb, n_t, pos, species, w, st);
        if (rc != TACAW_OK) return rc;
        const size_t n_rec = (size_t)n_t * n_atoms;
        if (n_rec > 0) {
            atom_weights_kernel<<<(unsigned)((n_rec + 255) / 256), 256, 0, st>>>(w.binned, wts, pb, n_rec);
            TACAW_LAUNCH_CHECK();
        }
        const int vec4 = (g.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(V) % 16 == 0);
        // the column-factor recurrence needs every factor within reach of a thread's columns to stay a
        // normal float: exponent (6 s + kB2Cols d)^2 log2(e) / (2 s^2) below 120 for every species
        bool recur = true;
        for (int i = 0; i < n_species; ++i) {
            const double sg = amp_sigma[2 * i + 1], reach = 6.0 * sg + kB2Cols * (g.lx / g.nx);
            recur = recur && reach * reach * 1.4426950408889634 / (2.0 * sg * sg) < 120.0;
        }
        const int asm_bytes = (int)(sizeof(BandSmem) + (size_t)g.n_slices * sizeof(int));
        const void* accum = recur ? (const void*)potential_accum_kernel<true> : (const void*)potential_accum_kernel<false>;
        TACAW_CUDA_CHECK(ensure_smem(accum, asm_bytes));
        // snapshots per chunk: as many as the list budget allows, rounded down to whole waves of
        // resident accumulating blocks (one block per band and snapshot) where that leaves any
        int chunk = list_chunk(g, n_t);
        int resident = 0;
        TACAW_CUDA_CHECK(resident_blocks(accum, kB2Threads, asm_bytes, &resident));
        if (resident > 0 && chunk < n_t) {
            const long long waves = (long long)chunk * pb.n_bands / resident;
            if (waves >= 1) chunk = (int)(waves * resident / pb.n_bands);
        }
        const size_t n_lists = (size_t)chunk * g.n_slices * pb.n_bands;
        unsigned char* lists = cv.take<unsigned char>(n_lists * kLBytes);
        int* n_list = cv.take<int>(n_lists);
        for (int t0 = 0; t0 < n_t; t0 += chunk) {
            const int nc = n_t - t0 < chunk ? n_t - t0 : chunk;
            potential_lists_kernel<<<dim3((pb.n_bands + kLWarps - 1) / kLWarps, g.n_slices, nc), 32 * kLWarps, 0,
                                     st>>>(w.bin_off, w.binned, w.binned_px, wts, pb, t0, lists, n_list);
            TACAW_LAUNCH_CHECK();
            if (recur)
                potential_accum_kernel<true><<<dim3(pb.n_bands, nc), kB2Threads, asm_bytes, st>>>(
                    w.bin_off, w.binned, w.binned_px, wts, pb, vec4, V, lists, n_list, t0);
            else
                potential_accum_kernel<false><<<dim3(pb.n_bands, nc), kB2Threads, asm_bytes, st>>>(
                    w.bin_off, w.binned, w.binned_px, wts, pb, vec4, V, lists, n_list, t0);
            TACAW_LAUNCH_CHECK();
        }
        return TACAW_OK;
    }
    Carver cv(ws);
    PotWs w = carve_pot(cv, n_t, n_atoms, p.n_bins);
    rc = run_binning(p, n_t, pos, species, w, st);
    if (rc != TACAW_OK) return rc;
    const int n_tx = (g.nx + kTC - 1) / kTC, n_ty = (g.ny + kTR - 1) / kTR;
    const int vec_out = (g.nx % 4 == 0) && (reinterpret_cast<uintptr_t>(V) % 16 == 0);
    if (p.slab_reach <= 1 && p.nb_max * p.nc_max <= kSBins) {
        // atoms reach at most the neighbouring slices: walk the slabs once per tile
        const int ssm = (int)sizeof(SlabSmem);
        TACAW_CUDA_CHECK(ensure_smem((const void*)potential_slab_kernel, ssm));
        potential_slab_kernel<<<dim3(n_tx * n_ty, n_t), kPotThreads, ssm, st>>>(w.bin_off, w.binned, w.binned_px,
                                                                              p, n_tx, vec_out, V);
        TACAW_LAUNCH_CHECK();
        return TACAW_OK;
    }
    const int smem = (int)sizeof(TileSmem);
    TACAW_CUDA_CHECK(ensure_smem((const void*)potential_tile_kernel, smem));
    potential_tile_kernel<<<dim3(n_tx * n_ty, g.n_slices, n_t), kPotThreads, smem, st>>>(
        w.bin_off, w.binned, w.binned_px, p, n_tx, vec_out, V);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

int potential_backward_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos,
                           const int* species, int n_species, const float* amp_sigma, const float* dV,
                           double* grad, void* ws, cudaStream_t st) {
    PotParams p;
    int rc = make_params(g, n_atoms, n_species, amp_sigma, BinLayout::Bands, &p);
    if (rc == TACAW_OK) rc = check_launch_dims(g, n_t);
    if (rc == TACAW_OK)
        TACAW_REQUIRE(g.nx <= 4 * 32 * kSegs, TACAW_EUNSUPPORTED,
                      "tacaw_potential_backward: nx = %d above the supported %d", g.nx, 4 * 32 * kSegs);
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
