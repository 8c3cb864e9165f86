// Slice-potential builder: Gaussian atoms projected onto the grid and split
// over slices (the scattering potential of a configuration that the
// multislice step of the paper's procedure propagates through).
//
//   v_s(r) = sum_a amp_a exp(-|r - R_a|^2 / (2 s_a^2)) w_s(z_a)
//   w_s(z) = (erf((z_{s+1} - z)/(sqrt2 s)) - erf((z_s - z)/(sqrt2 s))) / 2
//
// Laterally the Gaussian is cut at rho <= 6 s with the minimum periodic image;
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
constexpr float kFixScale = 4294967296.0f;            // 2^32
constexpr float kFixInv = 2.3283064365386963e-10f;    // 2^-32

struct PotParams {
    int nx, ny, n_slices, n_atoms, n_species;
    int n_bands, n_bins, slab_reach, band_reach;
    float lx, ly, dx, dy, inv_dx, inv_ly, z0, dz, inv_dz, inv_band_h;
    float amp[TACAW_MAX_SPECIES], sigma[TACAW_MAX_SPECIES];
};

// The bin is computed twice per atom (count, then scatter); explicit
// round-to-nearest operations keep the compiler from contracting the two
// copies differently, so both passes always agree.
__device__ __forceinline__ int atom_bin(float y, float z, const PotParams& p) {
    const float yw = __fsub_rn(y, __fmul_rn(floorf(__fmul_rn(y, p.inv_ly)), p.ly));
    int band = (int)floorf(__fmul_rn(yw, p.inv_band_h));
    band = min(max(band, 0), p.n_bands - 1);
    int slab = (int)floorf(__fmul_rn(__fsub_rn(z, p.z0), p.inv_dz));
    slab = min(max(slab, 0), p.n_slices - 1);
    return slab * p.n_bands + band;
}

__global__ void __launch_bounds__(kBinThreads)
bin_kernel(const float* __restrict__ pos, const int* __restrict__ species, PotParams p,
           int* __restrict__ bin_off, float4* __restrict__ binned) {
    extern __shared__ int cnt[];
    __shared__ int warp_off[kBinThreads / 32];
    const size_t t = blockIdx.x;
    const float* P = pos + t * (size_t)p.n_atoms * 3;
    for (int b = threadIdx.x; b < p.n_bins; b += blockDim.x) cnt[b] = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < p.n_atoms; a += blockDim.x)
        atomicAdd(&cnt[atom_bin(P[3 * a + 1], P[3 * a + 2], p)], 1);
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
    for (int a = threadIdx.x; a < p.n_atoms; a += blockDim.x) {
        const float x = P[3 * a], y = P[3 * a + 1], z = P[3 * a + 2];
        const int slot = atomicAdd(&cnt[atom_bin(y, z, p)], 1);
        out[slot] = make_float4(x, y, z, __int_as_float(__ldg(species + a)));
    }
}

__global__ void __launch_bounds__(kPotThreads)
potential_kernel(const int* __restrict__ bin_off, const float4* __restrict__ binned, PotParams p,
                 float* __restrict__ V) {
    extern __shared__ unsigned long long acc[];
    const int band = blockIdx.x, s = blockIdx.y;
    const size_t t = blockIdx.z;
    const int r0 = band * kBandRows;
    const int nrows = min(kBandRows, p.ny - r0);
    for (int i = threadIdx.x; i < kBandRows * p.nx; i += blockDim.x) acc[i] = 0ull;
    __syncthreads();

    const int* off = bin_off + t * (size_t)(p.n_bins + 1);
    const float4* atoms = binned + t * (size_t)p.n_atoms;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const bool first = (s == 0), lastsl = (s == p.n_slices - 1);
    const float lo = first ? -INFINITY : p.z0 + (float)s * p.dz;
    const float hi = lastsl ? INFINITY : p.z0 + (float)(s + 1) * p.dz;
    const int slab0 = max(0, s - p.slab_reach), slab1 = min(p.n_slices - 1, s + p.slab_reach);
    const bool all_bands = 2 * p.band_reach + 1 >= p.n_bands;
    const int nb = all_bands ? p.n_bands : 2 * p.band_reach + 1;

    for (int slab = slab0; slab <= slab1; ++slab) {
        for (int k = 0; k < nb; ++k) {
            int b = all_bands ? k : band - p.band_reach + k;
            b = ((b % p.n_bands) + p.n_bands) % p.n_bands;
            const int bin = slab * p.n_bands + b;
            const int a1 = off[bin + 1];
            for (int a = off[bin] + warp; a < a1; a += nwarps) {
                const float4 at = atoms[a];
                const int sp = __float_as_int(at.w);
                if (sp < 0 || sp >= p.n_species) continue;
                const float sg = p.sigma[sp];
                const float rc = 6.0f * sg;
                if (!(hi > at.z - rc && lo < at.z + rc)) continue;
                const float kz = 0.70710678118654752f / sg;
                const float fh = lastsl ? 0.5f : 0.5f * erff((hi - at.z) * kz);
                const float fl = first ? -0.5f : 0.5f * erff((lo - at.z) * kz);
                const float aw = p.amp[sp] * (fh - fl);
                const float inv2s2 = 0.5f / (sg * sg);
                const float rc2 = rc * rc;
                // one spare column on each side: the disc test below decides
                const int i0 = (int)ceilf((at.x - rc) * p.inv_dx) - 1;
                const int wx = (int)floorf(2.0f * rc * p.inv_dx) + 3;
                for (int row = 0; row < nrows; ++row) {
                    float ddy = (float)(r0 + row) * p.dy - at.y;
                    ddy -= p.ly * rintf(ddy * p.inv_ly);
                    const float ddy2 = ddy * ddy;
                    if (ddy2 > rc2) continue;
                    for (int ii = lane; ii < wx; ii += 32) {
                        const int i = i0 + ii;
                        const float ddx = (float)i * p.dx - at.x;
                        const float r2 = ddx * ddx + ddy2;
                        if (r2 <= rc2) {
                            const float c = aw * expf(-r2 * inv2s2);
                            const long long f = __float2ll_rn(c * kFixScale);
                            int iw = i % p.nx;
                            if (iw < 0) iw += p.nx;
                            atomicAdd(&acc[row * p.nx + iw], (unsigned long long)f);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    float* out = V + ((t * p.n_slices + s) * (size_t)p.ny + r0) * p.nx;
    for (int i = threadIdx.x; i < nrows * p.nx; i += blockDim.x)
        out[i] = __ll2float_rn((long long)acc[i]) * kFixInv;
}

struct PotWs {
    int* bin_off;
    float4* binned;
};

PotWs carve_pot(Carver& cv, int n_t, int n_atoms, int n_bins) {
    PotWs w;
    w.bin_off = cv.take<int>((size_t)n_t * (n_bins + 1));
    w.binned = cv.take<float4>((size_t)n_t * n_atoms);
    return w;
}

int make_params(const tacaw_grid& g, int n_atoms, int n_species, const float* amp_sigma,
                PotParams* p) {
    float smax = 0.f;
    for (int i = 0; i < n_species; ++i) {
        TACAW_REQUIRE(amp_sigma[2 * i + 1] > 0.f && isfinite(amp_sigma[2 * i + 1]) &&
                          isfinite(amp_sigma[2 * i]),
                      TACAW_EINVAL, "tacaw_potential: species %d has a bad amplitude/width", i);
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
    p->band_reach = (int)ceil(rc / (kBandRows * dy));
    p->slab_reach = (int)ceil(rc / g.dz);
    p->lx = (float)g.lx;
    p->ly = (float)g.ly;
    p->dx = (float)(g.lx / g.nx);
    p->dy = (float)dy;
    p->inv_dx = (float)(g.nx / g.lx);
    p->inv_ly = (float)(1.0 / g.ly);
    p->z0 = (float)g.z0;
    p->dz = (float)g.dz;
    p->inv_dz = (float)(1.0 / g.dz);
    p->inv_band_h = (float)(1.0 / (kBandRows * dy));
    return TACAW_OK;
}

}  // namespace

int potential_ws_bytes(const tacaw_grid& g, int n_t, int n_atoms, size_t* bytes) {
    const int n_bins = g.n_slices * ((g.ny + kBandRows - 1) / kBandRows);
    Carver cv(nullptr);
    carve_pot(cv, n_t, n_atoms, n_bins);
    *bytes = cv.bytes();
    return TACAW_OK;
}

int potential_run(const tacaw_grid& g, int n_t, int n_atoms, const float* pos, const int* species,
                  int n_species, const float* amp_sigma, float* V, void* ws, cudaStream_t st) {
    PotParams p;
    int rc = make_params(g, n_atoms, n_species, amp_sigma, &p);
    if (rc != TACAW_OK) return rc;
    const size_t bin_smem = (size_t)p.n_bins * sizeof(int);
    TACAW_REQUIRE(bin_smem <= 200 * 1024, TACAW_EUNSUPPORTED,
                  "tacaw_potential: %d bins exceed the shared-memory histogram", p.n_bins);
    const size_t pot_smem = (size_t)kBandRows * g.nx * sizeof(unsigned long long);
    TACAW_REQUIRE(pot_smem <= 200 * 1024, TACAW_EUNSUPPORTED,
                  "tacaw_potential: nx = %d too large for the band accumulator", g.nx);
    Carver cv(ws);
    PotWs w = carve_pot(cv, n_t, n_atoms, p.n_bins);
    TACAW_CUDA_CHECK(cudaFuncSetAttribute(bin_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)bin_smem));
    TACAW_CUDA_CHECK(cudaFuncSetAttribute(potential_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pot_smem));
    bin_kernel<<<n_t, kBinThreads, bin_smem, st>>>(pos, species, p, w.bin_off, w.binned);
    TACAW_LAUNCH_CHECK();
    dim3 grid(p.n_bands, g.n_slices, n_t);
    potential_kernel<<<grid, kPotThreads, pot_smem, st>>>(w.bin_off, w.binned, p, V);
    TACAW_LAUNCH_CHECK();
    return TACAW_OK;
}

}  // namespace tacaw
