// tacaw_multislice_static: the multislice of tacaw_multislice with its
// scratch in a fixed device array of this library instead of a caller
// workspace, for callers that cannot allocate device memory at all -- for
// example a plug-in whose host application owns every device allocation,
// or a real-time service that forbids allocation after start-up -- and so
// can neither call cudaMalloc nor hand over a workspace buffer.
//
// The scratch holds only the per-call tables of the slice step (twiddles,
// separable propagator factors, band-limit extents): 37120 bytes for the
// largest supported grid, 1024 x 1024 (four 8192-byte float2 tables and
// 1025 ints, each table starting on a 256-byte boundary), so
// kStaticScratchBytes = 64 KiB covers every supported size.  Every GPU that
// loads the library keeps this array until the process exits.

#include "common.cuh"

namespace tacaw {

size_t multislice_ws_bytes(const tacaw_grid& g);
int multislice_run(const tacaw_grid& g, int n_t, const float* V, const float2* psi_in,
                   float2* psi_q, double2* psi_sum, void* ws, cudaStream_t st, int flags);
bool multislice_size_supported(int n);

namespace {

constexpr size_t kStaticScratchBytes = 64 * 1024;
constexpr size_t kLargestTablesBytes = 37120;   // multislice_ws_bytes at 1024 x 1024
static_assert(kLargestTablesBytes <= kStaticScratchBytes, "the fixed scratch must hold the largest grid's tables");

// One shared scratch block per device.  All calls on a device reuse it, so
// two calls whose kernels overlap on the GPU (different streams, or graphs
// replayed concurrently) overwrite each other's tables and race.
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// In host code g_static_scratch names a host-side shadow, not device memory.
// Its device address belongs to the current CUDA context; device_symbol looks
// it up with that context current and caches it under the context's unique
// id, so a context made after a device reset is looked up afresh.
int static_scratch(void** out) {
    return device_symbol((const void*)g_static_scratch, out, "tacaw_multislice_static");
}

}  // namespace
}  // namespace tacaw

using namespace tacaw;

extern "C" int tacaw_multislice_static(const tacaw_grid* grid, int32_t n_t, const float* V,
                                       const void* psi_in, void* psi_q, void* psi_sum,
                                       int32_t flags, void* stream) {
    clear_error();
    const char* fn = "tacaw_multislice_static";
    TACAW_REQUIRE(grid != nullptr, TACAW_EINVAL, "%s: grid is NULL", fn);
    TACAW_REQUIRE(grid->nx > 0 && grid->ny > 0 && grid->n_slices > 0 && grid->n_slices <= 65535 &&
                      grid->lx > 0 && grid->ly > 0 && grid->dz > 0 && grid->kev > 0 &&
                      grid->bandlimit > 0 && isfinite(grid->lx) && isfinite(grid->ly) &&
                      isfinite(grid->dz) && isfinite(grid->z0) && isfinite(grid->kev) &&
                      isfinite(grid->bandlimit),
                  TACAW_EINVAL, "%s: bad grid", fn);
    TACAW_REQUIRE(multislice_size_supported(grid->nx) && multislice_size_supported(grid->ny),
                  TACAW_EUNSUPPORTED, "%s: nx = %d, ny = %d not in {64, 128, 256, 384, 512, 768, 1024}", fn,
                  grid->nx, grid->ny);
    const size_t need = multislice_ws_bytes(*grid);
    if (grid->nx == 1024 && grid->ny == 1024 && need != kLargestTablesBytes) {
        set_error("%s: the tables of a 1024 x 1024 grid take %zu bytes, not the %zu this file states", fn, need,
                  kLargestTablesBytes);
        return TACAW_EUNSUPPORTED;
    }
    TACAW_REQUIRE(need <= kStaticScratchBytes, TACAW_EINVAL,
                  "%s: this grid needs %zu bytes of scratch, more than the fixed %zu", fn, need,
                  kStaticScratchBytes);
    TACAW_REQUIRE(n_t >= 0 && n_t <= 65535, TACAW_EINVAL, "%s: n_t must be in [0, 65535]", fn);
    TACAW_REQUIRE((flags & ~(TACAW_MS_WARP_ROWS | TACAW_MS_BLOCK_COLS)) == 0, TACAW_EINVAL, "%s: unknown flags", fn);
    if (n_t == 0) return TACAW_OK;
    TACAW_REQUIRE(V && psi_q, TACAW_EINVAL, "%s: NULL array", fn);
    int rc = inject_launch_fault(fn);
    if (rc) return rc;
    void* scratch = nullptr;
    rc = static_scratch(&scratch);
    if (rc != TACAW_OK) return rc;
    // The tables are rewritten in full at the start of every call, so no part
    // of the shared array has to start at zero.
    return multislice_run(*grid, n_t, V, (const float2*)psi_in, (float2*)psi_q, (double2*)psi_sum,
                          scratch, (cudaStream_t)stream, flags);
}
