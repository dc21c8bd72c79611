// Composite variable tracking (Methods, "Composite variable tracking",
// Eq. 10 and Eq. 11): beside its size V, each cell keeps the integer sums S
// of its sites' coordinates, so that its centroid is S / V.  Under periodic
// boundaries a site counts at its periodic image nearest a reference point
// of the cell.  The round kernel keeps the sums up to date on every accepted
// copy (reference: the cell's centroid as the round began); the kernels here
// start them from a lattice (reference: the cell's first site in raster
// order) and move them by multiples of n V so that every centroid lies in
// [0, n) on each axis, which the paper does to keep its 32-bit sums in range
// and which here runs at the start and after every MCS.

#include <cstdint>

#include "cpm_internal.h"

namespace cpmgb {
namespace {

constexpr int kTrackThreads = 256;

__global__ void track_anchor_kernel(const int32_t *lat, uint64_t n, uint32_t *anchor)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t s = cell_id(lat[x]);
        if (s > 0) atomicMin(anchor + s, (uint32_t)x);
    }
}

template <int DIM>
__global__ void track_sum_kernel(const int32_t *lat, uint32_t nx, uint32_t ny, uint32_t nz, const uint32_t *anchor,
                                 long long *S)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t s = cell_id(lat[x]);
        if (s <= 0) continue;
        const uint32_t a = anchor[s];
        const int64_t px = (int64_t)(x % nx), py = (int64_t)((x / nx) % ny), pz = (int64_t)(x / ((uint64_t)nx * ny));
        const int64_t ax = a % nx, ay = (a / nx) % ny, az = a / (nx * ny);
        atomicAdd((unsigned long long *)(S + 3 * s), (unsigned long long)(px + nx * track_image_shift(px, ax, 1, nx)));
        atomicAdd((unsigned long long *)(S + 3 * s + 1),
                  (unsigned long long)(py + ny * track_image_shift(py, ay, 1, ny)));
        if (DIM == 3)
            atomicAdd((unsigned long long *)(S + 3 * s + 2),
                      (unsigned long long)(pz + nz * track_image_shift(pz, az, 1, nz)));
    }
}

__device__ __forceinline__ int64_t floor_div_p(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if (a % b != 0 && a < 0) q -= 1;
    return q;
}

// cell c's centroid into [0, n): the shift from the complete buffer, applied to both
__device__ __forceinline__ void rewrap_cell(int dim, uint32_t nx, uint32_t ny, uint32_t nz, int32_t c,
                                            const int32_t *V, long long *S_complete, long long *S_other)
{
    const int64_t v = V[c];
    if (v <= 0) return;
    for (int d = 0; d < dim; ++d) {
        const int64_t nv = (int64_t)(d == 0 ? nx : (d == 1 ? ny : nz)) * v;
        const int64_t shift = floor_div_p(S_complete[3 * c + d], nv) * nv;
        if (shift == 0) continue;
        S_complete[3 * c + d] -= shift;
        if (S_other) S_other[3 * c + d] -= shift;
    }
}

// one thread per cell id 1..n_cells; S_other may be null
__global__ void track_rewrap_kernel(int dim, uint32_t nx, uint32_t ny, uint32_t nz, int32_t n_cells,
                                    const int32_t *V, long long *S_complete, long long *S_other)
{
    const int32_t c = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x) + 1;
    if (c <= n_cells) rewrap_cell(dim, nx, ny, nz, c, V, S_complete, S_other);
}

// one CTA per batch member, after the advance of its MCS and round counters:
// buffer g_start & 1 is then the complete one
__global__ void batch_track_rewrap_kernel(int dim, const BatchLattice *lats)
{
    const BatchLattice &L = lats[blockIdx.x];
    if (!L.S[0]) return;
    const uint32_t par = (uint32_t)(L.g_start & 1u);
    for (int32_t c = (int32_t)threadIdx.x + 1; c <= L.n_cells; c += (int32_t)blockDim.x)
        rewrap_cell(dim, L.base.nx, L.base.ny, L.base.nz, c, L.V[par], L.S[par], L.S[par ^ 1u]);
}

unsigned grid_of(uint64_t n)
{
    uint64_t g = (n + kTrackThreads - 1) / kTrackThreads;
    if (g > 152ull * 32) g = 152ull * 32;
    return (unsigned)(g == 0 ? 1 : g);
}

}  // namespace

cudaError_t launch_track_rewrap(int dim, uint32_t nx, uint32_t ny, uint32_t nz, int32_t n_cells, const int32_t *V,
                                long long *S_complete, long long *S_other, cudaStream_t st)
{
    if (n_cells <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)(((uint32_t)n_cells + kTrackThreads - 1) / kTrackThreads);
    track_rewrap_kernel<<<blocks, kTrackThreads, 0, st>>>(dim, nx, ny, nz, n_cells, V, S_complete, S_other);
    return cudaGetLastError();
}

cudaError_t launch_batch_track_rewrap(int dim, const BatchLattice *lats, uint32_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    batch_track_rewrap_kernel<<<n, kTrackThreads, 0, st>>>(dim, lats);
    return cudaGetLastError();
}

cudaError_t launch_track_init(int dim, const int32_t *lat, uint32_t nx, uint32_t ny, uint32_t nz, int32_t n_cells,
                              const int32_t *V, uint32_t *anchor, long long *S, cudaStream_t st)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    cudaError_t e = cudaMemsetAsync(anchor, 0xFF, sizeof(uint32_t) * ((size_t)n_cells + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S, 0, sizeof(long long) * 3 * ((size_t)n_cells + 1), st);
    if (e != cudaSuccess) return e;
    track_anchor_kernel<<<grid_of(n), kTrackThreads, 0, st>>>(lat, n, anchor);
    if (dim == 3)
        track_sum_kernel<3><<<grid_of(n), kTrackThreads, 0, st>>>(lat, nx, ny, nz, anchor, S);
    else
        track_sum_kernel<2><<<grid_of(n), kTrackThreads, 0, st>>>(lat, nx, ny, nz, anchor, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_track_rewrap(dim, nx, ny, nz, n_cells, V, S, nullptr, st);
}

}  // namespace cpmgb
