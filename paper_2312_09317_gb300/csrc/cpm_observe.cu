// Observations of a batch of lattices and the summary statistics made of
// them.  Observations: per cell its
// anchor (first site in raster order), volume, integer sums of the
// minimal-image offsets of its sites from the anchor (a centroid in one
// periodic image, Methods, "Composite variable tracking", Eq. 10), their
// second moments (cell shape) and its interface count (Eq. 3); per lattice the cell-medium neighbour pairs and
// the accepted copies so far.
//
// Sites of one warp are mostly of one or two cells, so every per-cell sum is
// reduced over the lanes that share the cell id (__match_any_sync, then
// __reduce_*_sync over that group) and added by the group's first lane.
#include <cuda_runtime.h>

#include <cstdint>

#include "cpm_internal.h"

namespace cpmgb {
namespace {

constexpr int kObsThreads = 256;
constexpr double kArrestSpeed = 0.05;  // sites / MCS over a 50-MCS sub-track

__device__ __forceinline__ int min_image(int d, int n)
{
    // d in (-n, n); result in [-n/2, n - n/2)
    d += n / 2;
    if (d >= n) d -= n;
    if (d < 0) d += n;
    return d - n / 2;
}

__global__ void observe_init_kernel(const ObserveItem *items, int64_t *cells, int64_t *member)
{
    const ObserveItem it = items[blockIdx.x];
    for (int64_t r = threadIdx.x; r <= it.n_cells; r += blockDim.x) {
        int64_t *row = cells + (it.row0 + r) * kObsFields;
        row[0] = -1;  // all ones: the identity of the unsigned minimum
        for (int f = 1; f < kObsFields; ++f) row[f] = 0;
    }
    if (threadIdx.x == 0) {
        member[2 * blockIdx.x] = 0;
        member[2 * blockIdx.x + 1] = (int64_t)*it.accepts;
    }
}

__global__ void __launch_bounds__(kObsThreads) observe_anchor_kernel(const ObserveItem *items, int64_t *cells)
{
    const ObserveItem it = items[blockIdx.y];
    const int64_t n = (int64_t)it.nx * it.ny * it.nz;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int id = i < n ? cell_id(it.lat[i]) : 0;
        if (id > it.n_cells) id = 0;  // never present in a validated lattice; keeps the write in bounds
        const unsigned grp = __match_any_sync(0xffffffffu, id);
        const unsigned lo = __reduce_min_sync(grp, (unsigned)(i < n ? i : 0xffffffffu));
        if (id > 0 && lane == __ffs(grp) - 1)
            atomicMin(reinterpret_cast<unsigned long long *>(cells + (it.row0 + id) * kObsFields), (unsigned long long)lo);
    }
}

template <int DIM>
__global__ void __launch_bounds__(kObsThreads) observe_sums_kernel(const ObserveItem *items, int64_t *cells,
                                                                   int64_t *member)
{
    const ObserveItem it = items[blockIdx.y];
    const int nx = (int)it.nx, ny = (int)it.ny, nz = (int)it.nz;
    const int64_t plane = (int64_t)nx * ny, n = plane * nz;
    const int lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = base + threadIdx.x;
        int id = i < n ? cell_id(it.lat[i]) : 0;
        if (id > it.n_cells) id = 0;
        int ox = 0, oy = 0, oz = 0, iface = 0, medium = 0;
        if (id > 0) {
            const int z = (int)(i / plane), y = (int)((i / nx) % ny), x = (int)(i % nx);
            const int64_t a = cells[(it.row0 + id) * kObsFields];
            const int az = (int)(a / plane), ay = (int)((a / nx) % ny), ax = (int)(a % nx);
            ox = min_image(x - ax, nx);
            oy = min_image(y - ay, ny);
            oz = min_image(z - az, nz);
            const int zlo = DIM == 3 ? -1 : 0, zhi = DIM == 3 ? 1 : 0;
            for (int dz = zlo; dz <= zhi; ++dz) {
                int zz = z + dz;
                zz = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
                for (int dy = -1; dy <= 1; ++dy) {
                    int yy = y + dy;
                    yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (dx == 0 && dy == 0 && dz == 0) continue;
                        int xx = x + dx;
                        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                        const int v = cell_id(it.lat[(int64_t)zz * plane + (int64_t)yy * nx + xx]);
                        iface += v != id;
                        medium += v == 0;
                    }
                }
            }
        }
        const unsigned grp = __match_any_sync(0xffffffffu, id);
        const int cnt = __reduce_add_sync(grp, id > 0 ? 1 : 0);
        const int sx = __reduce_add_sync(grp, ox), sy = __reduce_add_sync(grp, oy), sz = __reduce_add_sync(grp, oz);
        const int sf = __reduce_add_sync(grp, iface);
        const int sxx = __reduce_add_sync(grp, ox * ox), syy = __reduce_add_sync(grp, oy * oy);
        const int szz = __reduce_add_sync(grp, oz * oz), sxy = __reduce_add_sync(grp, ox * oy);
        const int sxz = __reduce_add_sync(grp, ox * oz), syz = __reduce_add_sync(grp, oy * oz);
        const int sm = __reduce_add_sync(0xffffffffu, medium);
        if (id > 0 && lane == __ffs(grp) - 1) {
            unsigned long long *row = reinterpret_cast<unsigned long long *>(cells + (it.row0 + id) * kObsFields);
            atomicAdd(row + 1, (unsigned long long)(int64_t)cnt);
            atomicAdd(row + 2, (unsigned long long)(int64_t)sx);
            atomicAdd(row + 3, (unsigned long long)(int64_t)sy);
            atomicAdd(row + 4, (unsigned long long)(int64_t)sz);
            atomicAdd(row + 5, (unsigned long long)(int64_t)sf);
            atomicAdd(row + 6, (unsigned long long)(int64_t)sxx);
            atomicAdd(row + 7, (unsigned long long)(int64_t)syy);
            atomicAdd(row + 8, (unsigned long long)(int64_t)szz);
            atomicAdd(row + 9, (unsigned long long)(int64_t)sxy);
            atomicAdd(row + 10, (unsigned long long)(int64_t)sxz);
            atomicAdd(row + 11, (unsigned long long)(int64_t)syz);
        }
        if (lane == 0 && sm)
            atomicAdd(reinterpret_cast<unsigned long long *>(member + 2 * blockIdx.y), (unsigned long long)sm);
    }
}

constexpr int kSumThreads = 128;
constexpr int kMaxLag = 20;  // step-direction autocorrelation lags (x every MCS)
// scalar accumulators of one lattice
enum {
    A_MSD = 0,       // 3 sums, then 3 counts
    A_SP = 6,        // speed sum, sum of squares, count
    A_ST = 9,        // straightness sum, count
    A_DAC = 11,      // 50-MCS direction cosine sum, count
    A_SLOW = 13,     // slow 50-MCS sub-tracks, count
    A_EL = 15,       // elongation sum, count
    A_AC = 17,       // autocorrelation sums, lags 0..kMaxLag
    A_ACN = A_AC + kMaxLag + 1,
    A_N = A_ACN + kMaxLag + 1
};

// One CTA per lattice, threads over its cells.  Per cell: the centroid at
// every snapshot (anchor + offset sums / volume), unwrapped across
// snapshots by minimal-image steps; a cell absent at any snapshot has no
// track.  Per-snapshot volume and interface moments and every track
// statistic are accumulated in shared memory, then thread 0 forms the
// sixteen statistics.
__global__ void __launch_bounds__(kSumThreads) summarize_kernel(const ObserveItem *items, const int64_t *cells,
                                                                int64_t rows, const int64_t *member, int n_items,
                                                                int S1, int every, double *traj, double *out)
{
    extern __shared__ double snap[];  // sV, sV2, sA, sA2, sN: S1 each
    __shared__ double acc[A_N];
    const int run = blockIdx.x;
    const ObserveItem it = items[run];
    double *sV = snap, *sV2 = snap + S1, *sA = snap + 2 * S1, *sA2 = snap + 3 * S1, *sN = snap + 4 * S1;
    for (int i = threadIdx.x; i < 5 * S1; i += blockDim.x) snap[i] = 0.0;
    for (int i = threadIdx.x; i < A_N; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    const int nx = (int)it.nx, ny = (int)it.ny;
    const int lags[3] = {10, 50, 200};
    const int k50 = 50 % every == 0 ? 50 / every : 0;
    const int n_ac = S1 - 1 < kMaxLag + 1 ? S1 - 1 : kMaxLag + 1;  // lags 1 .. n_ac - 1
    for (int c = 1 + threadIdx.x; c <= it.n_cells; c += blockDim.x) {
        const int64_t row = it.row0 + c;
        double *tr = traj + row * 2 * S1;
        bool track = true;
        double px = 0.0, py = 0.0, qx = 0.0, qy = 0.0, el = 0.0, eln = 0.0;
        for (int s = 0; s < S1; ++s) {
            const int64_t *r = cells + ((int64_t)s * rows + row) * kObsFields;
            if (r[1] <= 0) {
                track = false;
                continue;
            }
            const double V = (double)r[1], A = (double)r[5];
            atomicAdd(&sV[s], V);
            atomicAdd(&sV2[s], V * V);
            atomicAdd(&sA[s], A);
            atomicAdd(&sA2[s], A * A);
            atomicAdd(&sN[s], 1.0);
            const double mx = (double)r[2] / V, my = (double)r[3] / V;
            const double cxx = (double)r[6] / V - mx * mx, cyy = (double)r[7] / V - my * my;
            const double cxy = (double)r[9] / V - mx * my;
            const double t2 = cxx + cyy, det = cxx * cyy - cxy * cxy;
            const double disc = sqrt(fmax(t2 * t2 / 4.0 - det, 0.0));
            const double l1 = t2 / 2.0 + disc, l2 = t2 / 2.0 - disc;
            if (l2 > 1e-9) {
                el += sqrt(l1 / l2);
                eln += 1.0;
            }
            const double cx = (double)(r[0] % nx) + mx, cy = (double)(r[0] / nx) + my;
            if (track) {
                if (s > 0) {
                    double dx = cx - qx, dy = cy - qy;
                    dx -= nx * rint(dx / nx);
                    dy -= ny * rint(dy / ny);
                    px += dx;
                    py += dy;
                }
                tr[2 * s] = px;
                tr[2 * s + 1] = py;
            }
            qx = cx;
            qy = cy;
        }
        atomicAdd(&acc[A_EL], el);
        atomicAdd(&acc[A_EL + 1], eln);
        if (!track) continue;
        for (int j = 0; j < 3; ++j) {
            if (lags[j] % every) continue;
            const int k = lags[j] / every;
            if (k <= 0 || k >= S1) continue;
            double sum = 0.0;
            for (int s = 0; s + k < S1; ++s) {
                const double dx = tr[2 * (s + k)] - tr[2 * s], dy = tr[2 * (s + k) + 1] - tr[2 * s + 1];
                sum += dx * dx + dy * dy;
            }
            atomicAdd(&acc[A_MSD + j], sum);
            atomicAdd(&acc[A_MSD + 3 + j], (double)(S1 - k));
        }
        if (S1 > 1) {
            double ssum = 0.0, ssq = 0.0, path = 0.0;
            for (int s = 0; s + 1 < S1; ++s) {
                const double dx = tr[2 * s + 2] - tr[2 * s], dy = tr[2 * s + 3] - tr[2 * s + 1];
                const double nrm = sqrt(dx * dx + dy * dy);
                ssum += nrm / every;
                ssq += (nrm / every) * (nrm / every);
                path += nrm;
            }
            atomicAdd(&acc[A_SP], ssum);
            atomicAdd(&acc[A_SP + 1], ssq);
            atomicAdd(&acc[A_SP + 2], (double)(S1 - 1));
            if (path > 0.0) {
                const double nx_ = tr[2 * (S1 - 1)] - tr[0], ny_ = tr[2 * (S1 - 1) + 1] - tr[1];
                atomicAdd(&acc[A_ST], sqrt(nx_ * nx_ + ny_ * ny_) / path);
                atomicAdd(&acc[A_ST + 1], 1.0);
            }
            for (int k = 1; k < n_ac; ++k) {
                double sum = 0.0, cnt = 0.0;
                for (int s = 0; s + k + 1 < S1; ++s) {
                    const double ax = tr[2 * s + 2] - tr[2 * s], ay = tr[2 * s + 3] - tr[2 * s + 1];
                    const double bx = tr[2 * (s + k) + 2] - tr[2 * (s + k)];
                    const double by = tr[2 * (s + k) + 3] - tr[2 * (s + k) + 1];
                    const double na = sqrt(ax * ax + ay * ay), nb = sqrt(bx * bx + by * by);
                    if (na > 0.0 && nb > 0.0) {
                        sum += (ax / na) * (bx / nb) + (ay / na) * (by / nb);
                        cnt += 1.0;
                    }
                }
                atomicAdd(&acc[A_AC + k], sum);
                atomicAdd(&acc[A_ACN + k], cnt);
            }
        }
        if (k50 > 0 && 2 * k50 < S1) {
            double dsum = 0.0, dcnt = 0.0, slow = 0.0;
            for (int s = 0; s + k50 < S1; ++s) {
                const double ax = tr[2 * (s + k50)] - tr[2 * s], ay = tr[2 * (s + k50) + 1] - tr[2 * s + 1];
                const double na = sqrt(ax * ax + ay * ay);
                slow += na / 50.0 < kArrestSpeed ? 1.0 : 0.0;
                if (s + 2 * k50 < S1) {
                    const double bx = tr[2 * (s + 2 * k50)] - tr[2 * (s + k50)];
                    const double by = tr[2 * (s + 2 * k50) + 1] - tr[2 * (s + k50) + 1];
                    const double nb = sqrt(bx * bx + by * by);
                    if (na > 0.0 && nb > 0.0) {
                        dsum += (ax * bx + ay * by) / (na * nb);
                        dcnt += 1.0;
                    }
                }
            }
            atomicAdd(&acc[A_DAC], dsum);
            atomicAdd(&acc[A_DAC + 1], dcnt);
            atomicAdd(&acc[A_SLOW], slow);
            atomicAdd(&acc[A_SLOW + 1], (double)(S1 - k50));
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    double *o = out + (int64_t)run * kSummaryStats;
    for (int k = 0; k < kSummaryStats; ++k) o[k] = qnan;
    double tv = 0.0, ta = 0.0, tn = 0.0, vv = 0.0, av = 0.0, nv = 0.0;
    for (int s = 0; s < S1; ++s) {
        tv += sV[s];
        ta += sA[s];
        tn += sN[s];
        if (sN[s] > 0.0) {
            const double mv = sV[s] / sN[s], ma = sA[s] / sN[s];
            vv += fmax(sV2[s] / sN[s] - mv * mv, 0.0);
            av += fmax(sA2[s] / sN[s] - ma * ma, 0.0);
            nv += 1.0;
        }
    }
    // a statistic scaled by a target of 0 (no volume or perimeter constraint) is undefined: NaN
    if (tn > 0.0) {
        if (it.v_ref != 0.0) o[0] = tv / tn / it.v_ref;
        if (it.a_ref != 0.0) o[2] = ta / tn / it.a_ref;
    }
    if (nv > 0.0) {
        if (it.v_ref != 0.0) o[1] = sqrt(vv / nv) / it.v_ref;
        if (it.a_ref != 0.0) o[3] = sqrt(av / nv) / it.a_ref;
    }
    for (int j = 0; j < 3; ++j)
        if (acc[A_MSD + 3 + j] > 0.0) o[4 + j] = acc[A_MSD + j] / acc[A_MSD + 3 + j];
    if (acc[A_SP + 2] > 0.0) {
        const double m = acc[A_SP] / acc[A_SP + 2];
        o[7] = m;
        o[8] = sqrt(fmax(acc[A_SP + 1] / acc[A_SP + 2] - m * m, 0.0));
    }
    if (acc[A_DAC + 1] > 0.0) o[9] = acc[A_DAC] / acc[A_DAC + 1];
    if (S1 > 1) {
        double pers = 0.5 * every;
        for (int k = 1; k < n_ac; ++k) {
            const double ck = acc[A_ACN + k] > 0.0 ? acc[A_AC + k] / acc[A_ACN + k] : 0.0;
            if (!(ck > 0.0)) break;
            pers += ck * every;
        }
        o[10] = pers;
    }
    if (acc[A_SLOW + 1] > 0.0) o[11] = acc[A_SLOW] / acc[A_SLOW + 1];
    if (S1 > 1) {
        const int64_t m0 = member[2 * (int64_t)run + 1];
        const int64_t m1 = member[2 * ((int64_t)(S1 - 1) * n_items + run) + 1];
        const double sites = (double)it.nx * it.ny * it.nz;
        o[12] = (double)(m1 - m0) / ((double)(S1 - 1) * every * sites);
    }
    double cf = 0.0, cfn = 0.0;
    for (int s = 0; s < S1; ++s) {
        const double cm = (double)member[2 * ((int64_t)s * n_items + run)];
        const double cc = (sA[s] - cm) / 2.0, tot = cc + cm;
        if (tot > 0.0) {
            cf += cc / tot;
            cfn += 1.0;
        }
    }
    if (cfn > 0.0) o[13] = cf / cfn;
    if (acc[A_ST + 1] > 0.0) o[14] = acc[A_ST] / acc[A_ST + 1];
    if (acc[A_EL + 1] > 0.0) o[15] = acc[A_EL] / acc[A_EL + 1];
}

// Persistence update (Eq. 6, Eq. 7) for every cell, one thread per cell,
// from this MCS's observation rows: record the centroid (anchor + offset
// sums / volume, NaN for an absent cell) in history slot t % H, then blend
// the unit displacement over dt MCS into p_hat.  Every operation is a single
// rounded double operation in the order the replay uses (no contraction).
__global__ void pers_update_kernel(const int64_t *cells, int32_t n_cells, uint32_t nx, uint32_t ny, uint32_t nz,
                                   const uint8_t *cell_type, const PersParams pp, double *hist, int32_t H,
                                   int64_t t, int64_t t0, double *dir)
{
    const int64_t c = 1 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n_cells) return;
    const int64_t nc = (int64_t)n_cells + 1;
    const int64_t *r = cells + c * kObsFields;
    double *Xn = hist + 3 * (nc * (t % H) + c);
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    if (r[1] <= 0) {
        Xn[0] = Xn[1] = Xn[2] = qnan;
        return;
    }
    const int64_t an = r[0], plane = (int64_t)nx * ny;
    const double V = (double)r[1];
    const double ac[3] = {(double)(an % nx), (double)((an / nx) % ny), (double)(an / plane)};
    for (int d = 0; d < 3; ++d) Xn[d] = __dadd_rn(ac[d], __ddiv_rn((double)r[2 + d], V));
    const int tp = cell_type[c];
    const int dt = pp.dt[tp];
    if (pp.lambda[tp] == 0 || dt < 1 || t - dt < t0) return;
    const double *Xo = hist + 3 * (nc * ((t - dt) % H) + c);
    if (isnan(Xo[0])) return;
    const double L[3] = {(double)nx, (double)ny, (double)nz};
    double D[3];
    for (int d = 0; d < 3; ++d) {
        const double v = __dsub_rn(Xn[d], Xo[d]);
        D[d] = __dsub_rn(v, __dmul_rn(L[d], rint(__ddiv_rn(v, L[d]))));
    }
    double n2 = __dmul_rn(D[0], D[0]);
    n2 = __dadd_rn(n2, __dmul_rn(D[1], D[1]));
    n2 = __dadd_rn(n2, __dmul_rn(D[2], D[2]));
    if (n2 == 0.0) return;
    const double n = __dsqrt_rn(n2), mu = pp.mu[tp], am = __dsub_rn(1.0, mu);
    double *ph = dir + 3 * c, q[3];
    for (int d = 0; d < 3; ++d) {
        const double u = __ddiv_rn(D[d], n);
        q[d] = __dadd_rn(__dmul_rn(am, u), __dmul_rn(mu, ph[d]));
    }
    double m2 = __dmul_rn(q[0], q[0]);
    m2 = __dadd_rn(m2, __dmul_rn(q[1], q[1]));
    m2 = __dadd_rn(m2, __dmul_rn(q[2], q[2]));
    if (m2 == 0.0) {
        ph[0] = ph[1] = ph[2] = 0.0;
        return;
    }
    const double m = __dsqrt_rn(m2);
    for (int d = 0; d < 3; ++d) ph[d] = __ddiv_rn(q[d], m);
}

}  // namespace

cudaError_t launch_pers_update(const int64_t *cells, int32_t n_cells, uint32_t nx, uint32_t ny, uint32_t nz,
                               const uint8_t *cell_type, const PersParams &pp, double *hist, int32_t H, int64_t t,
                               int64_t t0, double *dir, cudaStream_t st)
{
    if (n_cells < 1) return cudaSuccess;
    pers_update_kernel<<<(n_cells + 127) / 128, 128, 0, st>>>(cells, n_cells, nx, ny, nz, cell_type, pp, hist, H, t,
                                                              t0, dir);
    return cudaPeekAtLastError();
}

cudaError_t launch_summarize(const ObserveItem *d_items, uint32_t n_items, int32_t max_cells, const int64_t *cells,
                             int64_t rows, const int64_t *member, int32_t n_snap, int32_t every, double *traj,
                             double *out, cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    if (n_snap < 1 || n_snap > kSummaryMaxSnap || every < 1) return cudaErrorInvalidValue;
    int threads = ((max_cells + 31) / 32) * 32;
    threads = threads < 32 ? 32 : (threads > kSumThreads ? kSumThreads : threads);
    const size_t smem = sizeof(double) * 5 * (size_t)n_snap;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(summarize_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    summarize_kernel<<<n_items, threads, smem, st>>>(d_items, cells, rows, member, (int)n_items, n_snap, every, traj,
                                                     out);
    return cudaPeekAtLastError();
}

cudaError_t launch_observe(int dim, const ObserveItem *d_items, uint32_t n_items, int64_t max_sites, int64_t *cells,
                           int64_t *member, cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    if (n_items > 65535u) return cudaErrorInvalidValue;
    observe_init_kernel<<<n_items, 256, 0, st>>>(d_items, cells, member);
    int64_t bx = (max_sites + kObsThreads - 1) / kObsThreads;
    if (bx > 64) bx = 64;
    const dim3 grid((unsigned)bx, n_items);
    observe_anchor_kernel<<<grid, kObsThreads, 0, st>>>(d_items, cells);
    if (dim == 3) observe_sums_kernel<3><<<grid, kObsThreads, 0, st>>>(d_items, cells, member);
    else observe_sums_kernel<2><<<grid, kObsThreads, 0, st>>>(d_items, cells, member);
    return cudaPeekAtLastError();
}

}  // namespace cpmgb
