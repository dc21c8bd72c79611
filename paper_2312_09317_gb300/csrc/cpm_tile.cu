// Tiled schedule of the CPM sweep: one CTA per active tile, all rounds of an
// epoch run on a shared-memory copy of the tile and its halo.
//
// Tiles of edge T (a multiple of the area edge a) lie on a grid shifted per
// MCS; tiles of one tile colour (parity of the tile coordinates) are active
// together in an epoch while the tiles around them are dormant, so the halo a
// tile reads does not change during the epoch.  An active tile runs its share
// of the MCS's sub-passes in order (the same colours, rounds and Philox
// counters as the global schedule, restricted to the blocks inside the tile),
// with a barrier after every round (Results, Fig. 3A) and the paper's copy
// attempt (Methods, Eq. 1-3, Eq. 8-9).  Tallies read by the tile are the
// snapshot at the epoch start plus the tile's own changes of earlier rounds,
// kept in a shared-memory hash; at the end of the epoch the tile writes its
// interior back and adds its changes into the next tally buffer.
//
// Traffic per epoch: the tile and halo are read once and the interior written
// once, instead of the whole lattice per round.
#include <cstdint>

#include "cpm_internal.h"

namespace cpmgb {
namespace {

constexpr int kTileThreads = 256;

struct TileSmemTables {
    int32_t J[kMaxTypes * kMaxTypes];
    int32_t lv[kMaxTypes], vt[kMaxTypes], lp[kMaxTypes], at[kMaxTypes], la[kMaxTypes], ma[kMaxTypes];
    int32_t ln[kLnEntries];
    int32_t colours[kMaxEpochSubpasses];
    int overflow;
    unsigned long long accepts;
};

__device__ __forceinline__ uint32_t wrapc(int32_t v, uint32_t n)
{
    // v in [-n, 2n)
    return v < 0 ? (uint32_t)(v + (int32_t)n) : ((uint32_t)v >= n ? (uint32_t)v - n : (uint32_t)v);
}

__device__ __forceinline__ int act_of(uint8_t stamp, uint32_t t8, int max_act)
{
    const int age = (int)((t8 - (uint32_t)stamp) & 255u);
    const int v = max_act - age;
    return v > 0 ? v : 0;
}

// Shared-memory lattice words (16 bit): bits 0..11 a local slot (0 = medium,
// 1 = obstacle, 2.. = the cells present in the tile and its halo), bits
// 12..14 the type.  Per slot, shared memory holds the cell's global id, its
// tallies at the epoch start and the tile's changes, so an attempt reads no
// global memory except the tail of the threshold table.
constexpr int kGroup = 8;            // lanes that evaluate one candidate attempt together
constexpr uint32_t kSlotBits = 12;
constexpr uint32_t kSlotMask = (1u << kSlotBits) - 1u;

__device__ __forceinline__ uint32_t slot_of(uint32_t w) { return w & kSlotMask; }
__device__ __forceinline__ int type_in(uint32_t w) { return (int)(w >> kSlotBits); }

struct TileLayout {
    uint16_t *lat;
    uint8_t *stamp;
    int32_t *hkeys;      // hash: global id -> slot
    uint16_t *hslot;
    int32_t *gid;        // per slot
    int32_t *sV, *sA, *dV, *dA;
    uint8_t *stype;
    uint32_t *thr;       // first thr_n entries of the threshold table
    uint2 *cand;
    int4 *chg;
    int32_t *off;        // linear offsets of the 3^d stencil (centre included), lexicographic
};

__device__ __forceinline__ uint32_t hslot_of(int32_t key, uint32_t mask)
{
    return ((uint32_t)key * 2654435761u >> 7) & mask;
}

template <int DIM, bool PERIM, bool ACT>
__global__ void __launch_bounds__(kTileThreads) tile_epoch_kernel(const TileArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileSmemTables sm;
    __shared__ uint32_t n_cand[2];
    __shared__ uint32_t n_slots;
    constexpr int NB = DIM == 3 ? 26 : 8;
    constexpr int NS = NB + 1;
    constexpr uint32_t H = 2;
    const uint32_t T = a.T;
    const uint32_t W = T + 2 * H;
    const uint32_t WZ = DIM == 3 ? W : 1;
    const uint32_t n_local = W * W * WZ;
    const uint32_t per_axis = T / (a.s * a.c);
    const uint32_t n_blk = per_axis * per_axis * (DIM == 3 ? per_axis : 1);
    const uint32_t cap = a.hash_cap;          // slots
    const uint32_t hcap = 2 * cap;            // hash entries
    const uint32_t hmask = hcap - 1;

    // carve shared memory (every piece 16-byte aligned)
    TileLayout L;
    {
        unsigned char *p = smem_raw;
        auto take = [&](size_t bytes) { unsigned char *q = p; p += (bytes + 15) & ~(size_t)15; return q; };
        L.lat = (uint16_t *)take(sizeof(uint16_t) * n_local);
        L.stamp = ACT ? (uint8_t *)take(n_local) : nullptr;
        L.hkeys = (int32_t *)take(sizeof(int32_t) * hcap);
        L.hslot = (uint16_t *)take(sizeof(uint16_t) * hcap);
        L.gid = (int32_t *)take(sizeof(int32_t) * cap);
        L.sV = (int32_t *)take(sizeof(int32_t) * cap);
        L.sA = (int32_t *)take(sizeof(int32_t) * cap);
        L.dV = (int32_t *)take(sizeof(int32_t) * cap);
        L.dA = (int32_t *)take(sizeof(int32_t) * cap);
        L.stype = (uint8_t *)take(cap);
        L.thr = (uint32_t *)take(sizeof(uint32_t) * a.thr_smem);
        L.cand = (uint2 *)take(sizeof(uint2) * n_blk);
        L.chg = (int4 *)take(sizeof(int4) * n_blk);
        L.off = (int32_t *)take(sizeof(int32_t) * 27);
    }

    // tables
    for (int k = threadIdx.x; k < kMaxTypes * kMaxTypes; k += blockDim.x) sm.J[k] = a.tp.J[k / kMaxTypes][k % kMaxTypes];
    if (threadIdx.x < kMaxTypes) {
        const int k = threadIdx.x;
        sm.lv[k] = a.tp.lambda_v[k];
        sm.vt[k] = a.tp.v_target[k];
        sm.lp[k] = a.tp.lambda_p[k];
        sm.at[k] = a.tp.a_target[k];
        sm.la[k] = a.tp.lambda_act[k];
        sm.ma[k] = a.tp.max_act[k];
    }
    if (ACT)
        for (int k = threadIdx.x; k < kLnEntries; k += blockDim.x) sm.ln[k] = a.ln_tab[k];
    for (int k = threadIdx.x; k < (int)a.n_sub; k += blockDim.x) sm.colours[k] = a.colours[k];
    for (uint32_t k = threadIdx.x; k < a.thr_smem; k += blockDim.x) L.thr[k] = __ldg(a.thr + k);
    if (threadIdx.x < (unsigned)(DIM == 3 ? 27 : 9)) {
        const int k = threadIdx.x;
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = DIM == 3 ? k / 9 - 1 : 0;
        L.off[k] = dx + (int)W * (dy + (int)W * dz);
    }
    if (threadIdx.x == 0) {
        sm.overflow = 0;
        sm.accepts = 0;
        n_cand[0] = 0;
        n_cand[1] = 0;
        n_slots = 2;
    }
    for (uint32_t k = threadIdx.x; k < hcap; k += blockDim.x) L.hkeys[k] = 0;
    if (threadIdx.x < 2) {
        L.gid[threadIdx.x] = threadIdx.x == 0 ? 0 : -1;
        L.stype[threadIdx.x] = threadIdx.x == 0 ? 0 : (uint8_t)a.tp.obstacle_type;
    }
    __syncthreads();

    // this CTA's tile: the blockIdx.x-th tile of the active tile colour
    const uint32_t ntx = a.nx / T, nty = a.ny / T;
    const uint32_t hx = ntx / 2, hy = nty / 2;
    const uint32_t m = blockIdx.x;
    const uint32_t kx = (m % hx) * 2 + a.tcx;
    const uint32_t ky = ((m / hx) % hy) * 2 + a.tcy;
    const uint32_t kz = DIM == 3 ? (m / (hx * hy)) * 2 + a.tcz : 0;
    const uint32_t ox = (a.offx + kx * T) % a.nx;
    const uint32_t oy = (a.offy + ky * T) % a.ny;
    const uint32_t oz = DIM == 3 ? (a.offz + kz * T) % a.nz : 0;
    auto global_of = [&](uint32_t l) -> uint64_t {
        const uint32_t lx = l % W, ly = (l / W) % W, lz = l / (W * W);
        const uint32_t gx = wrapc((int32_t)(ox + lx) - (int32_t)H, a.nx);
        const uint32_t gy = wrapc((int32_t)(oy + ly) - (int32_t)H, a.ny);
        const uint32_t gz = DIM == 3 ? wrapc((int32_t)(oz + lz) - (int32_t)H, a.nz) : 0;
        return gx + (uint64_t)a.nx * (gy + (uint64_t)a.ny * gz);
    };

    // staging pass 1: give every cell of the tile and halo a slot
    constexpr int kStage = 8;
    for (uint32_t base = 0; base < n_local; base += kStage * blockDim.x) {
        int32_t v[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const uint32_t l = base + u * blockDim.x + threadIdx.x;
            v[u] = l < n_local ? cell_id(__ldg(a.lat + global_of(l))) : 0;
        }
        int32_t last = 0;
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int32_t g = v[u];
            if (g <= 0 || g == last) continue;
            last = g;
            uint32_t h = hslot_of(g, hmask);
            for (uint32_t probe = 0; probe <= hmask; ++probe) {
                int32_t k = L.hkeys[h];
                if (k == 0) {
                    k = atomicCAS(L.hkeys + h, 0, g);
                    if (k == 0) {
                        const uint32_t sl = atomicAdd(&n_slots, 1u);
                        if (sl < cap) {
                            L.hslot[h] = (uint16_t)sl;
                            L.gid[sl] = g;
                        } else {
                            sm.overflow = 1;
                            L.hslot[h] = 0;
                        }
                        break;
                    }
                }
                if (k == g) break;
                h = (h + 1) & hmask;
            }
        }
    }
    __syncthreads();
    const uint32_t ns = min(n_slots, cap);
    for (uint32_t sl = 2 + threadIdx.x; sl < ns; sl += blockDim.x) {
        const int32_t g = L.gid[sl];
        L.sV[sl] = __ldg(a.Vc + g);
        L.sA[sl] = __ldg(a.Ac + g);
        L.dV[sl] = 0;
        L.dA[sl] = 0;
        L.stype[sl] = __ldg(a.cell_type + g);
    }
    __syncthreads();
    // staging pass 2: lattice words (the tile was just read, so this hits L2) and stamps
    for (uint32_t base = 0; base < n_local; base += kStage * blockDim.x) {
        int32_t v[kStage];
        uint8_t st[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const uint32_t l = base + u * blockDim.x + threadIdx.x;
            v[u] = 0;
            if (l < n_local) {
                const uint64_t g = global_of(l);
                const int32_t w = __ldcs(a.lat + g);
                v[u] = cell_id(w);
                if (ACT) st[u] = (uint8_t)word_stamp(w);
            }
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const uint32_t l = base + u * blockDim.x + threadIdx.x;
            if (l >= n_local) continue;
            const int32_t g = v[u];
            uint32_t sl = g == 0 ? 0u : (g < 0 ? 1u : 0u);
            if (g > 0) {
                uint32_t h = hslot_of(g, hmask);
                for (uint32_t probe = 0; probe <= hmask; ++probe) {
                    if (L.hkeys[h] == g) { sl = L.hslot[h]; break; }
                    h = (h + 1) & hmask;
                }
            }
            L.lat[l] = (uint16_t)(sl | ((uint32_t)L.stype[sl] << kSlotBits));
            if (ACT) L.stamp[l] = st[u];
        }
    }
    __syncthreads();

    const uint32_t bx0 = ox / a.s, by0 = oy / a.s, bz0 = oz / a.s;
    const uint32_t t8 = a.t & 255u;
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t glane = threadIdx.x % kGroup;
    const uint32_t group = threadIdx.x / kGroup;
    const uint32_t n_groups = blockDim.x / kGroup;
    const unsigned gmask = ((1u << kGroup) - 1u) << (lane & ~(uint32_t)(kGroup - 1));
    const uint32_t s = a.s, cc_ = a.c;
    uint32_t my_accepts = 0;
    uint32_t parity = 0;
    uint32_t prev_nc = 0;  // changes of the previous round still to apply

    for (uint32_t q = 0; q < a.n_sub; ++q) {
        const uint32_t col = (uint32_t)sm.colours[q];
        const uint32_t cx = col % cc_, cy = (col / cc_) % cc_, cz = col / (cc_ * cc_);
        const uint32_t sp = a.sp0 + q;
        for (uint32_t r = 0; r < a.k; ++r, parity ^= 1u) {
            // ---- the previous round's changes become visible (slot tallies) ...
            for (uint32_t c = threadIdx.x; c < prev_nc; c += blockDim.x) {
                const int4 ch = L.chg[c];
                if (ch.x == ch.y) continue;
                if (ch.x >= 2) { atomicAdd(L.dV + ch.x, 1); atomicAdd(L.dA + ch.x, ch.z); }
                if (ch.y >= 2) { atomicAdd(L.dV + ch.y, -1); atomicAdd(L.dA + ch.y, ch.w); }
            }
            // ---- ... while phase A draws this round's attempts and keeps the candidates
            for (uint32_t base = 0; base < n_blk; base += blockDim.x) {
                const uint32_t ib = base + threadIdx.x;
                bool keep = false;
                uint2 item = make_uint2(0, 0);
                if (ib < n_blk) {
                    const uint32_t mx = ib % per_axis, my = (ib / per_axis) % per_axis, mz = ib / (per_axis * per_axis);
                    const uint32_t lbx = mx * cc_ + cx, lby = my * cc_ + cy, lbz = DIM == 3 ? mz * cc_ + cz : 0;
                    uint32_t gbx = bx0 + lbx, gby = by0 + lby, gbz = bz0 + lbz;
                    if (gbx >= a.nbx) gbx -= a.nbx;
                    if (gby >= a.nby) gby -= a.nby;
                    if (DIM == 3 && gbz >= a.nbz) gbz -= a.nbz;
                    const uint32_t b = gbx + a.nbx * (gby + a.nby * gbz);
                    const Philox4 w = philox4x32_10(b, r, a.t, sp, a.key0, a.key1);
                    const uint32_t jl = draw_below(w.v[0], a.sd);
                    const uint32_t jx = H + lbx * s + jl % s;
                    const uint32_t jy = H + lby * s + (jl / s) % s;
                    const uint32_t jz = DIM == 3 ? H + lbz * s + jl / (s * s) : 0;
                    const uint32_t n = draw_below(w.v[1], NB);
                    const uint32_t j = jx + W * (jy + W * jz);
                    const uint32_t i = (uint32_t)((int32_t)j + L.off[n + (n >= NB / 2 ? 1u : 0u)]);
                    const uint32_t wj = L.lat[j], wi = L.lat[i];
                    keep = wi != wj && slot_of(wi) != 1u && slot_of(wj) != 1u;
                    item = make_uint2(j | (i << 16), w.v[2]);
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                uint32_t slot0 = 0;
                if (lane == 0 && bal) slot0 = atomicAdd(&n_cand[parity], (uint32_t)__popc(bal));
                slot0 = __shfl_sync(0xffffffffu, slot0, 0);
                if (keep) L.cand[slot0 + __popc(bal & ((1u << lane) - 1u))] = item;
            }
            __syncthreads();

            // ---- phase B: kGroup lanes per candidate, everything in shared memory
            const uint32_t nc = n_cand[parity];
            if (threadIdx.x == 0) n_cand[parity ^ 1u] = 0;
            for (uint32_t c = group; c < nc; c += n_groups) {
                const uint2 it = L.cand[c];
                const uint32_t j = it.x & 0xFFFFu, i = it.x >> 16;
                const uint32_t wj = L.lat[j], wi = L.lat[i];
                const uint32_t slj = slot_of(wj), sli = slot_of(wi);
                const int tj = type_in(wj), ti = type_in(wi);
                int4 out = make_int4(0, 0, 0, 0);
                const int64_t Vj = slj >= 2 ? (int64_t)L.sV[slj] + L.dV[slj] : 0;
                if (!(slj >= 2 && Vj <= 1)) {
                    int32_t adhesion = 0, mi = 0, mj = 0;
                    for (int k = (int)glane; k < NB; k += kGroup) {
                        const uint32_t wn = L.lat[(int32_t)j + L.off[k + (k >= NB / 2 ? 1 : 0)]];
                        const int tn = type_in(wn);
                        if (wn != wi) adhesion += sm.J[ti * kMaxTypes + tn]; else ++mi;
                        if (wn != wj) adhesion -= sm.J[tj * kMaxTypes + tn]; else ++mj;
                    }
#pragma unroll
                    for (int o = kGroup / 2; o > 0; o >>= 1) {
                        adhesion += __shfl_xor_sync(gmask, adhesion, o, kGroup);
                        mi += __shfl_xor_sync(gmask, mi, o, kGroup);
                        mj += __shfl_xor_sync(gmask, mj, o, kGroup);
                    }
                    const int dAi = NB - 2 * mi, dAj = 2 * mj - NB;
                    int64_t dh = adhesion;
                    if (sli >= 2) {
                        const int64_t Vi = (int64_t)L.sV[sli] + L.dV[sli];
                        dh += (int64_t)sm.lv[ti] * (2 * (Vi - sm.vt[ti]) + 1);
                        if (PERIM) {
                            const int64_t Ai = (int64_t)L.sA[sli] + L.dA[sli];
                            dh += (int64_t)sm.lp[ti] * dAi * (2 * (Ai - sm.at[ti]) + dAi);
                        }
                    }
                    if (slj >= 2) {
                        dh += (int64_t)sm.lv[tj] * (1 - 2 * (Vj - sm.vt[tj]));
                        if (PERIM) {
                            const int64_t Aj = (int64_t)L.sA[slj] + L.dA[slj];
                            dh += (int64_t)sm.lp[tj] * dAj * (2 * (Aj - sm.at[tj]) + dAj);
                        }
                    }
                    int64_t dhq = 16 * dh;
                    if (ACT) {
                        const int tpar = sli >= 2 ? ti : tj;
                        const int64_t lam = sm.la[tpar], mxa = sm.ma[tpar];
                        if (lam != 0 && mxa != 0) {
                            const int maxi = sli >= 2 ? sm.ma[ti] : 0, maxj = slj >= 2 ? sm.ma[tj] : 0;
                            int32_t sum_i = 0, cnt_i = 0, zero_i = sli < 2, sum_j = 0, cnt_j = 0, zero_j = slj < 2;
                            for (int k = (int)glane; k < 2 * NS; k += kGroup) {
                                const bool for_i = k < NS;
                                const int kk = for_i ? k : k - NS;
                                const uint32_t wc = for_i ? wi : wj;
                                const uint32_t site = (uint32_t)((int32_t)(for_i ? i : j) + L.off[kk]);
                                if (kk != NS / 2 && L.lat[site] != wc) continue;
                                const int v = act_of(L.stamp[site], t8, for_i ? maxi : maxj);
                                if (for_i) {
                                    if (v == 0) zero_i = 1; else { sum_i += sm.ln[v]; ++cnt_i; }
                                } else {
                                    if (v == 0) zero_j = 1; else { sum_j += sm.ln[v]; ++cnt_j; }
                                }
                            }
#pragma unroll
                            for (int o = kGroup / 2; o > 0; o >>= 1) {
                                sum_i += __shfl_xor_sync(gmask, sum_i, o, kGroup);
                                cnt_i += __shfl_xor_sync(gmask, cnt_i, o, kGroup);
                                zero_i |= __shfl_xor_sync(gmask, zero_i, o, kGroup);
                                sum_j += __shfl_xor_sync(gmask, sum_j, o, kGroup);
                                cnt_j += __shfl_xor_sync(gmask, cnt_j, o, kGroup);
                                zero_j |= __shfl_xor_sync(gmask, zero_j, o, kGroup);
                            }
                            const int64_t gi = zero_i ? 0 : (int64_t)__ldg(a.expq + ((sum_i / cnt_i) >> 6));
                            const int64_t gj = zero_j ? 0 : (int64_t)__ldg(a.expq + ((sum_j / cnt_j) >> 6));
                            const int64_t num = lam * (gj - gi), den = mxa * 4096;
                            int64_t qd = num / den;
                            if (num % den != 0 && num < 0) qd -= 1;
                            dhq += qd;
                        }
                    }
                    bool ok = dhq <= 0;
                    if (!ok && dhq < a.L)
                        ok = it.y < (dhq < (int64_t)a.thr_smem ? L.thr[dhq] : __ldg(a.thr + dhq));
                    if (ok) out = make_int4((int)sli, (int)slj, dAi, dAj);
                }
                if (glane == 0) {
                    L.chg[c] = out;
                    if (out.x != out.y) {
                        L.lat[j] = (uint16_t)wi;  // no other attempt of this round reads j
                        if (ACT) L.stamp[j] = (uint8_t)(sli >= 2 ? t8 : ((a.t - 128u) & 255u));
                        ++my_accepts;
                    }
                }
            }
            prev_nc = nc;
            __syncthreads();
        }
    }
    // the last round's changes
    for (uint32_t c = threadIdx.x; c < prev_nc; c += blockDim.x) {
        const int4 ch = L.chg[c];
        if (ch.x == ch.y) continue;
        if (ch.x >= 2) { atomicAdd(L.dV + ch.x, 1); atomicAdd(L.dA + ch.x, ch.z); }
        if (ch.y >= 2) { atomicAdd(L.dV + ch.y, -1); atomicAdd(L.dA + ch.y, ch.w); }
    }
    __syncthreads();

    // write the interior back, flush the tile's tally changes
    const uint32_t TZ = DIM == 3 ? T : 1;
    for (uint32_t l = threadIdx.x; l < T * T * TZ; l += blockDim.x) {
        const uint32_t lx = l % T, ly = (l / T) % T, lz = l / (T * T);
        const uint32_t gx = (ox + lx) % a.nx, gy = (oy + ly) % a.ny, gz = DIM == 3 ? (oz + lz) % a.nz : 0;
        const uint64_t g = gx + (uint64_t)a.nx * (gy + (uint64_t)a.ny * gz);
        const uint32_t s_ = (lx + H) + W * ((ly + H) + W * (DIM == 3 ? lz + H : 0));
        const int32_t id = L.gid[slot_of(L.lat[s_])];
        a.lat[g] = ACT ? pack_word(id, L.stamp[s_]) : id;
    }
    for (uint32_t sl = 2 + threadIdx.x; sl < ns; sl += blockDim.x) {
        const int32_t g = L.gid[sl];
        if (L.dV[sl]) atomicAdd(a.Vn + g, L.dV[sl]);
        if (L.dA[sl]) atomicAdd(a.An + g, L.dA[sl]);
    }
    if (my_accepts) atomicAdd(&sm.accepts, (unsigned long long)my_accepts);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sm.accepts) atomicAdd(a.accepts, sm.accepts);
        if (sm.overflow) atomicExch(a.error_flag, 1);
    }
}

template <int DIM, bool PERIM, bool ACT>
cudaError_t launch_tile_t(const TileArgs &a, size_t dyn_smem, uint32_t n_tiles, cudaStream_t st)
{
    static size_t configured = 0;
    if (dyn_smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(tile_epoch_kernel<DIM, PERIM, ACT>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(tile_epoch_kernel<DIM, PERIM, ACT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        configured = dyn_smem;
    }
    tile_epoch_kernel<DIM, PERIM, ACT><<<n_tiles, kTileThreads, dyn_smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

size_t tile_dyn_smem(int dim, bool act, uint32_t T, uint32_t cap, uint32_t a, uint32_t thr_smem)
{
    auto al = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t W = T + 4;
    const size_t n = W * W * (dim == 3 ? W : 1);
    const size_t per = T / a;
    const size_t n_blk = per * per * (dim == 3 ? per : 1);
    return al(2 * n) + (act ? al(n) : 0) + al(4 * 2 * cap) + al(2 * 2 * cap) + 5 * al(4 * cap) + al(cap) +
           al(4 * (size_t)thr_smem) + al(8 * n_blk) + al(16 * n_blk) + al(4 * 27);
}

cudaError_t launch_tile_epoch(int dim, bool perim, bool act, const TileArgs &a, uint32_t n_tiles, cudaStream_t st)
{
    const size_t smem = tile_dyn_smem(dim, act, a.T, a.hash_cap, a.s * a.c, a.thr_smem);
    if (dim == 2) {
        if (act) return perim ? launch_tile_t<2, true, true>(a, smem, n_tiles, st) : launch_tile_t<2, false, true>(a, smem, n_tiles, st);
        return perim ? launch_tile_t<2, true, false>(a, smem, n_tiles, st) : launch_tile_t<2, false, false>(a, smem, n_tiles, st);
    }
    if (act) return perim ? launch_tile_t<3, true, true>(a, smem, n_tiles, st) : launch_tile_t<3, false, true>(a, smem, n_tiles, st);
    return perim ? launch_tile_t<3, true, false>(a, smem, n_tiles, st) : launch_tile_t<3, false, false>(a, smem, n_tiles, st);
}

}  // namespace cpmgb
