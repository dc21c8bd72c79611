// Device kernels of the GB300 CPM sweep: one round of copy attempts over the
// blocks of the active checkerboard colour, plus the bookkeeping kernels
// (tally recount and comparison, Act stamp clamp, Act read-out).
//
// One thread owns one active block for the round and makes its single copy
// attempt (Results, Fig. 3A: a barrier after every attempt; here the kernel
// boundary).  The energy change follows the paper's Methods: Eq. 1 (adhesion
// over the Moore neighbourhood, each pair counted once; volume term), Eq. 3
// (perimeter term) and Eq. 8/Eq. 9 (Act term, geometric mean), all in integers;
// Eq. 2 acceptance through the integer threshold table.
//
// Tallies are double-buffered so that every attempt of a round sees the
// tallies as they stood when the round began (deterministic form of the
// paper's atomic updates, Fig. 2B): round g reads buffer g&1 and adds both its
// own accepted changes and those of round g-1 into buffer (g+1)&1, which then
// equals the state after round g.  The change of round g-1 is carried in
// pend_prev, indexed by active-block number (equal for every colour); a
// one-byte flag per active block says whether it holds a change, so that
// only accepted copies (a few per cent) move a 16-byte entry.
#include <cstdint>

#include "cpm_internal.h"

namespace cpmgb {
namespace {

constexpr int kThreads = 256;

struct SmemTables {
    int32_t J[kMaxTypes * kMaxTypes];
    int32_t lv[kMaxTypes], vt[kMaxTypes], lp[kMaxTypes], at[kMaxTypes], la[kMaxTypes], ma[kMaxTypes];
    int32_t ln[kLnEntries];
};

__device__ __forceinline__ void load_tables(SmemTables &sm, const RoundArgs &a, bool with_ln)
{
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
    if (with_ln)
        for (int k = threadIdx.x; k < kLnEntries; k += blockDim.x) sm.ln[k] = a.ln_tab[k];
}

__device__ __forceinline__ int type_of(int32_t sigma, const uint8_t *cell_type, int obstacle_type)
{
    return sigma < 0 ? obstacle_type : (int)__ldg(cell_type + sigma);
}

// wrapped coordinates x-1, x, x+1 along an axis of extent n
__device__ __forceinline__ void around(uint32_t x, uint32_t n, uint32_t out[3])
{
    out[0] = x == 0 ? n - 1 : x - 1;
    out[1] = x;
    out[2] = x + 1 == n ? 0 : x + 1;
}

// x + d (d in -1, 0, 1) on a periodic axis of extent n, for x in [0, n)
__device__ __forceinline__ uint32_t wrap_step(uint32_t x, int d, uint32_t n)
{
    return d < 0 ? (x == 0 ? n - 1 : x - 1) : (d > 0 ? (x + 1 == n ? 0 : x + 1) : x);
}

// A lattice word of the round kernels.  With Act and areas of edge 8 or
// more, through the streaming cache path (ld.global.cs, evict first): the
// active blocks of a round are then 8 sites apart, a round touches each
// line of its stencils about once, and the tallies and type tables it also
// reads stay in L2 longer (4% faster on the 1024^3 tissue with a = 8).  With
// smaller areas the stencils of neighbouring blocks share lines and plain
// loads are faster (6% on the same tissue with a = 4).
template <bool ACT>
__device__ __forceinline__ int32_t lat_word(const RoundArgs &a, uint32_t site)
{
    return ACT && a.stream_loads ? __ldcs(a.lat + site) : a.lat[site];
}

// Act value of a site from its stamp: Max - age, clipped at 0.
__device__ __forceinline__ int act_value(uint32_t stamp, uint32_t t8, int max_act)
{
    const int age = (int)((t8 - stamp) & 255u);
    const int v = max_act - age;
    return v > 0 ? v : 0;
}

// Integer geometric mean of Act (Q16) over site (x,y,z) with id sigma and its
// same-cell Moore neighbours: EXPQ[(sum LN / count) >> 6]; 0 for the medium
// or when any of those Act values is 0.  ROLL is the code-size level of the
// calling kernel (see round_attempt): the stencil loops are rolled from the
// outside in as it rises; the visiting order and the result do not change.
template <int DIM, int ROLL>
__device__ int64_t gm_q(const RoundArgs &a, const SmemTables &sm, uint32_t x, uint32_t y, uint32_t z, int32_t sigma,
                        int max_act)
{
    if (sigma <= 0) return 0;
    int32_t sum = 0, cnt = 0;
#pragma unroll(ROLL >= 1 ? 1 : 3)
    for (int dz = (DIM == 3 ? 0 : 1); dz < (DIM == 3 ? 3 : 2); ++dz) {
        const uint32_t zz = DIM == 3 ? wrap_step(z, dz - 1, a.nz) : 0;
#pragma unroll(ROLL >= 2 ? 1 : 3)
        for (int dy = 0; dy < 3; ++dy) {
            const uint32_t row = a.nx * (wrap_step(y, dy - 1, a.ny) + a.ny * zz);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const uint32_t site = wrap_step(x, dx - 1, a.nx) + row;
                const bool centre = dx == 1 && dy == 1 && dz == 1;
                const int32_t w = lat_word<true>(a, site);
                if (!centre && cell_id(w) != sigma) continue;
                const int v = act_value(word_stamp(w), a.t & 255u, max_act);
                if (v == 0) return 0;
                sum += sm.ln[v];
                cnt += 1;
            }
        }
    }
    return (int64_t)__ldg(a.expq + ((sum / cnt) >> 6));
}

__device__ __forceinline__ int64_t floor_div_pos(int64_t num, int64_t den)
{
    int64_t q = num / den;
    if (num % den != 0 && num < 0) q -= 1;
    return q;
}

// Motility terms (Eq. 4, Eq. 5) of the copy from the source (stencil index
// ox, oy, oz around the target) into the target, in 1/16 energy units: the
// moving cell is si (sj when si is the medium), d = target - source, and
// each term is floor(e) with e formed by the same rounded double operations,
// in the same order, as the replay: chemotaxis
// e = ((double)(-16 lambda (d . C_q)) / 16384) * (1/|d|), persistence
// e = ((d_x p_x + d_y p_y + d_z p_z) * (double)(-16 lambda)) * (1/|d|).
// Kept out of line: the round kernels call it only when a field or a
// persistence direction is set, and inlining its FP64 code into every round
// kernel enlarges them (instruction-fetch stalls).
template <int DIM>
__device__ __noinline__ int64_t motility_q(const RoundArgs &a, int32_t si, int32_t sj, int ti, int tj, int ox,
                                              int oy, int oz, uint32_t isite)
{
    const int32_t m = si > 0 ? si : sj;
    const int tp = si > 0 ? ti : tj;
    const int dx = 1 - ox, dy = 1 - oy, dz = DIM == 3 ? 1 - oz : 0;
    const double il = a.tp.inv_len[dx * dx + dy * dy + dz * dz];
    int64_t dh = 0;
    if (a.chem && a.tp.lambda_chem[tp] != 0) {
        const int16_t *c = a.chem + (size_t)isite * DIM;
        int64_t dc = (int64_t)dx * c[0] + (int64_t)dy * c[1];
        if (DIM == 3) dc += (int64_t)dz * c[2];
        const double e = __dmul_rn((double)(-16 * (int64_t)a.tp.lambda_chem[tp] * dc) / 16384.0, il);
        dh += (int64_t)floor(e);
    }
    if (a.pers_dir && a.tp.lambda_pers[tp] != 0 && m > 0) {
        const double *ph = a.pers_dir + 3 * (size_t)m;
        double sd = __dmul_rn((double)dx, ph[0]);
        sd = __dadd_rn(sd, __dmul_rn((double)dy, ph[1]));
        sd = __dadd_rn(sd, __dmul_rn((double)dz, ph[2]));
        const double e = __dmul_rn(__dmul_rn(sd, (double)(-16 * (int64_t)a.tp.lambda_pers[tp])), il);
        dh += (int64_t)floor(e);
    }
    return dh;
}

// Composite variable tracking (Eq. 11).  A copy into site j adds j to sigma_i and
// removes it from sigma_j, each at its periodic image nearest that cell's centroid
// as the round began (Sc / Vc); the image shifts (-3..3 per axis, 3 bits each:
// sigma_i's in bits 0..8, sigma_j's in bits 9..17) travel with the pending change,
// so that the next round adds the same amounts to the other buffer.
template <int DIM>
__device__ __noinline__ int2 track_accept(const RoundArgs &a, int32_t si, int32_t sj, uint32_t j, uint32_t jx,
                                          uint32_t jy, uint32_t jz)
{
    uint32_t bits = 0;
    const int64_t Vi = si > 0 ? a.Vc[si] : 0, Vj = sj > 0 ? a.Vc[sj] : 0;
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int64_t x = d == 0 ? jx : (d == 1 ? jy : jz);
        const int64_t n = d == 0 ? a.nx : (d == 1 ? a.ny : a.nz);
        if (si > 0) {
            const int64_t k = track_image_shift(x, a.Sc[3 * si + d], Vi, n);
            atomicAdd((unsigned long long *)(a.Sn + 3 * si + d), (unsigned long long)(x + n * k));
            bits |= (uint32_t)(k + 3) << (3 * d);
        }
        if (sj > 0) {
            const int64_t k = track_image_shift(x, a.Sc[3 * sj + d], Vj, n);
            atomicAdd((unsigned long long *)(a.Sn + 3 * sj + d), (unsigned long long)(-(x + n * k)));
            bits |= (uint32_t)(k + 3) << (9 + 3 * d);
        }
    }
    return make_int2((int32_t)j, (int32_t)bits);
}

// the previous round's tracked change (see track_accept) into the other buffer
template <int DIM>
__device__ __noinline__ void track_carry(const RoundArgs &a, int32_t si, int32_t sj, int2 e)
{
    const uint32_t j = (uint32_t)e.x, bits = (uint32_t)e.y;
    const uint32_t jx = j % a.nx, jy = (j / a.nx) % a.ny, jz = j / (a.nx * a.ny);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        const int64_t x = d == 0 ? jx : (d == 1 ? jy : jz);
        const int64_t n = d == 0 ? a.nx : (d == 1 ? a.ny : a.nz);
        if (si > 0) {
            const int64_t k = (int64_t)((bits >> (3 * d)) & 7u) - 3;
            atomicAdd((unsigned long long *)(a.Sn + 3 * si + d), (unsigned long long)(x + n * k));
        }
        if (sj > 0) {
            const int64_t k = (int64_t)((bits >> (9 + 3 * d)) & 7u) - 3;
            atomicAdd((unsigned long long *)(a.Sn + 3 * sj + d), (unsigned long long)(-(x + n * k)));
        }
    }
}

// One copy attempt of active block (ix, iy, iz) (active index i) in the round
// described by a; also carries the previous round's change of index i into
// the next tallies.  Returns whether the copy was accepted.
//
// The target's Act geometric mean (Eq. 9) is gathered in the neighbour sum,
// which reads the same 3^3 window around the target; only the source's mean
// reads a window of its own, and only when the Act term decides the test.
//
// ROLL is a code-size level.  The fully unrolled stencil loops make the Act
// kernels large enough that instruction fetch stalls them (a warp's lanes sit
// in different phases of the attempt), so those kernels roll loops from the
// outside in: level 1 (single-lattice Act kernels, batched 2D Act kernel)
// rolls the outer (z) loop of the neighbour sum and keeps the source's
// geometric mean unrolled (its 27 loads issue together); level 2 (batched 3D
// Act kernel, whose CTAs mix lattices) also rolls the middle (y) loop and
// rolls the geometric mean like the neighbour sum.  Level 0 (kernels without
// Act) stays fully unrolled.  The level changes only the code layout: every
// sum visits the same sites, and integer sums do not depend on the order.
template <int DIM, bool PERIM, bool ACT, int ROLL, bool TRACK = false>
__device__ __forceinline__ bool round_attempt(const RoundArgs &a, const SmemTables &sm, uint32_t ix, uint32_t iy,
                                              uint32_t iz, uint32_t i)
{
    constexpr int NB = DIM == 3 ? 26 : 8;
    bool accepted = false;

        // the active block of this thread
        const uint32_t bx = ix * a.c + a.cx, by = iy * a.c + a.cy, bz = DIM == 3 ? iz * a.c + a.cz : 0;
        const uint32_t b = bx + a.nbx * (by + a.nby * bz);

        const Philox4 w = philox4x32_10(b, a.r, a.t, a.sp, a.key0, a.key1);
        const uint32_t jl = draw_below(w.v[0], a.sd);
        const uint32_t jx = bx * a.s + jl % a.s;
        const uint32_t jy = by * a.s + (jl / a.s) % a.s;
        const uint32_t jz = DIM == 3 ? bz * a.s + jl / (a.s * a.s) : 0;
        const uint32_t n = draw_below(w.v[1], NB);
        const uint32_t idx = n + (n >= NB / 2 ? 1u : 0u);  // skip the centre of the 3^d stencil
        const int ox = (int)(idx % 3), oy = (int)((idx / 3) % 3), oz = DIM == 3 ? (int)(idx / 9) : 1;

        // wrapped coordinates are computed, not indexed from small arrays: an array
        // indexed by a run-time value would live in local memory
        const uint32_t j = jx + a.nx * (jy + a.ny * jz);
        const uint32_t ix_ = wrap_step(jx, ox - 1, a.nx), iy_ = wrap_step(jy, oy - 1, a.ny);
        const uint32_t iz_ = DIM == 3 ? wrap_step(jz, oz - 1, a.nz) : 0;
        const uint32_t isite = ix_ + a.nx * (iy_ + a.ny * iz_);

        // everything above depends on the launch arguments only; the lattice, flags and
        // tallies below are the previous round's output, so a round launched as a
        // programmatic dependent of the previous one waits for it here
        if (a.pdl) asm volatile("griddepcontrol.wait;" ::: "memory");
        // the previous round's accepted change goes into the next tallies
        if (a.flag_prev[i]) {
            const int4 e = a.pend_prev[i];
            if (e.x > 0) { atomicAdd(a.Vn + e.x, 1); atomicAdd(a.An + e.x, e.z); }
            if (e.y > 0) { atomicAdd(a.Vn + e.y, -1); atomicAdd(a.An + e.y, e.w); }
            if (TRACK) track_carry<DIM>(a, e.x, e.y, a.tpend_prev[i]);
        }
        const int32_t wj = lat_word<ACT>(a, j);
        const int32_t sj = cell_id(wj);
        const int32_t si = cell_id(lat_word<ACT>(a, isite));

        if (si != sj && si >= 0 && sj >= 0) {
            const int32_t Vj = sj > 0 ? a.Vc[sj] : 0;
            if (!(sj > 0 && Vj <= 1)) {
                const int ti = type_of(si, a.cell_type, a.tp.obstacle_type);
                const int tj = type_of(sj, a.cell_type, a.tp.obstacle_type);
                int32_t adhesion = 0;
                int mi = 0, mj = 0;
                // target's Act log-sum over its same-cell 3^3 window (centre first), gathered in
                // the neighbour sum; negative once a zero Act value is met (the mean is then 0)
                const int maxj = ACT && sj > 0 ? (int)sm.ma[tj] : 0;
                int32_t lsj = 0;
                if (ACT) {
                    const int v = act_value(word_stamp(wj), a.t & 255u, maxj);
                    lsj = v == 0 ? INT32_MIN / 2 : (int32_t)sm.ln[v];
                }
#pragma unroll(ROLL >= 1 ? 1 : 3)
                for (int dz = (DIM == 3 ? 0 : 1); dz < (DIM == 3 ? 3 : 2); ++dz) {
                    const uint32_t zz = DIM == 3 ? wrap_step(jz, dz - 1, a.nz) : 0;
#pragma unroll(ROLL >= 2 ? 1 : 3)
                    for (int dy = 0; dy < 3; ++dy) {
                        const uint32_t row = a.nx * (wrap_step(jy, dy - 1, a.ny) + a.ny * zz);
#pragma unroll
                        for (int dx = 0; dx < 3; ++dx) {
                            if (dx == 1 && dy == 1 && dz == 1) continue;
                            const int32_t wn = lat_word<ACT>(a, wrap_step(jx, dx - 1, a.nx) + row);
                            const int32_t sn = cell_id(wn);
                            const int tn = type_of(sn, a.cell_type, a.tp.obstacle_type);
                            if (sn != si) adhesion += sm.J[ti * kMaxTypes + tn]; else ++mi;
                            if (sn != sj) adhesion -= sm.J[tj * kMaxTypes + tn];
                            else {
                                ++mj;
                                if (ACT) {
                                    const int v = act_value(word_stamp(wn), a.t & 255u, maxj);
                                    lsj = v == 0 ? INT32_MIN / 2 : lsj + (int32_t)sm.ln[v];
                                }
                            }
                        }
                    }
                }
                const int dAi = NB - 2 * mi, dAj = 2 * mj - NB;
                int64_t dh = adhesion;
                if (si > 0) {
                    const int64_t Vi = a.Vc[si];
                    dh += (int64_t)sm.lv[ti] * (2 * (Vi - sm.vt[ti]) + 1);
                    if (PERIM) {
                        const int64_t Ai = a.Ac[si];
                        dh += (int64_t)sm.lp[ti] * dAi * (2 * (Ai - sm.at[ti]) + dAi);
                    }
                }
                if (sj > 0) {
                    dh += (int64_t)sm.lv[tj] * (1 - 2 * ((int64_t)Vj - sm.vt[tj]));
                    if (PERIM) {
                        const int64_t Aj = a.Ac[sj];
                        dh += (int64_t)sm.lp[tj] * dAj * (2 * (Aj - sm.at[tj]) + dAj);
                    }
                }
                int64_t dhq = 16 * dh;
                if (a.chem || a.pers_dir) dhq += motility_q<DIM>(a, si, sj, ti, tj, ox, oy, oz, isite);
                // decided: 1 accept, 0 reject, -1 open
                int decided = -1;
                if (ACT) {
                    const int tp = si > 0 ? ti : tj;
                    const int64_t lam = sm.la[tp], mx = sm.ma[tp];
                    if (lam != 0 && mx != 0) {
                        // the Act term lies in [floor(-lam Gmax_i / (Max 4096)), floor(lam Gmax_j / (Max 4096))]
                        // (GM in [0, Gmax] per cell, lambda >= 0); when every value in that range gives the same
                        // outcome of the test below (THR is non-increasing), the geometric means are not needed
                        const int64_t lo = dhq + floor_div_pos(-lam * (si > 0 ? a.tp.gm_max[ti] : 0), mx * 4096);
                        const int64_t hi = dhq + floor_div_pos(lam * (sj > 0 ? a.tp.gm_max[tj] : 0), mx * 4096);
                        if (hi <= 0) decided = 1;
                        else if (lo >= a.L || (lo > 0 && w.v[2] >= __ldg(a.thr + lo))) decided = 0;
                        else {
                            // target: the log-sum gathered above over the sites gm_q would visit
                            // (the centre and the mj same-cell neighbours)
                            const int64_t gj =
                                sj > 0 && lsj >= 0 ? (int64_t)__ldg(a.expq + ((lsj / (mj + 1)) >> 6)) : 0;
                            const int64_t gi = gm_q<DIM, (ROLL >= 2 ? ROLL : 0)>(a, sm, ix_, iy_, iz_, si,
                                                                                 si > 0 ? sm.ma[ti] : 0);
                            dhq += floor_div_pos(lam * (gj - gi), mx * 4096);
                        }
                    }
                }
                const bool ok = decided >= 0 ? decided == 1 : (dhq <= 0 || (dhq < a.L && w.v[2] < __ldg(a.thr + dhq)));
                if (ok) {
                    // a copy stamps the site with this MCS (a medium copy: age 128, no activity)
                    a.lat[j] = ACT && a.packed ? pack_word(si, si > 0 ? (a.t & 255u) : ((a.t - 128u) & 255u)) : si;
                    if (si > 0) { atomicAdd(a.Vn + si, 1); atomicAdd(a.An + si, dAi); }
                    if (sj > 0) { atomicAdd(a.Vn + sj, -1); atomicAdd(a.An + sj, dAj); }
                    a.pend_cur[i] = make_int4(si, sj, dAi, dAj);
                    if (TRACK) a.tpend_cur[i] = track_accept<DIM>(a, si, sj, j, jx, jy, jz);
                    accepted = true;
                }
            }
        }
        a.flag_cur[i] = accepted ? 1 : 0;
    return accepted;
}

// Resident CTAs per SM (register budget): the round kernel is latency-bound.
// Measured on GB300 in same-box A/B runs: without Act, four CTAs of 256
// (64 registers) are fastest (256^3 cube cells: 1.05 ms per MCS against 1.31
// at 32 registers); with Act, eight (32 registers, a few spills) are fastest
// (1024^3 fibre tissue: slower at 40, 48 and 64 registers, whose lower
// occupancy costs more than the spills they save).
#ifndef CPM_ROUND_MIN_BLOCKS
#define CPM_ROUND_MIN_BLOCKS 4
#endif
#ifndef CPM_ROUND_MIN_BLOCKS_ACT
#define CPM_ROUND_MIN_BLOCKS_ACT 8
#endif

// TRACK: composite variable tracking on (a.Sc, a.Sn, a.tpend_* set), a kernel
// of its own so that the sweep without it carries none of its code
template <int DIM, bool PERIM, bool ACT, bool TRACK>
__global__ void __launch_bounds__(kThreads, ACT ? CPM_ROUND_MIN_BLOCKS_ACT : CPM_ROUND_MIN_BLOCKS)
    round_kernel(const RoundArgs a)
{
    __shared__ SmemTables sm;
    // the next round may place its CTAs on free SM slots from now on; they compute
    // their sites and random numbers, then wait for this round to finish
    if (a.pdl) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    load_tables(sm, a, ACT);
    __syncthreads();

    // each CTA covers a brick of bx_ x by_ x bz_ active blocks, so that the
    // stencils of its threads overlap in L1
    const uint32_t bx_ = a.brick_x, by_ = a.brick_y, bz_ = DIM == 3 ? a.brick_z : 1;
    const uint32_t nbrx = (a.nax + bx_ - 1) / bx_, nbry = (a.nay + by_ - 1) / by_;
    const uint32_t brick = blockIdx.x;
    const uint32_t tx = threadIdx.x % bx_, ty = (threadIdx.x / bx_) % by_, tz = threadIdx.x / (bx_ * by_);
    const uint32_t ix = (brick % nbrx) * bx_ + tx;
    const uint32_t iy = ((brick / nbrx) % nbry) * by_ + ty;
    const uint32_t iz = (brick / (nbrx * nbry)) * bz_ + tz;
    const uint32_t naz = a.n_active / (a.nax * a.nay);
    const bool valid = threadIdx.x < bx_ * by_ * bz_ && ix < a.nax && iy < a.nay && iz < naz;
    const uint32_t i = ix + a.nax * (iy + a.nay * iz);
    bool accepted = false;
    if (valid) {
        accepted = round_attempt<DIM, PERIM, ACT, ACT ? 1 : 0, TRACK>(a, sm, ix, iy, iz, i);
    }
    const unsigned m = __ballot_sync(0xffffffffu, accepted);
    if ((threadIdx.x & 31) == 0 && m != 0) atomicAdd(a.accepts, (unsigned long long)__popc(m));
}

// Batched round: every CTA takes one (lattice, chunk of 128 active blocks)
// item and runs that lattice's round number g_start + q, exactly as the
// single-lattice round kernel would (same colour, counters and tallies).
// Register budget of the batched round as for round_kernel: with Act eight
// CTAs of 256 per SM (the 512-member ensemble: 31.2 ms per MCS against 36.7
// at two CTAs), without Act four.
#ifndef CPM_BATCH_MIN_BLOCKS
#define CPM_BATCH_MIN_BLOCKS 4
#endif
#ifndef CPM_BATCH_MIN_BLOCKS_ACT
#define CPM_BATCH_MIN_BLOCKS_ACT 8
#endif
// One (lattice, brick) item of batch round q: lattice it.x's round number
// g_start + q, exactly as the single-lattice round kernel would run it (same
// colour, counters and tallies).  ra and sm are the CTA's shared set-up.
template <int DIM, bool PERIM, bool ACT, bool TRACK = false>
__device__ __forceinline__ void batch_round_item(RoundArgs &ra, SmemTables &sm, const BatchLattice *lats, int2 it,
                                                 uint32_t q)
{
    __syncthreads();  // the previous item of this CTA is done with ra and sm
    if (threadIdx.x == 0) {
        const BatchLattice &L = lats[it.x];
        ra = L.base;
        const uint64_t t = (uint64_t)L.t_start + q / L.R;
        const uint32_t mm = q % L.R;
        const uint32_t sp = mm / L.k, r = mm % L.k;
        // colour: Fisher-Yates over the C colours of cycle sp / C, swap i from counter (i, cycle, t, 1<<24)
        uint32_t perm[27];
        for (uint32_t c = 0; c < L.C; ++c) perm[c] = c;
        for (uint32_t k = L.C - 1; k >= 1; --k) {
            const Philox4 w = philox4x32_10(k, sp / L.C, (uint32_t)t, 1u << 24, ra.key0, ra.key1);
            const uint32_t j = draw_below(w.v[0], k + 1);
            const uint32_t tmp = perm[k];
            perm[k] = perm[j];
            perm[j] = tmp;
        }
        const uint32_t col = perm[sp % L.C];
        ra.cx = col % ra.c;
        ra.cy = (col / ra.c) % ra.c;
        ra.cz = col / (ra.c * ra.c);
        ra.t = (uint32_t)t;
        ra.sp = sp;
        ra.r = r;
        const uint32_t par = (uint32_t)((L.g_start + q) & 1u);
        ra.Vc = L.V[par];
        ra.Ac = L.A[par];
        ra.Vn = L.V[par ^ 1u];
        ra.An = L.A[par ^ 1u];
        ra.pend_prev = L.pend[par ^ 1u];
        ra.pend_cur = L.pend[par];
        ra.flag_prev = L.flag[par ^ 1u];
        ra.flag_cur = L.flag[par];
        if (TRACK) {
            ra.Sc = L.S[par];
            ra.Sn = L.S[par ^ 1u];
            ra.tpend_prev = L.tpend[par ^ 1u];
            ra.tpend_cur = L.tpend[par];
        }
    }
    __syncthreads();
    load_tables(sm, ra, ACT);
    __syncthreads();
    // brick it.y of bx x by x bz active blocks (bricks in x-fastest order)
    const uint32_t bx_ = ra.brick_x, by_ = ra.brick_y, bz_ = DIM == 3 ? ra.brick_z : 1;
    const uint32_t nbrx = (ra.nax + bx_ - 1) / bx_, nbry = (ra.nay + by_ - 1) / by_;
    const uint32_t brick = (uint32_t)it.y;
    const uint32_t tx = threadIdx.x % bx_, ty = (threadIdx.x / bx_) % by_, tz = threadIdx.x / (bx_ * by_);
    const uint32_t ix = (brick % nbrx) * bx_ + tx;
    const uint32_t iy = ((brick / nbrx) % nbry) * by_ + ty;
    const uint32_t iz = (brick / (nbrx * nbry)) * bz_ + tz;
    const uint32_t naz = ra.n_active / (ra.nax * ra.nay);
    bool accepted = false;
    if (threadIdx.x < bx_ * by_ * bz_ && ix < ra.nax && iy < ra.nay && iz < naz) {
        const uint32_t i = ix + ra.nax * (iy + ra.nay * iz);
        accepted = round_attempt<DIM, PERIM, ACT, ACT ? (DIM == 3 ? 2 : 1) : 0, TRACK>(ra, sm, ix, iy, iz, i);
    }
    const unsigned m = __ballot_sync(0xffffffffu, accepted);
    if ((threadIdx.x & 31) == 0 && m != 0) atomicAdd(ra.accepts, (unsigned long long)__popc(m));
}

// Batched round: every CTA takes one (lattice, chunk of active blocks) item.
// Register budget of the batched round as for round_kernel: with Act eight
// CTAs of 256 per SM (the 512-member ensemble: 31.2 ms per MCS against 36.7
// at two CTAs), without Act four.
#ifndef CPM_BATCH_MIN_BLOCKS
#define CPM_BATCH_MIN_BLOCKS 4
#endif
#ifndef CPM_BATCH_MIN_BLOCKS_ACT
#define CPM_BATCH_MIN_BLOCKS_ACT 8
#endif
// TRACK: every member keeps its tracked centroid sums (BatchLattice::S)
template <int DIM, bool PERIM, bool ACT, bool TRACK>
__global__ void __launch_bounds__(kBatchMaxThreads, ACT ? CPM_BATCH_MIN_BLOCKS_ACT : CPM_BATCH_MIN_BLOCKS)
    batch_round_kernel(const BatchLattice *lats, const int2 *items, uint32_t q)
{
    __shared__ RoundArgs ra;
    __shared__ SmemTables sm;
    batch_round_item<DIM, PERIM, ACT, TRACK>(ra, sm, lats, items[blockIdx.x], q);
}

// Stamps whose age is 128 or more are reset to age exactly 128, so that ages
// stay below 256 until the next clamp (run every 64 MCS).  Obstacle words are
// left as they are (their stamp is never read).
__device__ __forceinline__ void clamp_word(int32_t *p, uint32_t t8)
{
    const int32_t w = *p;
    if (cell_id(w) < 0) return;
    const uint32_t age = (t8 - word_stamp(w)) & 255u;
    if (age >= 128u) *p = pack_word(cell_id(w), (t8 - 128u) & 255u);
}

// Act stamp clamp of one (member, chunk of 65,536 sites) item, for a member
// whose MCS t_start is a multiple of 64 (run at the start of its MCS).
__device__ __forceinline__ void batch_clamp_item(const BatchLattice *lats, int2 it)
{
    const BatchLattice &L = lats[it.x];
    if (!L.base.packed || (L.t_start % 64) != 0) return;
    const uint64_t n = (uint64_t)L.base.nx * L.base.ny * L.base.nz;
    const uint32_t t8 = (uint32_t)L.t_start & 255u;
    const uint64_t lo = (uint64_t)it.y * 65536u, hi = lo + 65536u < n ? lo + 65536u : n;
    for (uint64_t x = lo + threadIdx.x; x < hi; x += blockDim.x) clamp_word(L.base.lat + x, t8);
}


__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier of a co-resident (cooperative) grid on a 64-bit counter
// that starts at 0 (a call may pass billions of arrivals): the k-th barrier
// waits for k * gridDim.x arrivals.  The wait is bounded: after max_polls
// polls (about 100 ns apart) the CTA records the timeout in *err and the
// barrier returns false; the caller then returns.
__device__ __forceinline__ bool grid_barrier(unsigned long long *bar, unsigned long long target, long long max_polls,
                                             int *err, int &ok_s)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1ull);
        int ok = 1;
        long long polls = 0;
        while (ld_acquire_gpu(bar) < target) {
            if (polls++ >= max_polls) {
                ok = 0;
                atomicExch(err, 1);
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// The persistent batched MCS loop: n_mcs MCS of every member in one
// cooperative launch.  Per MCS: the Act clamp items, then rounds q = 0 ..
// r_max - 1 over the items of the members that still have rounds
// (upto_q[q] items), then the advance of every member's MCS and round
// counters, each phase closed by a grid barrier.  The work and its order
// within a phase are those of the per-round launches, so the result is the
// same bit for bit.
template <int DIM, bool PERIM, bool ACT>
__global__ void __launch_bounds__(kBatchMaxThreads, ACT ? CPM_BATCH_MIN_BLOCKS_ACT : CPM_BATCH_MIN_BLOCKS)
    batch_loop_kernel(BatchLattice *lats, uint32_t n_lats, const int2 *items, const uint32_t *upto_q, uint32_t r_max,
                      const int2 *clamp, uint32_t n_clamp, uint32_t n_mcs, unsigned long long *bar, unsigned *next,
                      long long max_polls, int *err, int test_absent)
{
    __shared__ RoundArgs ra;
    __shared__ SmemTables sm;
    __shared__ int ok_s;
    __shared__ uint32_t claim_s;
    // test of the timeout path: the first CTA never arrives, so the others' first barrier wait runs out
    if (test_absent && blockIdx.x == 0) return;
    unsigned long long target = 0;
    for (uint32_t m = 0; m < n_mcs; ++m) {
        if (ACT) {
            for (uint32_t c = blockIdx.x; c < n_clamp; c += gridDim.x) batch_clamp_item(lats, clamp[c]);
            target += gridDim.x;
            if (!grid_barrier(bar, target, max_polls, err, ok_s)) return;
        }
        for (uint32_t q = 0; q < r_max; ++q) {
            const uint32_t n_items = upto_q[q];
            // items are claimed one at a time from the round's counter, so that CTAs that drew cheap items
            // take more of them (a fixed grid-stride split leaves the round waiting for the unluckiest CTA)
            for (;;) {
                __syncthreads();
                if (threadIdx.x == 0) claim_s = atomicAdd(next + q, 1u);
                __syncthreads();
                const uint32_t k = claim_s;
                if (k >= n_items) break;
                batch_round_item<DIM, PERIM, ACT>(ra, sm, lats, items[k], q);
            }
            target += gridDim.x;
            if (!grid_barrier(bar, target, max_polls, err, ok_s)) return;
        }
        if (blockIdx.x == 0) {
            for (uint32_t l = threadIdx.x; l < n_lats; l += blockDim.x) {
                lats[l].t_start += 1;
                lats[l].g_start += lats[l].R;
            }
            for (uint32_t q = threadIdx.x; q < r_max; q += blockDim.x) next[q] = 0;  // the next MCS claims anew
        }
        target += gridDim.x;
        if (!grid_barrier(bar, target, max_polls, err, ok_s)) return;
    }
}

template <int DIM>
__global__ void recount_kernel(const int32_t *__restrict__ lat, int32_t *V, int32_t *A, uint32_t nx, uint32_t ny,
                               uint32_t nz, uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t s = cell_id(lat[x]);
        if (s <= 0) continue;
        const uint32_t px = (uint32_t)(x % nx), py = (uint32_t)((x / nx) % ny), pz = (uint32_t)(x / ((uint64_t)nx * ny));
        uint32_t xs[3], ys[3], zs[3];
        around(px, nx, xs);
        around(py, ny, ys);
        if (DIM == 3) around(pz, nz, zs); else zs[0] = zs[1] = zs[2] = 0;
        int cnt = 0;
        for (int dz = (DIM == 3 ? 0 : 1); dz < (DIM == 3 ? 3 : 2); ++dz)
            for (int dy = 0; dy < 3; ++dy)
                for (int dx = 0; dx < 3; ++dx) {
                    if (dx == 1 && dy == 1 && dz == 1) continue;
                    cnt += cell_id(lat[xs[dx] + nx * (ys[dy] + ny * zs[dz])]) != s;
                }
        atomicAdd(V + s, 1);
        atomicAdd(A + s, cnt);
    }
}

__global__ void compare_kernel(const int32_t *V, const int32_t *A, const int32_t *V2, const int32_t *A2, int32_t n,
                               unsigned long long *n_bad)
{
    for (int32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
        if (k > 0 && (V[k] != V2[k] || A[k] != A2[k])) atomicAdd(n_bad, 1ull);
}

__global__ void clamp_kernel(int32_t *lat, uint64_t n, uint32_t t)
{
    const uint32_t t8 = t & 255u;
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        clamp_word(lat + x, t8);
}

__global__ void act_values_kernel(const int32_t *lat, const uint8_t *cell_type, TypeParams tp, uint64_t n,
                                  uint32_t t_last, uint8_t *out)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x) {
        const int32_t w = lat[x];
        const int32_t s = cell_id(w);
        int v = 0;
        if (s > 0) v = act_value(word_stamp(w), t_last & 255u, tp.max_act[cell_type[s]]);
        out[x] = (uint8_t)v;
    }
}

__global__ void unpack_ids_kernel(const int32_t *lat, int32_t *ids, uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        ids[x] = cell_id(lat[x]);
}

__global__ void pack_ids_kernel(int32_t *lat, const int32_t *ids, const uint8_t *stamps, uint64_t n)
{
    for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
        lat[x] = pack_word(ids[x], stamps ? (uint32_t)stamps[x] : word_stamp(lat[x]));
}

unsigned grid_for(uint64_t n, unsigned threads)
{
    uint64_t g = (n + threads - 1) / threads;
    if (g > 152ull * 64) g = 152ull * 64;
    return (unsigned)(g == 0 ? 1 : g);
}

template <int DIM, bool PERIM, bool ACT, bool TRACK>
cudaError_t launch_round_t(const RoundArgs &a, cudaStream_t st)
{
    const uint32_t naz = a.n_active / (a.nax * a.nay);
    const uint32_t bz = DIM == 3 ? a.brick_z : 1;
    const unsigned blocks = ((a.nax + a.brick_x - 1) / a.brick_x) * ((a.nay + a.brick_y - 1) / a.brick_y) *
                            ((naz + bz - 1) / bz);
    const unsigned threads = a.brick_x * a.brick_y * bz;
    if (!a.pdl) {
        round_kernel<DIM, PERIM, ACT, TRACK><<<blocks, threads, 0, st>>>(a);
        return cudaGetLastError();
    }
    // programmatic dependent launch: the CTAs of this round may start while the
    // previous kernel of the stream drains (it allows it once all its CTAs have
    // started); they wait for its completion before they touch the lattice
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, round_kernel<DIM, PERIM, ACT, TRACK>, a);
}

template <int DIM, bool PERIM, bool ACT>
cudaError_t launch_round_t(const RoundArgs &a, cudaStream_t st)
{
    return a.Sc ? launch_round_t<DIM, PERIM, ACT, true>(a, st) : launch_round_t<DIM, PERIM, ACT, false>(a, st);
}

}  // namespace

cudaError_t launch_round(int dim, bool perim, bool act, const RoundArgs &a, cudaStream_t st)
{
    if (dim == 2) {
        if (act) return perim ? launch_round_t<2, true, true>(a, st) : launch_round_t<2, false, true>(a, st);
        return perim ? launch_round_t<2, true, false>(a, st) : launch_round_t<2, false, false>(a, st);
    }
    if (act) return perim ? launch_round_t<3, true, true>(a, st) : launch_round_t<3, false, true>(a, st);
    return perim ? launch_round_t<3, true, false>(a, st) : launch_round_t<3, false, false>(a, st);
}

__global__ void batch_clamp_kernel(const BatchLattice *lats, const int2 *items)
{
    batch_clamp_item(lats, items[blockIdx.x]);
}

// End of one batch MCS: every member moves to its next MCS.
__global__ void batch_advance_kernel(BatchLattice *lats, uint32_t n)
{
    for (uint32_t l = blockIdx.x * blockDim.x + threadIdx.x; l < n; l += gridDim.x * blockDim.x) {
        lats[l].t_start += 1;
        lats[l].g_start += lats[l].R;
    }
}

cudaError_t launch_batch_clamp(const BatchLattice *lats, const int2 *items, uint32_t n_items, cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    batch_clamp_kernel<<<n_items, 256, 0, st>>>(lats, items);
    return cudaGetLastError();
}

cudaError_t launch_batch_advance(BatchLattice *lats, uint32_t n, cudaStream_t st)
{
    batch_advance_kernel<<<(n + 255) / 256, 256, 0, st>>>(lats, n);
    return cudaGetLastError();
}

template <int DIM, bool PERIM, bool ACT>
cudaError_t launch_batch_loop_t(const BatchLoopArgs &p, uint32_t threads, cudaStream_t st, uint32_t *grid_out)
{
    auto kern = batch_loop_kernel<DIM, PERIM, ACT>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (int)threads, 0);
    if (e != cudaSuccess) return e;
    uint64_t grid = (uint64_t)sms * (uint64_t)(per_sm > 0 ? per_sm : 1);
    if (grid > p.max_items) grid = p.max_items;
    if (grid < 2 && p.test_absent) grid = 2;  // someone must wait for the absent CTA
    if (grid < 1) grid = 1;
    *grid_out = (uint32_t)grid;
    BatchLattice *lats = p.lats;
    uint32_t n_lats = p.n_lats, r_max = p.r_max, n_clamp = p.n_clamp, n_mcs = p.n_mcs;
    const int2 *items = p.items, *clamp = p.clamp;
    const uint32_t *upto = p.upto_q;
    unsigned long long *bar = p.bar;
    unsigned *next = p.next;
    long long polls = p.max_polls;
    int *err = p.err;
    int absent = p.test_absent;
    void *args[] = {&lats, &n_lats, &items, &upto, &r_max, &clamp, &n_clamp, &n_mcs, &bar, &next, &polls, &err,
                    &absent};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3((unsigned)grid), dim3(threads), args, 0, st);
}

cudaError_t launch_batch_loop(int dim, bool perim, bool act, const BatchLoopArgs &p, uint32_t threads, cudaStream_t st,
                              uint32_t *grid_out)
{
    if (dim == 2) {
        if (act) return perim ? launch_batch_loop_t<2, true, true>(p, threads, st, grid_out)
                              : launch_batch_loop_t<2, false, true>(p, threads, st, grid_out);
        return perim ? launch_batch_loop_t<2, true, false>(p, threads, st, grid_out)
                     : launch_batch_loop_t<2, false, false>(p, threads, st, grid_out);
    }
    if (act) return perim ? launch_batch_loop_t<3, true, true>(p, threads, st, grid_out)
                          : launch_batch_loop_t<3, false, true>(p, threads, st, grid_out);
    return perim ? launch_batch_loop_t<3, true, false>(p, threads, st, grid_out)
                 : launch_batch_loop_t<3, false, false>(p, threads, st, grid_out);
}

template <int DIM, bool PERIM, bool ACT>
void batch_round_t(bool track, const BatchLattice *lats, const int2 *items, uint32_t n_items, uint32_t q,
                   uint32_t threads, cudaStream_t st)
{
    if (track) batch_round_kernel<DIM, PERIM, ACT, true><<<n_items, threads, 0, st>>>(lats, items, q);
    else batch_round_kernel<DIM, PERIM, ACT, false><<<n_items, threads, 0, st>>>(lats, items, q);
}

cudaError_t launch_batch_round(int dim, bool perim, bool act, bool track, const BatchLattice *lats,
                               const int2 *items, uint32_t n_items, uint32_t q, uint32_t threads, cudaStream_t st)
{
    if (n_items == 0) return cudaSuccess;
    if (dim == 2) {
        if (act) {
            if (perim) batch_round_t<2, true, true>(track, lats, items, n_items, q, threads, st);
            else batch_round_t<2, false, true>(track, lats, items, n_items, q, threads, st);
        } else {
            if (perim) batch_round_t<2, true, false>(track, lats, items, n_items, q, threads, st);
            else batch_round_t<2, false, false>(track, lats, items, n_items, q, threads, st);
        }
    } else {
        if (act) {
            if (perim) batch_round_t<3, true, true>(track, lats, items, n_items, q, threads, st);
            else batch_round_t<3, false, true>(track, lats, items, n_items, q, threads, st);
        } else {
            if (perim) batch_round_t<3, true, false>(track, lats, items, n_items, q, threads, st);
            else batch_round_t<3, false, false>(track, lats, items, n_items, q, threads, st);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_recount(int dim, const int32_t *lat, const uint8_t *, int32_t *V, int32_t *A, uint32_t nx,
                           uint32_t ny, uint32_t nz, cudaStream_t st)
{
    const uint64_t n = (uint64_t)nx * ny * nz;
    if (dim == 2)
        recount_kernel<2><<<grid_for(n, 256), 256, 0, st>>>(lat, V, A, nx, ny, nz, n);
    else
        recount_kernel<3><<<grid_for(n, 256), 256, 0, st>>>(lat, V, A, nx, ny, nz, n);
    return cudaGetLastError();
}

cudaError_t launch_compare(const int32_t *V, const int32_t *A, const int32_t *V2, const int32_t *A2, int32_t n,
                           unsigned long long *n_bad, cudaStream_t st)
{
    compare_kernel<<<grid_for((uint64_t)n, 256), 256, 0, st>>>(V, A, V2, A2, n, n_bad);
    return cudaGetLastError();
}

cudaError_t launch_clamp_stamps(int32_t *lat, uint64_t n, uint32_t t, cudaStream_t st)
{
    clamp_kernel<<<grid_for(n, 256), 256, 0, st>>>(lat, n, t);
    return cudaGetLastError();
}

cudaError_t launch_act_values(const int32_t *lat, const uint8_t *cell_type, const TypeParams &tp, uint64_t n,
                              uint32_t t_last, uint8_t *out, cudaStream_t st)
{
    act_values_kernel<<<grid_for(n, 256), 256, 0, st>>>(lat, cell_type, tp, n, t_last, out);
    return cudaGetLastError();
}

cudaError_t launch_unpack_ids(const int32_t *lat, int32_t *ids, uint64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    unpack_ids_kernel<<<grid_for(n, 256), 256, 0, st>>>(lat, ids, n);
    return cudaGetLastError();
}

cudaError_t launch_pack_ids(int32_t *lat, const int32_t *ids, const uint8_t *stamps, uint64_t n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    pack_ids_kernel<<<grid_for(n, 256), 256, 0, st>>>(lat, ids, stamps, n);
    return cudaGetLastError();
}

}  // namespace cpmgb
