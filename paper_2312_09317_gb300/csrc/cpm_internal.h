// Internal declarations of the GB300 CPM sweep library, shared by its host
// and device translation units.  Not part of the public C ABI (include/cpm.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace cpmgb {

constexpr int kMaxTypes = 8;
constexpr int kLnEntries = 129;  // LN[a], a in 0..128

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications whose halves are mixed with the other words and a
// round key; the key advances by the two Weyl increments after each round.
struct Philox4 {
    uint32_t v[4];
};

__host__ __device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                          uint32_t k0, uint32_t k1)
{
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kBumpA = 0x9E3779B9u, kBumpB = 0xBB67AE85u;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
#ifdef __CUDA_ARCH__
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
#else
        const uint64_t pA = (uint64_t)kMulA * c0, pB = (uint64_t)kMulB * c2;
        const uint32_t hiA = (uint32_t)(pA >> 32), loA = (uint32_t)pA;
        const uint32_t hiB = (uint32_t)(pB >> 32), loB = (uint32_t)pB;
#endif
        const uint32_t n0 = hiB ^ c1 ^ k0;
        const uint32_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kBumpA;
        k1 += kBumpB;
    }
    Philox4 r;
    r.v[0] = c0; r.v[1] = c1; r.v[2] = c2; r.v[3] = c3;
    return r;
}

// Uniform index in [0, n) from a 32-bit draw: the high word of w*n.
__host__ __device__ __forceinline__ uint32_t draw_below(uint32_t w, uint32_t n)
{
#ifdef __CUDA_ARCH__
    return __umulhi(w, n);
#else
    return (uint32_t)(((uint64_t)w * n) >> 32);
#endif
}

// Lattice words.  With the Act term on, a site's word carries its cell id in
// the low 24 bits (two's complement: -1 is a frozen obstacle) and its Act
// time stamp (MCS mod 256 of its last update) in the high 8 bits, so that one
// load gives both; without Act the word is the plain id.  Either way
// cell_id() recovers the id (ids up to 2^23 - 1).
constexpr int32_t kMaxCellId = (1 << 23) - 1;
__host__ __device__ __forceinline__ int32_t cell_id(int32_t w) { return (int32_t)((uint32_t)w << 8) >> 8; }
__host__ __device__ __forceinline__ uint32_t word_stamp(int32_t w) { return (uint32_t)w >> 24; }
__host__ __device__ __forceinline__ int32_t pack_word(int32_t id, uint32_t stamp)
{
    return (int32_t)((stamp << 24) | ((uint32_t)id & 0x00FFFFFFu));
}

// Composite variable tracking (Eq. 11): the shift k of coordinate x to its periodic image
// nearest the point S / V on an axis of extent n, k = floor((S - x V) / (n V) + 1/2), V >= 1.
__host__ __device__ __forceinline__ int64_t track_image_shift(int64_t x, int64_t S, int64_t V, int64_t n)
{
    const int64_t num = 2 * (S - x * V) + n * V, den = 2 * n * V;
    int64_t q = num / den;
    if (num % den != 0 && num < 0) q -= 1;
    return q;
}

// Per-type model parameters, integer-scaled.
struct TypeParams {
    int32_t J[kMaxTypes][kMaxTypes];
    int32_t lambda_v[kMaxTypes], v_target[kMaxTypes];
    int32_t lambda_p[kMaxTypes], a_target[kMaxTypes];
    int32_t lambda_act[kMaxTypes], max_act[kMaxTypes];
    int32_t obstacle_type;
    int32_t lambda_chem[kMaxTypes], lambda_pers[kMaxTypes];  // motility weights, scaled
    double inv_len[4];                                        // 1 / sqrt(k), k = |d|^2 of a copy direction
    int32_t gm_max[kMaxTypes];  // EXPQ[LN[Max_act] >> 6]: the largest Act geometric mean a type's site can have
};

// Everything one round of the sweep needs.
struct RoundArgs {
    int32_t *lat;              // lattice words (see cell_id), x fastest
    uint32_t packed;           // 1: the words carry Act stamps (Act on for this lattice)
    uint32_t stream_loads;     // 1: lattice words through the streaming cache path (Act, area edge >= 8)
    uint32_t pdl;              // 1: launched as a programmatic dependent of the previous round
    const uint8_t *cell_type;  // per cell id
    const int32_t *Vc, *Ac;    // tallies as of the start of this round
    int32_t *Vn, *An;          // tallies being built for the next round
    const int4 *pend_prev;     // accepted change of the previous round, per active index (valid where flagged)
    int4 *pend_cur;            // accepted change of this round, per active index (written on accept only)
    const uint8_t *flag_prev;  // 1 where the previous round accepted a copy, per active index
    uint8_t *flag_cur;         // this round's flags (every active index written)
    // composite variable tracking (Eq. 11); null when off.  Coordinate sums of every cell,
    // [n_cells + 1][3], as of the start of this round and being built for the next round, and
    // per active index the site and image shifts of an accepted change (valid where flagged).
    const long long *Sc;
    long long *Sn;
    const int2 *tpend_prev;
    int2 *tpend_cur;
    const uint32_t *thr;       // acceptance thresholds, L entries
    const int32_t *ln_tab;     // LN[0..128]
    const int32_t *expq;       // EXPQ[m]
    unsigned long long *accepts;
    int32_t L;
    uint32_t nx, ny, nz;
    uint32_t s, c, sd;         // block edge, divisions, sites per block
    uint32_t nbx, nby;         // blocks per axis
    uint32_t nax, nay;         // active blocks per axis (nbx / c, nby / c)
    uint32_t n_active;
    uint32_t cx, cy, cz;       // active colour, per axis
    uint32_t t, sp, r;         // MCS (low 32 bits), sub-pass, round
    uint32_t key0, key1;
    uint32_t brick_x, brick_y, brick_z;  // active blocks per CTA along each axis (product <= 256)
    const int16_t *chem;       // chemotaxis field, dim int16 per site (Q14), or null
    const double *pers_dir;    // persistence directions, 3 per cell id, or null
    TypeParams tp;
};

// Batched ensembles: one lattice of the batch.  base carries its buffers and
// constants (per-round fields are filled in by the kernel); the round of
// lattice l at batch step q is round g_start + q of that lattice, in MCS
// t_start + q / R.
constexpr uint32_t kBatchMaxThreads = 256;
struct BatchLattice {
    RoundArgs base;
    int32_t *V[2], *A[2];
    int4 *pend[2];
    uint8_t *flag[2];
    long long *S[2];     // tracked centroid sums, when the batch tracks them (else null)
    int2 *tpend[2];
    uint32_t R, k, C;
    int32_t n_cells;
    int64_t t_start;
    uint64_t g_start;
};
cudaError_t launch_batch_round(int dim, bool perim, bool act, bool track, const BatchLattice *lats,
                               const int2 *items, uint32_t n_items, uint32_t q, uint32_t threads, cudaStream_t st);
// every tracking member's centroids into [0, n) after its MCS (csrc/cpm_track.cu)
cudaError_t launch_batch_track_rewrap(int dim, const BatchLattice *lats, uint32_t n, cudaStream_t st);
cudaError_t launch_batch_clamp(const BatchLattice *lats, const int2 *items, uint32_t n_items, cudaStream_t st);
cudaError_t launch_batch_advance(BatchLattice *lats, uint32_t n, cudaStream_t st);
// The persistent batched MCS loop (one cooperative launch for n_mcs MCS).
struct BatchLoopArgs {
    BatchLattice *lats;
    uint32_t n_lats;
    const int2 *items;        // round items, members by rounds per MCS (descending)
    const uint32_t *upto_q;   // items of round q: the first upto_q[q]
    uint32_t r_max;           // rounds per MCS of the longest member
    const int2 *clamp;        // Act clamp items
    uint32_t n_clamp;
    uint32_t n_mcs;
    unsigned long long *bar;  // grid barrier counter, 0 at launch
    unsigned *next;           // per round: items claimed so far (r_max counters, 0 at launch)
    long long max_polls;      // bound of every barrier wait
    int *err;                 // set to 1 when a wait runs out
    uint32_t max_items;       // items of the fullest round (bounds the grid)
    int test_absent;          // test of the timeout path: CTA 0 leaves before its first barrier
};
cudaError_t launch_batch_loop(int dim, bool perim, bool act, const BatchLoopArgs &p, uint32_t threads, cudaStream_t st,
                              uint32_t *grid_out);

// Observations of a batch (cpm_batch_observe): one item per lattice.
constexpr int kObsFields = 12;  // anchor, volume, offset sums x y z, interface count, xx yy zz xy xz yz
struct ObserveItem {
    const int32_t *lat;
    const unsigned long long *accepts;
    uint32_t nx, ny, nz, dim;
    int64_t row0;  // first output row of this lattice (its medium row)
    int32_t n_cells, pad_;
    double v_ref, a_ref;  // V_t and A_t of cell 1's type: the scale of the volume / interface statistics
};
cudaError_t launch_observe(int dim, const ObserveItem *d_items, uint32_t n_items, int64_t max_sites, int64_t *cells,
                           int64_t *member, cudaStream_t st);

// Persistence update at the end of an MCS (Eq. 6, Eq. 7) from one observation of the lattice.
struct PersParams {
    int32_t lambda[kMaxTypes], dt[kMaxTypes];
    double mu[kMaxTypes];
};
cudaError_t launch_pers_update(const int64_t *cells, int32_t n_cells, uint32_t nx, uint32_t ny, uint32_t nz,
                               const uint8_t *cell_type, const PersParams &pp, double *hist, int32_t H, int64_t t,
                               int64_t t0, double *dir, cudaStream_t st);

// Summary statistics of 2D lattices from a stack of observations (cpm_batch_summarize).
constexpr int kSummaryStats = 16;
constexpr int kSummaryMaxSnap = 1024;
cudaError_t launch_summarize(const ObserveItem *d_items, uint32_t n_items, int32_t max_cells, const int64_t *cells,
                             int64_t rows, const int64_t *member, int32_t n_snap, int32_t every, double *traj,
                             double *out, cudaStream_t st);

// Tiled schedule: everything one epoch of one tile colour needs.
constexpr int kMaxEpochSubpasses = 512;
constexpr uint32_t kTileHashCap = 512;  // distinct ids a tile and its halo may hold (incl. medium, obstacle)
constexpr uint32_t kTileThrSmem = 2048;  // threshold-table entries kept in shared memory

struct TileArgs {
    int32_t *lat;              // lattice words (see cell_id)
    const uint8_t *cell_type;
    const int32_t *Vc, *Ac;    // tallies at the start of the epoch (read-only during it)
    int32_t *Vn, *An;          // copy of Vc/Ac that receives every tile's changes
    const uint32_t *thr;
    const int32_t *ln_tab;
    const int32_t *expq;
    unsigned long long *accepts;
    int *error_flag;           // set when a tile's change table overflows
    int32_t L;
    uint32_t nx, ny, nz;
    uint32_t s, c, sd, k;      // block edge, divisions, sites per block, rounds per sub-pass
    uint32_t nbx, nby, nbz;
    uint32_t T, hash_cap, thr_smem;
    uint32_t n_sub, sp0;       // sub-passes of the epoch: sp0 .. sp0 + n_sub - 1
    uint32_t t;                // MCS (low 32 bits)
    uint32_t key0, key1;
    uint32_t offx, offy, offz; // tile grid offset of this MCS
    uint32_t tcx, tcy, tcz;    // active tile colour, per axis
    int32_t colours[kMaxEpochSubpasses];
    TypeParams tp;
};

size_t tile_dyn_smem(int dim, bool act, uint32_t T, uint32_t cap, uint32_t a, uint32_t thr_smem);
cudaError_t launch_tile_epoch(int dim, bool perim, bool act, const TileArgs &a, uint32_t n_tiles, cudaStream_t st);

// CTA brick of active blocks for the round kernel, measured on GB300 against
// other shapes and row-major mapping.  3D: 8x4x4 (128 threads) when active
// blocks are less than 16 sites apart (areas of edge < 16), where the
// stencils of neighbouring threads share lines; 16x8x2 (256 threads) when
// they are 16 or more apart and a row has at least 16 of them: no lines are
// shared, and a warp's loads then fall on 16 consecutive 64-byte granules of
// a row (1024^3 tissue with 16^3 areas: 193.5 against 201.6 ms per MCS).
// 2D: 16x16.
inline void pick_bricks(int dim, uint32_t nax, uint32_t nay, RoundArgs &a)
{
    if (dim == 3) {
        if (a.s * a.c >= 16 && nax >= 16) {
            a.brick_x = 16; a.brick_y = 8; a.brick_z = 2;
        } else {
            a.brick_x = 8; a.brick_y = 4; a.brick_z = 4;
        }
    } else {
        a.brick_x = 16; a.brick_y = 16; a.brick_z = 1;
    }
    (void)nay;
}

// Launchers (defined in the per-dimension translation units).
cudaError_t launch_round(int dim, bool perim, bool act, const RoundArgs &a, cudaStream_t st);
cudaError_t launch_recount(int dim, const int32_t *lat, const uint8_t *cell_type, int32_t *V, int32_t *A,
                           uint32_t nx, uint32_t ny, uint32_t nz, cudaStream_t st);
cudaError_t launch_compare(const int32_t *V, const int32_t *A, const int32_t *V2, const int32_t *A2, int32_t n,
                           unsigned long long *n_bad, cudaStream_t st);
cudaError_t launch_clamp_stamps(int32_t *lat, uint64_t n, uint32_t t, cudaStream_t st);
// Composite variable tracking (csrc/cpm_track.cu): sums of a lattice's cells from scratch (anchor:
// n_cells + 1 words of scratch), and the move of every live cell's centroid into [0, n) applied to
// both tally buffers (V: the complete volume tally).
cudaError_t launch_track_init(int dim, const int32_t *lat, uint32_t nx, uint32_t ny, uint32_t nz, int32_t n_cells,
                              const int32_t *V, uint32_t *anchor, long long *S, cudaStream_t st);
cudaError_t launch_track_rewrap(int dim, uint32_t nx, uint32_t ny, uint32_t nz, int32_t n_cells, const int32_t *V,
                                long long *S_complete, long long *S_other, cudaStream_t st);
cudaError_t launch_act_values(const int32_t *lat, const uint8_t *cell_type, const TypeParams &tp, uint64_t n,
                              uint32_t t_last, uint8_t *out, cudaStream_t st);
// Lattice words <-> ids: unpack n words into ids; pack n ids into the words
// of lat, keeping their stamps (or, with stamps != null, taking stamps[x]).
cudaError_t launch_unpack_ids(const int32_t *lat, int32_t *ids, uint64_t n, cudaStream_t st);
cudaError_t launch_pack_ids(int32_t *lat, const int32_t *ids, const uint8_t *stamps, uint64_t n, cudaStream_t st);

}  // namespace cpmgb
