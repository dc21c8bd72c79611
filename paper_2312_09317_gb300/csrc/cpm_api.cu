// Host side of the C ABI declared in include/cpm.h: configuration checks,
// device state, the integer tables, the colour schedule and the launch loop.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <thread>
#include <string>
#include <vector>

#include "../../include/cpm.h"
#include "cpm_internal.h"

using namespace cpmgb;

struct cpm_handle {
    cpm_config cfg;  // pointers inside are not kept
    TypeParams tp;
    cudaStream_t stream = nullptr;
    int dim = 2, nb = 8;
    uint64_t n_sites = 0;
    int32_t n_cells = 0;
    uint32_t s = 1, C = 1, sd = 1, k = 1, per_mcs = 1, per_sub_mcs = 1;
    uint32_t nbx = 1, nby = 1, nbz = 1, n_active = 0;
    bool perim = false, act = false;
    // device state
    int32_t *lat = nullptr;        // lattice words: ids, with the Act stamps in the high byte when act
    int32_t *stage = nullptr;      // staging for host reads and loads of packed words (lazily allocated)
    uint64_t stage_n = 0;
    uint8_t *cell_type = nullptr;
    int32_t *tallies = nullptr;  // V0, A0, V1, A1, Vtmp, Atmp; each n_cells + 1
    int4 *pend = nullptr;        // two buffers of n_active
    uint8_t *flags = nullptr;    // two buffers of n_active: pend entry valid
    uint32_t *thr = nullptr;
    int32_t *ln_tab = nullptr;
    int32_t *expq = nullptr;
    unsigned long long *counters = nullptr;  // [0] accepts, [1] scratch
    uint8_t *act_tmp = nullptr;
    int32_t L = 0;
    // tiled schedule
    uint32_t tile = 0, tile_cycles = 1, CT = 1;
    int *error_flag = nullptr;
    bool shared_tables = false;  // thr / ln_tab / expq belong to a batch's table cache
    double v_ref = 0.0, a_ref = 0.0;  // V_t, A_t of cell 1's type (scales of the summary statistics)
    // motility (Eq. 4 to Eq. 7)
    int16_t *chem = nullptr;          // field, dim int16 per site
    bool pers = false;
    PersParams pp{};
    double *pers_dir = nullptr;       // (n_cells + 1) x 3
    double *pers_hist = nullptr;      // H x (n_cells + 1) x 3 centroids
    int32_t pers_H = 0;
    ObserveItem *pers_item = nullptr; // one observation item for this lattice
    int64_t *pers_cells = nullptr;    // observation rows, (n_cells + 1) x kObsFields
    int64_t *pers_member = nullptr;   // [2]
    // composite variable tracking (Eq. 11), off until cpm_track_centroids
    long long *csum = nullptr;        // two buffers of (n_cells + 1) x 3 coordinate sums
    int2 *tpend = nullptr;            // two buffers of n_active: site and image shifts of a pending change
    uint32_t *track_anchor = nullptr; // n_cells + 1 words of scratch for starting the sums
    // position
    int64_t t = 0;
    int32_t sp = 0;
    uint64_t g = 0;  // global round index
    int64_t launches = 0;
    int64_t attempts = 0;
    std::string err;
};

namespace {

thread_local std::string g_create_error;  // per calling thread: creations may run concurrently

int fail(cpm_handle *h, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return code;
}

#define CUDA_TRY(h, expr)                                                                        \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail((h), e_ == cudaErrorMemoryAllocation ? CPM_E_NOMEM : CPM_E_CUDA, "%s: %s", \
                        #expr, cudaGetErrorString(e_));                                          \
    } while (0)

uint32_t ipow(uint32_t b, int e)
{
    uint32_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

int32_t *V_buf(cpm_handle *h, int which) { return h->tallies + (size_t)(2 * which) * (h->n_cells + 1); }
long long *S_buf(cpm_handle *h, int which) { return h->csum + (size_t)which * 3 * (h->n_cells + 1); }
int32_t *A_buf(cpm_handle *h, int which) { return h->tallies + (size_t)(2 * which + 1) * (h->n_cells + 1); }

int validate(const cpm_config *c)
{
    if (!c) return fail(nullptr, CPM_E_INVALID, "cfg is NULL");
    if (c->dim != 2 && c->dim != 3) return fail(nullptr, CPM_E_INVALID, "dim must be 2 or 3");
    if (c->nx < 3 || c->ny < 3 || (c->dim == 3 && c->nz < 3) || (c->dim == 2 && c->nz != 1))
        return fail(nullptr, CPM_E_INVALID, "extents must be >= 3 (nz = 1 in 2D)");
    const uint64_t n = (uint64_t)c->nx * c->ny * c->nz;
    if (n > (1ull << 31)) return fail(nullptr, CPM_E_INVALID, "at most 2^31 sites");
    if (c->c < 2 || c->a < 2 || c->a % c->c) return fail(nullptr, CPM_E_INVALID, "need c >= 2 and c | a");
    const int s = c->a / c->c;
    if (c->a - s < 2) return fail(nullptr, CPM_E_INVALID, "blocks of one colour must be >= 2 sites apart (a - a/c >= 2)");
    if (c->nx % c->a || c->ny % c->a || (c->dim == 3 && c->nz % c->a))
        return fail(nullptr, CPM_E_INVALID, "extents must be multiples of a");
    if (ipow(c->c, c->dim) > 27) return fail(nullptr, CPM_E_INVALID, "at most 27 colours");
    const uint32_t sd = ipow(s, c->dim);
    if (c->P < 1 || sd % c->P) return fail(nullptr, CPM_E_INVALID, "P must divide s^d");
    if (!(c->temperature > 0.0) || c->temperature > 2900.0)
        return fail(nullptr, CPM_E_INVALID, "temperature must be in (0, 2900]");
    if (c->obstacle_type < 1 || c->obstacle_type >= CPM_MAX_TYPES) return fail(nullptr, CPM_E_INVALID, "bad obstacle_type");
    // ids share the lattice word with the Act stamp: 24-bit two's complement
    if (c->n_cells < 0 || c->n_cells > kMaxCellId)
        return fail(nullptr, CPM_E_INVALID, "n_cells must be in 0..%d", (int)kMaxCellId);
    if (!c->cell_type || !c->init_lattice) return fail(nullptr, CPM_E_INVALID, "cell_type and init_lattice are required");
    if (c->cell_type[0] != 0) return fail(nullptr, CPM_E_INVALID, "cell_type[0] (medium) must be 0");
    for (int i = 1; i <= c->n_cells; i++)
        if (c->cell_type[i] < 1 || c->cell_type[i] >= CPM_MAX_TYPES)
            return fail(nullptr, CPM_E_INVALID, "cell_type[%d] out of range", i);
    for (int a = 0; a < CPM_MAX_TYPES; a++) {
        for (int b = 0; b < CPM_MAX_TYPES; b++)
            if (c->J[a][b] != c->J[b][a]) return fail(nullptr, CPM_E_INVALID, "J must be symmetric");
        if (c->max_act[a] < 0 || c->max_act[a] > 127) return fail(nullptr, CPM_E_INVALID, "max_act must be in 0..127");
        if (c->lambda_v[a] < 0 || c->lambda_p[a] < 0 || c->lambda_act[a] < 0)
            return fail(nullptr, CPM_E_INVALID, "lambdas must be >= 0");
    }
    bool motility = c->chem_field != nullptr;
    for (int a = 0; a < CPM_MAX_TYPES; a++) {
        if (c->lambda_pers[a] != 0) {
            motility = true;
            if (c->dt_pers[a] < 1 || c->dt_pers[a] > 255)
                return fail(nullptr, CPM_E_INVALID, "dt_pers must be in 1..255 where lambda_pers != 0");
            if (!(c->mu_pers[a] >= 0.0 && c->mu_pers[a] <= 1.0))
                return fail(nullptr, CPM_E_INVALID, "mu_pers must be in [0, 1]");
        }
        if (c->lambda_chem[a] < -(1 << 24) || c->lambda_chem[a] > (1 << 24) || c->lambda_pers[a] < -(1 << 24) ||
            c->lambda_pers[a] > (1 << 24))
            return fail(nullptr, CPM_E_INVALID, "motility weights out of range");
    }
    if (motility && c->tile > 0) return fail(nullptr, CPM_E_INVALID, "motility terms need the global schedule");
    if (c->t0 < 0) return fail(nullptr, CPM_E_INVALID, "t0 must be >= 0");
    if (c->tile < 0) return fail(nullptr, CPM_E_INVALID, "tile must be >= 0");
    if (c->tile > 0) {
        const int T = c->tile;
        if (T % c->a) return fail(nullptr, CPM_E_INVALID, "tile must be a multiple of a");
        if ((c->dim == 3 && T > 36) || T > 250) return fail(nullptr, CPM_E_INVALID, "tile edge too large");
        if (c->nx % (2 * T) || c->ny % (2 * T) || (c->dim == 3 && c->nz % (2 * T)))
            return fail(nullptr, CPM_E_INVALID, "extents must be multiples of 2*tile");
        if (c->tile_cycles < 1 || c->P % c->tile_cycles) return fail(nullptr, CPM_E_INVALID, "tile_cycles must divide P");
        const uint32_t per = (uint32_t)(T / c->a);
        if (ipow(per, c->dim) > 1024) return fail(nullptr, CPM_E_INVALID, "at most 1024 blocks per tile colour");
        if ((uint32_t)c->P * ipow(c->c, c->dim) / (uint32_t)c->tile_cycles > (uint32_t)kMaxEpochSubpasses)
            return fail(nullptr, CPM_E_INVALID, "too many sub-passes per epoch");
        bool act = false;
        for (int a = 0; a < CPM_MAX_TYPES; a++)
            if (c->lambda_act[a]) act = true;
        if (tile_dyn_smem(c->dim, act, (uint32_t)T, kTileHashCap, (uint32_t)c->a, kTileThrSmem) > 220 * 1024)
            return fail(nullptr, CPM_E_INVALID, "tile too large for shared memory");
    }
    for (uint64_t x = 0; x < n; x++) {
        const int32_t v = c->init_lattice[x];
        if (v < -1 || v > c->n_cells) return fail(nullptr, CPM_E_INVALID, "init_lattice[%llu] = %d out of range",
                                                  (unsigned long long)x, v);
        if (c->init_act && c->init_act[x]) {
            if (v <= 0) return fail(nullptr, CPM_E_INVALID, "init_act must be 0 outside cells");
            if (c->init_act[x] > c->max_act[c->cell_type[v]])
                return fail(nullptr, CPM_E_INVALID, "init_act above max_act at site %llu", (unsigned long long)x);
        }
    }
    return CPM_OK;
}

// Colour visited at sub-pass sp of MCS t: a Fisher-Yates shuffle of the C
// colours per cycle, swap i (C-1 down to 1) drawn from counter (i, cycle, t, 1<<24).
uint32_t colour_of(const cpm_handle *h, int64_t t, int32_t sp)
{
    uint32_t perm[27];
    for (uint32_t q = 0; q < h->C; q++) perm[q] = q;
    const uint32_t cycle = (uint32_t)sp / h->C;
    for (uint32_t i = h->C - 1; i >= 1; i--) {
        const Philox4 w = philox4x32_10(i, cycle, (uint32_t)t, 1u << 24, (uint32_t)h->cfg.seed,
                                        (uint32_t)(h->cfg.seed >> 32));
        const uint32_t j = draw_below(w.v[0], i + 1);
        const uint32_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    return perm[(uint32_t)sp % h->C];
}

int recount(cpm_handle *h, int32_t *V, int32_t *A)
{
    const size_t bytes = sizeof(int32_t) * (h->n_cells + 1);
    CUDA_TRY(h, cudaMemsetAsync(V, 0, bytes, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(A, 0, bytes, h->stream));
    CUDA_TRY(h, launch_recount(h->dim, h->lat, h->cell_type, V, A, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->stream));
    h->launches += 1;
    return CPM_OK;
}

// Recompute the tallies from the lattice into both buffers and forget pending changes.
int reset_tallies(cpm_handle *h)
{
    const int cur = (int)(h->g & 1);
    int rc = recount(h, V_buf(h, cur), A_buf(h, cur));
    if (rc) return rc;
    const size_t bytes = sizeof(int32_t) * (h->n_cells + 1);
    CUDA_TRY(h, cudaMemcpyAsync(V_buf(h, cur ^ 1), V_buf(h, cur), bytes, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(A_buf(h, cur ^ 1), A_buf(h, cur), bytes, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->flags, 0, 2 * (size_t)h->n_active, h->stream));
    if (h->csum) {
        CUDA_TRY(h, launch_track_init(h->dim, h->lat, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->n_cells, V_buf(h, cur),
                                      h->track_anchor, S_buf(h, cur), h->stream));
        CUDA_TRY(h, cudaMemcpyAsync(S_buf(h, cur ^ 1), S_buf(h, cur), sizeof(long long) * 3 * (h->n_cells + 1),
                                    cudaMemcpyDeviceToDevice, h->stream));
        h->launches += 3;
    }
    return CPM_OK;
}

// Staging buffer of up to 64 Mi words (256 MiB) for host reads and loads of a
// packed lattice: large enough that each chunk's copy runs at the link's speed.
int ensure_stage(cpm_handle *h)
{
    if (h->stage) return CPM_OK;
    const uint64_t n = std::min<uint64_t>(h->n_sites, (uint64_t)1 << 26);
    CUDA_TRY(h, cudaMalloc(&h->stage, sizeof(int32_t) * n));
    h->stage_n = n;
    return CPM_OK;
}

// Persistence update at the end of the MCS that brought the handle to time h->t
// (and at creation): observe the lattice, record the centroids, update p_hat.
int pers_step(cpm_handle *h)
{
    CUDA_TRY(h, launch_observe(h->dim, h->pers_item, 1, (int64_t)h->n_sites, h->pers_cells, h->pers_member,
                               h->stream));
    CUDA_TRY(h, launch_pers_update(h->pers_cells, h->n_cells, (uint32_t)h->cfg.nx, (uint32_t)h->cfg.ny,
                                   (uint32_t)h->cfg.nz, h->cell_type, h->pp, h->pers_hist, h->pers_H, h->t,
                                   h->cfg.t0, h->pers_dir, h->stream));
    h->launches += 4;
    return CPM_OK;
}

int run_subpass(cpm_handle *h)
{
    if (h->act && h->sp == 0 && h->t % 64 == 0) {
        CUDA_TRY(h, launch_clamp_stamps(h->lat, h->n_sites, (uint32_t)h->t, h->stream));
        h->launches += 1;
    }
    const uint32_t col = colour_of(h, h->t, h->sp);
    RoundArgs a;
    memset(&a, 0, sizeof a);
    a.lat = h->lat;
    a.packed = h->act ? 1u : 0u;
    a.stream_loads = h->act && h->cfg.a >= 8 ? 1u : 0u;
    a.pdl = 1;  // each round overlaps its set-up with the previous round's tail
    a.cell_type = h->cell_type;
    a.thr = h->thr;
    a.ln_tab = h->ln_tab;
    a.expq = h->expq;
    a.accepts = h->counters;
    a.L = h->L;
    a.nx = h->cfg.nx; a.ny = h->cfg.ny; a.nz = h->cfg.nz;
    a.s = h->s; a.c = h->cfg.c; a.sd = h->sd;
    a.nbx = h->nbx; a.nby = h->nby;
    a.nax = h->nbx / h->cfg.c; a.nay = h->nby / h->cfg.c;
    a.n_active = h->n_active;
    a.cx = col % h->cfg.c;
    a.cy = (col / h->cfg.c) % h->cfg.c;
    a.cz = col / (h->cfg.c * h->cfg.c);
    a.t = (uint32_t)h->t;
    a.sp = (uint32_t)h->sp;
    a.key0 = (uint32_t)h->cfg.seed;
    a.key1 = (uint32_t)(h->cfg.seed >> 32);
    a.tp = h->tp;
    a.chem = h->chem;
    a.pers_dir = h->pers ? h->pers_dir : nullptr;
    pick_bricks(h->dim, a.nax, a.nay, a);
    for (uint32_t r = 0; r < h->k; r++) {
        const int cur = (int)(h->g & 1);
        a.r = r;
        a.Vc = V_buf(h, cur);
        a.Ac = A_buf(h, cur);
        a.Vn = V_buf(h, cur ^ 1);
        a.An = A_buf(h, cur ^ 1);
        a.pend_prev = h->pend + (size_t)(cur ^ 1) * h->n_active;
        a.pend_cur = h->pend + (size_t)cur * h->n_active;
        a.flag_prev = h->flags + (size_t)(cur ^ 1) * h->n_active;
        a.flag_cur = h->flags + (size_t)cur * h->n_active;
        if (h->csum) {
            a.Sc = S_buf(h, cur);
            a.Sn = S_buf(h, cur ^ 1);
            a.tpend_prev = h->tpend + (size_t)(cur ^ 1) * h->n_active;
            a.tpend_cur = h->tpend + (size_t)cur * h->n_active;
        }
        CUDA_TRY(h, launch_round(h->dim, h->perim, h->act, a, h->stream));
        h->launches += 1;
        h->g += 1;
        h->attempts += h->n_active;
    }
    if (++h->sp == (int32_t)h->per_mcs) {
        h->sp = 0;
        h->t += 1;
        if (h->csum) {
            // every centroid back into [0, n): the same shift in both buffers
            const int cur = (int)(h->g & 1);
            CUDA_TRY(h, launch_track_rewrap(h->dim, h->cfg.nx, h->cfg.ny, h->cfg.nz, h->n_cells, V_buf(h, cur),
                                            S_buf(h, cur), S_buf(h, cur ^ 1), h->stream));
            h->launches += 1;
        }
        if (h->pers) return pers_step(h);
    }
    return CPM_OK;
}

// Tile grid offset of MCS t: per axis a multiple of a below T, from counter (0, 0, t, 2<<24).
void tile_offset(const cpm_handle *h, int64_t t, uint32_t off[3])
{
    const Philox4 w = philox4x32_10(0u, 0u, (uint32_t)t, 2u << 24, (uint32_t)h->cfg.seed, (uint32_t)(h->cfg.seed >> 32));
    const uint32_t units = h->tile / (uint32_t)h->cfg.a;
    off[0] = (uint32_t)h->cfg.a * draw_below(w.v[0], units);
    off[1] = (uint32_t)h->cfg.a * draw_below(w.v[1], units);
    off[2] = h->dim == 3 ? (uint32_t)h->cfg.a * draw_below(w.v[2], units) : 0u;
}

// Tile colour of epoch e of cycle: Fisher-Yates over 2^d colours, swap i from (i, cycle, t, 3<<24).
uint32_t tile_colour_of(const cpm_handle *h, int64_t t, uint32_t cycle, uint32_t q)
{
    uint32_t perm[8];
    for (uint32_t i = 0; i < h->CT; i++) perm[i] = i;
    for (uint32_t i = h->CT - 1; i >= 1; i--) {
        const Philox4 w = philox4x32_10(i, cycle, (uint32_t)t, 3u << 24, (uint32_t)h->cfg.seed,
                                        (uint32_t)(h->cfg.seed >> 32));
        const uint32_t j = draw_below(w.v[0], i + 1);
        const uint32_t tmp = perm[i];
        perm[i] = perm[j];
        perm[j] = tmp;
    }
    return perm[q];
}

int run_epoch(cpm_handle *h)
{
    if (h->act && h->sp == 0 && h->t % 64 == 0) {
        CUDA_TRY(h, launch_clamp_stamps(h->lat, h->n_sites, (uint32_t)h->t, h->stream));
        h->launches += 1;
    }
    const uint32_t cycle = (uint32_t)h->sp / h->CT;
    const uint32_t tcol = tile_colour_of(h, h->t, cycle, (uint32_t)h->sp % h->CT);
    const uint32_t n_sub = h->per_sub_mcs / h->tile_cycles;
    TileArgs a;
    memset(&a, 0, sizeof a);
    a.lat = h->lat;
    a.cell_type = h->cell_type;
    const int cur = (int)(h->g & 1);
    a.Vc = V_buf(h, cur);
    a.Ac = A_buf(h, cur);
    a.Vn = V_buf(h, cur ^ 1);
    a.An = A_buf(h, cur ^ 1);
    a.thr = h->thr;
    a.ln_tab = h->ln_tab;
    a.expq = h->expq;
    a.accepts = h->counters;
    a.error_flag = h->error_flag;
    a.L = h->L;
    a.nx = h->cfg.nx; a.ny = h->cfg.ny; a.nz = h->cfg.nz;
    a.s = h->s; a.c = h->cfg.c; a.sd = h->sd; a.k = h->k;
    a.nbx = h->nbx; a.nby = h->nby; a.nbz = h->nbz;
    a.T = h->tile;
    a.hash_cap = kTileHashCap;
    a.thr_smem = (uint32_t)h->L < kTileThrSmem ? (uint32_t)h->L : kTileThrSmem;
    a.n_sub = n_sub;
    a.sp0 = cycle * n_sub;
    a.t = (uint32_t)h->t;
    a.key0 = (uint32_t)h->cfg.seed;
    a.key1 = (uint32_t)(h->cfg.seed >> 32);
    uint32_t off[3];
    tile_offset(h, h->t, off);
    a.offx = off[0]; a.offy = off[1]; a.offz = off[2];
    a.tcx = tcol & 1u; a.tcy = (tcol >> 1) & 1u; a.tcz = (tcol >> 2) & 1u;
    for (uint32_t q = 0; q < n_sub; q++) a.colours[q] = (int32_t)colour_of(h, h->t, (int32_t)(a.sp0 + q));
    a.tp = h->tp;
    const size_t bytes = sizeof(int32_t) * (h->n_cells + 1);
    CUDA_TRY(h, cudaMemcpyAsync(a.Vn, a.Vc, bytes, cudaMemcpyDeviceToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(a.An, a.Ac, bytes, cudaMemcpyDeviceToDevice, h->stream));
    const uint32_t ntx = h->cfg.nx / h->tile, nty = h->cfg.ny / h->tile;
    const uint32_t ntz = h->dim == 3 ? h->cfg.nz / h->tile : 1;
    const uint32_t n_tiles = (ntx / 2) * (nty / 2) * (h->dim == 3 ? ntz / 2 : 1);
    CUDA_TRY(h, launch_tile_epoch(h->dim, h->perim, h->act, a, n_tiles, h->stream));
    h->launches += 1;
    h->g += 1;
    h->attempts += (int64_t)(h->n_sites / ((uint64_t)h->CT * h->tile_cycles));
    if (++h->sp == (int32_t)h->per_mcs) {
        h->sp = 0;
        h->t += 1;
    }
    return CPM_OK;
}

int check_error_flag(cpm_handle *h)
{
    if (!h->error_flag) return CPM_OK;
    int flag = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&flag, h->error_flag, sizeof flag, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (flag) return fail(h, CPM_E_STATE, "a tile and its halo held more than %u distinct cells", kTileHashCap - 2);
    return CPM_OK;
}

// THR[h] = min(2^32-1, floor(2^32 exp(-h/(16T)))) up to the first zero; false when longer than 2^22
bool thr_table(double T, std::vector<uint32_t> &thr)
{
    thr.clear();
    for (int64_t e = 0;; e++) {
        const double v = std::floor(std::ldexp(std::exp(-(double)e / (16.0 * T)), 32));
        if (v <= 0.0) break;
        thr.push_back(v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v);
        if (thr.size() > (1u << 22)) return false;
    }
    return true;
}

// LN[a] = round(2^16 ln a), EXPQ[m] = round(2^16 exp(m/1024))
void ln_expq_tables(std::vector<int32_t> &ln, std::vector<int32_t> &ex)
{
    ln.assign(kLnEntries, 0);
    for (int a = 1; a < kLnEntries; a++) ln[a] = (int32_t)std::llround(std::ldexp(std::log((double)a), 16));
    const int32_t ne = (ln[kLnEntries - 1] >> 6) + 1;
    ex.resize(ne);
    for (int m = 0; m < ne; m++) ex[m] = (int32_t)std::llround(std::ldexp(std::exp((double)m / 1024.0), 16));
}

}  // namespace

// Tables shared by the lattices of a batch: LN / EXPQ once, THR once per
// temperature (keyed by the bit pattern of T).
struct TableCache {
    std::map<uint64_t, std::pair<uint32_t *, int32_t>> thr;
    std::map<uint64_t, std::vector<uint32_t>> host_thr;  // precomputed, not yet uploaded
    int32_t *ln = nullptr, *expq = nullptr;
    std::vector<void *> owned;
    ~TableCache()
    {
        for (void *p : owned) cudaFree(p);
    }
};

namespace {

uint64_t t_key(double T)
{
    uint64_t k;
    memcpy(&k, &T, sizeof k);
    return k;
}

int build_tables_cached(cpm_handle *h, TableCache *cache)
{
    if (!cache->ln) {
        std::vector<int32_t> ln, ex;
        ln_expq_tables(ln, ex);
        CUDA_TRY(h, cudaMalloc(&cache->ln, sizeof(int32_t) * ln.size()));
        cache->owned.push_back(cache->ln);
        CUDA_TRY(h, cudaMalloc(&cache->expq, sizeof(int32_t) * ex.size()));
        cache->owned.push_back(cache->expq);
        CUDA_TRY(h, cudaMemcpy(cache->ln, ln.data(), sizeof(int32_t) * ln.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(h, cudaMemcpy(cache->expq, ex.data(), sizeof(int32_t) * ex.size(), cudaMemcpyHostToDevice));
    }
    const uint64_t key = t_key(h->cfg.temperature);
    auto it = cache->thr.find(key);
    if (it == cache->thr.end()) {
        std::vector<uint32_t> local;
        auto pre = cache->host_thr.find(key);
        std::vector<uint32_t> &thr = pre != cache->host_thr.end() ? pre->second : local;
        if (pre == cache->host_thr.end() || thr.empty()) {
            if (!thr_table(h->cfg.temperature, thr)) return fail(h, CPM_E_INVALID, "threshold table too long");
        }
        uint32_t *d = nullptr;
        CUDA_TRY(h, cudaMalloc(&d, sizeof(uint32_t) * thr.size()));
        cache->owned.push_back(d);
        CUDA_TRY(h, cudaMemcpy(d, thr.data(), sizeof(uint32_t) * thr.size(), cudaMemcpyHostToDevice));
        it = cache->thr.emplace(key, std::make_pair(d, (int32_t)thr.size())).first;
        if (pre != cache->host_thr.end()) cache->host_thr.erase(pre);
    }
    h->thr = it->second.first;
    h->L = it->second.second;
    h->ln_tab = cache->ln;
    h->expq = cache->expq;
    h->shared_tables = true;
    return CPM_OK;
}

int build_tables(cpm_handle *h)
{
    std::vector<uint32_t> thr;
    if (!thr_table(h->cfg.temperature, thr)) return fail(h, CPM_E_INVALID, "threshold table too long");
    h->L = (int32_t)thr.size();
    std::vector<int32_t> ln, ex;
    ln_expq_tables(ln, ex);
    CUDA_TRY(h, cudaMalloc(&h->thr, sizeof(uint32_t) * thr.size()));
    CUDA_TRY(h, cudaMalloc(&h->ln_tab, sizeof(int32_t) * ln.size()));
    CUDA_TRY(h, cudaMalloc(&h->expq, sizeof(int32_t) * ex.size()));
    CUDA_TRY(h, cudaMemcpyAsync(h->thr, thr.data(), sizeof(uint32_t) * thr.size(), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->ln_tab, ln.data(), sizeof(int32_t) * ln.size(), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->expq, ex.data(), sizeof(int32_t) * ex.size(), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

void free_all(cpm_handle *h)
{
    cudaFree(h->lat);
    cudaFree(h->stage);
    cudaFree(h->cell_type);
    cudaFree(h->tallies);
    cudaFree(h->pend);
    cudaFree(h->flags);
    if (!h->shared_tables) {
        cudaFree(h->thr);
        cudaFree(h->ln_tab);
        cudaFree(h->expq);
    }
    cudaFree(h->chem);
    cudaFree(h->pers_dir);
    cudaFree(h->pers_hist);
    cudaFree(h->pers_item);
    cudaFree(h->pers_cells);
    cudaFree(h->pers_member);
    cudaFree(h->csum);
    cudaFree(h->tpend);
    cudaFree(h->track_anchor);
    cudaFree(h->counters);
    cudaFree(h->act_tmp);
    cudaFree(h->error_flag);
}

int create_impl(cpm_handle *h, const cpm_config *c, TableCache *cache = nullptr)
{
    h->cfg = *c;
    h->cfg.cell_type = nullptr;
    h->cfg.init_lattice = nullptr;
    h->cfg.init_act = nullptr;
    h->dim = c->dim;
    h->nb = c->dim == 3 ? 26 : 8;
    h->n_sites = (uint64_t)c->nx * c->ny * c->nz;
    h->n_cells = c->n_cells;
    h->s = (uint32_t)(c->a / c->c);
    h->C = ipow(c->c, c->dim);
    h->sd = ipow(h->s, c->dim);
    h->k = h->sd / c->P;
    h->per_sub_mcs = (uint32_t)c->P * h->C;
    h->per_mcs = h->per_sub_mcs;
    h->tile = (uint32_t)c->tile;
    h->tile_cycles = c->tile > 0 ? (uint32_t)c->tile_cycles : 1u;
    h->CT = c->dim == 3 ? 8u : 4u;
    if (h->tile) h->per_mcs = h->tile_cycles * h->CT;
    h->nbx = c->nx / h->s;
    h->nby = c->ny / h->s;
    h->nbz = c->dim == 3 ? c->nz / h->s : 1;
    h->n_active = (uint32_t)((uint64_t)h->nbx * h->nby * h->nbz / h->C);
    memcpy(h->tp.J, c->J, sizeof h->tp.J);
    memcpy(h->tp.lambda_v, c->lambda_v, sizeof h->tp.lambda_v);
    memcpy(h->tp.v_target, c->v_target, sizeof h->tp.v_target);
    memcpy(h->tp.lambda_p, c->lambda_p, sizeof h->tp.lambda_p);
    memcpy(h->tp.a_target, c->a_target, sizeof h->tp.a_target);
    memcpy(h->tp.lambda_act, c->lambda_act, sizeof h->tp.lambda_act);
    memcpy(h->tp.max_act, c->max_act, sizeof h->tp.max_act);
    h->tp.obstacle_type = c->obstacle_type;
    memcpy(h->tp.lambda_chem, c->lambda_chem, sizeof h->tp.lambda_chem);
    memcpy(h->tp.lambda_pers, c->lambda_pers, sizeof h->tp.lambda_pers);
    for (int k = 0; k < 4; k++) h->tp.inv_len[k] = k ? 1.0 / std::sqrt((double)k) : 0.0;
    h->cfg.chem_field = nullptr;
    for (int a = 0; a < CPM_MAX_TYPES; a++) {
        if (c->lambda_p[a]) h->perim = true;
        if (c->lambda_act[a]) h->act = true;
    }
    h->t = c->t0;
    h->sp = 0;
    h->g = 0;
    if (c->n_cells >= 1) {
        h->v_ref = c->v_target[c->cell_type[1]];
        h->a_ref = c->a_target[c->cell_type[1]];
    }

    const size_t nv = (size_t)h->n_cells + 1;
    CUDA_TRY(h, cudaMalloc(&h->lat, sizeof(int32_t) * h->n_sites));
    CUDA_TRY(h, cudaMalloc(&h->cell_type, nv));
    CUDA_TRY(h, cudaMalloc(&h->tallies, sizeof(int32_t) * nv * 6));
    CUDA_TRY(h, cudaMalloc(&h->pend, sizeof(int4) * 2 * (size_t)h->n_active));
    CUDA_TRY(h, cudaMalloc(&h->flags, 2 * (size_t)h->n_active));
    CUDA_TRY(h, cudaMalloc(&h->counters, sizeof(unsigned long long) * 2));
    if (h->tile) {
        CUDA_TRY(h, cudaMalloc(&h->error_flag, sizeof(int)));
        CUDA_TRY(h, cudaMemsetAsync(h->error_flag, 0, sizeof(int), h->stream));
    }
    CUDA_TRY(h, cudaMemsetAsync(h->counters, 0, sizeof(unsigned long long) * 2, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->lat, c->init_lattice, sizeof(int32_t) * h->n_sites, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(h->cell_type, c->cell_type, nv, cudaMemcpyHostToDevice, h->stream));
    if (h->act) {
        // stamps for the Act values as seen after MCS t0-1: age Max - act, or 128 (no activity)
        std::vector<uint8_t> st(h->n_sites);
        const int64_t tl = c->t0 - 1;
        for (uint64_t x = 0; x < h->n_sites; x++) {
            const int32_t v = c->init_lattice[x];
            const int a = c->init_act ? c->init_act[x] : 0;
            if (v > 0 && a > 0)
                st[x] = (uint8_t)((tl - (c->max_act[c->cell_type[v]] - a)) & 255);
            else
                st[x] = (uint8_t)((c->t0 - 128) & 255);
        }
        CUDA_TRY(h, cudaMalloc(&h->act_tmp, h->n_sites));
        // a copy from pageable memory returns once the source has been staged
        CUDA_TRY(h, cudaMemcpyAsync(h->act_tmp, st.data(), h->n_sites, cudaMemcpyHostToDevice, h->stream));
        // the stamps go into the high byte of the lattice words
        CUDA_TRY(h, launch_pack_ids(h->lat, h->lat, h->act_tmp, h->n_sites, h->stream));
        h->launches += 1;
    }
    int rc = cache ? build_tables_cached(h, cache) : build_tables(h);
    if (rc) return rc;
    {
        std::vector<int32_t> ln, ex;
        ln_expq_tables(ln, ex);
        for (int a = 0; a < CPM_MAX_TYPES; a++) {
            const int m = c->max_act[a] < 0 ? 0 : (c->max_act[a] > 127 ? 127 : c->max_act[a]);
            h->tp.gm_max[a] = m > 0 ? ex[ln[m] >> 6] : 0;
        }
    }
    rc = reset_tallies(h);
    if (rc) return rc;
    if (c->chem_field) {
        const size_t bytes = sizeof(int16_t) * (size_t)h->n_sites * (size_t)c->dim;
        CUDA_TRY(h, cudaMalloc(&h->chem, bytes));
        CUDA_TRY(h, cudaMemcpyAsync(h->chem, c->chem_field, bytes, cudaMemcpyHostToDevice, h->stream));
    }
    for (int a = 0; a < CPM_MAX_TYPES; a++) {
        h->pp.lambda[a] = c->lambda_pers[a];
        h->pp.dt[a] = c->dt_pers[a];
        h->pp.mu[a] = c->mu_pers[a];
        if (c->lambda_pers[a] != 0) {
            h->pers = true;
            h->pers_H = std::max<int32_t>(h->pers_H, c->dt_pers[a] + 1);
        }
    }
    if (h->pers) {
        const size_t nc = (size_t)h->n_cells + 1;
        CUDA_TRY(h, cudaMalloc(&h->pers_dir, sizeof(double) * 3 * nc));
        CUDA_TRY(h, cudaMalloc(&h->pers_hist, sizeof(double) * 3 * nc * (size_t)h->pers_H));
        CUDA_TRY(h, cudaMalloc(&h->pers_item, sizeof(ObserveItem)));
        CUDA_TRY(h, cudaMalloc(&h->pers_cells, sizeof(int64_t) * kObsFields * nc));
        CUDA_TRY(h, cudaMalloc(&h->pers_member, sizeof(int64_t) * 2));
        CUDA_TRY(h, cudaMemsetAsync(h->pers_dir, 0, sizeof(double) * 3 * nc, h->stream));
        // all-ones bytes are a NaN: no centroid recorded yet
        CUDA_TRY(h, cudaMemsetAsync(h->pers_hist, 0xFF, sizeof(double) * 3 * nc * (size_t)h->pers_H, h->stream));
        ObserveItem it{};
        it.lat = h->lat;
        it.accepts = h->counters;
        it.nx = (uint32_t)c->nx;
        it.ny = (uint32_t)c->ny;
        it.nz = (uint32_t)(c->dim == 3 ? c->nz : 1);
        it.dim = (uint32_t)c->dim;
        it.row0 = 0;
        it.n_cells = h->n_cells;
        CUDA_TRY(h, cudaMemcpyAsync(h->pers_item, &it, sizeof it, cudaMemcpyHostToDevice, h->stream));
        rc = pers_step(h);  // the centroids at t0: the first look-back point
        if (rc) return rc;
    }
    if (!cache) CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

// cpm_create for a member of a batch: tables from the batch's cache, no stream synchronisation
int create_member(const cpm_config *cfg, void *cuda_stream, TableCache *cache, cpm_handle **out)
{
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    cpm_handle *h = new (std::nothrow) cpm_handle();
    if (!h) return fail(nullptr, CPM_E_NOMEM, "host allocation failed");
    h->stream = (cudaStream_t)cuda_stream;
    rc = create_impl(h, cfg, cache);
    if (rc) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return CPM_OK;
}

bool bad(const cpm_handle *h) { return h == nullptr; }

}  // namespace

extern "C" {

int cpm_create(const cpm_config *cfg, void *cuda_stream, cpm_handle **out)
{
    if (!out) return fail(nullptr, CPM_E_INVALID, "out is NULL");
    *out = nullptr;
    int rc = validate(cfg);
    if (rc) return rc;
    cpm_handle *h = new (std::nothrow) cpm_handle();
    if (!h) return fail(nullptr, CPM_E_NOMEM, "host allocation failed");
    h->stream = (cudaStream_t)cuda_stream;
    rc = create_impl(h, cfg);
    if (rc) {
        g_create_error = h->err;
        free_all(h);
        delete h;
        return rc;
    }
    *out = h;
    return CPM_OK;
}

int cpm_step_subpasses(cpm_handle *h, int64_t n)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (n < 0) return fail(h, CPM_E_INVALID, "n must be >= 0");
    for (int64_t i = 0; i < n; i++) {
        int rc = h->tile ? run_epoch(h) : run_subpass(h);
        if (rc) return rc;
    }
    return CPM_OK;
}

int cpm_step(cpm_handle *h, int64_t n_mcs)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (n_mcs < 0) return fail(h, CPM_E_INVALID, "n_mcs must be >= 0");
    return cpm_step_subpasses(h, n_mcs * (int64_t)h->per_mcs);
}

int cpm_read_lattice(cpm_handle *h, int32_t *dst, int dst_is_device)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!dst) return fail(h, CPM_E_INVALID, "dst is NULL");
    if (int rc = check_error_flag(h)) return rc;
    if (!h->act) {
        CUDA_TRY(h, cudaMemcpyAsync(dst, h->lat, sizeof(int32_t) * h->n_sites,
                                    dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    } else if (dst_is_device) {
        CUDA_TRY(h, launch_unpack_ids(h->lat, dst, h->n_sites, h->stream));
        h->launches += 1;
    } else {
        // the ids of the packed words, chunk by chunk through the staging buffer
        if (int rc = ensure_stage(h)) return rc;
        for (uint64_t x = 0; x < h->n_sites; x += h->stage_n) {
            const uint64_t m = std::min<uint64_t>(h->stage_n, h->n_sites - x);
            CUDA_TRY(h, launch_unpack_ids(h->lat + x, h->stage, m, h->stream));
            CUDA_TRY(h, cudaMemcpyAsync(dst + x, h->stage, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, h->stream));
            h->launches += 1;
        }
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

int cpm_read_tallies(cpm_handle *h, int32_t *V, int32_t *A, int dst_is_device)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (int rc = check_error_flag(h)) return rc;
    const int cur = (int)(h->g & 1);
    const size_t bytes = sizeof(int32_t) * (h->n_cells + 1);
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (V) CUDA_TRY(h, cudaMemcpyAsync(V, V_buf(h, cur), bytes, kind, h->stream));
    if (A) CUDA_TRY(h, cudaMemcpyAsync(A, A_buf(h, cur), bytes, kind, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

int cpm_track_centroids(cpm_handle *h, int32_t on)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (on != 0 && on != 1) return fail(h, CPM_E_INVALID, "on must be 0 or 1");
    if (on && h->tile) return fail(h, CPM_E_INVALID, "centroid tracking runs on the global schedule only");
    if (int rc = check_error_flag(h)) return rc;
    if (!on) {
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->csum);
        cudaFree(h->tpend);
        cudaFree(h->track_anchor);
        h->csum = nullptr;
        h->tpend = nullptr;
        h->track_anchor = nullptr;
        return CPM_OK;
    }
    if (h->csum) return CPM_OK;
    const size_t nc = (size_t)h->n_cells + 1;
    cudaError_t e = cudaMalloc(&h->csum, sizeof(long long) * 6 * nc);
    if (e == cudaSuccess) e = cudaMalloc(&h->tpend, sizeof(int2) * 2 * (size_t)h->n_active);
    if (e == cudaSuccess) e = cudaMalloc(&h->track_anchor, sizeof(uint32_t) * nc);
    if (e != cudaSuccess) {
        cudaFree(h->csum);
        cudaFree(h->tpend);
        cudaFree(h->track_anchor);
        h->csum = nullptr;
        h->tpend = nullptr;
        h->track_anchor = nullptr;
        return fail(h, e == cudaErrorMemoryAllocation ? CPM_E_NOMEM : CPM_E_CUDA, "cudaMalloc: %s",
                    cudaGetErrorString(e));
    }
    // the tallies from the lattice into both buffers, pending changes dropped, the sums started
    return reset_tallies(h);
}

int cpm_read_centroid_sums(cpm_handle *h, int64_t *S, int dst_is_device)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!S) return fail(h, CPM_E_INVALID, "S is NULL");
    if (!h->csum) return fail(h, CPM_E_INVALID, "centroid tracking is off (cpm_track_centroids)");
    if (int rc = check_error_flag(h)) return rc;
    const int cur = (int)(h->g & 1);
    CUDA_TRY(h, cudaMemcpyAsync(S, S_buf(h, cur), sizeof(long long) * 3 * ((size_t)h->n_cells + 1),
                                dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

int cpm_read_persistence(cpm_handle *h, double *dir)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!dir) return fail(h, CPM_E_INVALID, "dir is NULL");
    const size_t n = 3 * ((size_t)h->n_cells + 1);
    if (!h->pers) {
        memset(dir, 0, sizeof(double) * n);
        return CPM_OK;
    }
    CUDA_TRY(h, cudaMemcpyAsync(dir, h->pers_dir, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

int cpm_read_act(cpm_handle *h, uint8_t *dst, int dst_is_device)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!dst) return fail(h, CPM_E_INVALID, "dst is NULL");
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!h->act) {
        if (dst_is_device)
            CUDA_TRY(h, cudaMemsetAsync(dst, 0, h->n_sites, h->stream));
        else
            memset(dst, 0, h->n_sites);
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        return CPM_OK;
    }
    if (!h->act_tmp) CUDA_TRY(h, cudaMalloc(&h->act_tmp, h->n_sites));
    const int64_t t_last = h->sp == 0 ? h->t - 1 : h->t;
    CUDA_TRY(h, launch_act_values(h->lat, h->cell_type, h->tp, h->n_sites, (uint32_t)t_last, h->act_tmp,
                                  h->stream));
    h->launches += 1;
    CUDA_TRY(h, cudaMemcpyAsync(dst, h->act_tmp, h->n_sites, kind, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return CPM_OK;
}

int cpm_load_lattice(cpm_handle *h, const int32_t *src, int src_is_device)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!src) return fail(h, CPM_E_INVALID, "src is NULL");
    if (!h->act) {
        CUDA_TRY(h, cudaMemcpyAsync(h->lat, src, sizeof(int32_t) * h->n_sites,
                                    src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    } else if (src_is_device) {
        // new ids into the words, their Act stamps kept
        CUDA_TRY(h, launch_pack_ids(h->lat, src, nullptr, h->n_sites, h->stream));
        h->launches += 1;
    } else {
        if (int rc = ensure_stage(h)) return rc;
        for (uint64_t x = 0; x < h->n_sites; x += h->stage_n) {
            const uint64_t m = std::min<uint64_t>(h->stage_n, h->n_sites - x);
            CUDA_TRY(h, cudaMemcpyAsync(h->stage, src + x, sizeof(int32_t) * m, cudaMemcpyHostToDevice, h->stream));
            CUDA_TRY(h, launch_pack_ids(h->lat + x, h->stage, nullptr, m, h->stream));
            h->launches += 1;
        }
    }
    return reset_tallies(h);
}

int cpm_stats(cpm_handle *h, cpm_stats_t *out)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!out) return fail(h, CPM_E_INVALID, "out is NULL");
    std::vector<int32_t> V(h->n_cells + 1), A(h->n_cells + 1);
    int rc = cpm_read_tallies(h, V.data(), A.data(), 0);
    if (rc) return rc;
    unsigned long long acc = 0;
    CUDA_TRY(h, cudaMemcpy(&acc, h->counters, sizeof acc, cudaMemcpyDeviceToHost));
    double sv = 0, sv2 = 0, sa = 0, sa2 = 0;
    int32_t live = 0;
    for (int32_t i = 1; i <= h->n_cells; i++) {
        if (V[i] <= 0) continue;
        live++;
        sv += V[i];
        sv2 += (double)V[i] * V[i];
        sa += A[i];
        sa2 += (double)A[i] * A[i];
    }
    memset(out, 0, sizeof *out);
    out->mcs = h->t;
    out->subpass = h->sp;
    out->n_live_cells = live;
    out->attempts = h->attempts;
    out->accepts = (int64_t)acc;
    if (live > 0) {
        out->volume_mean = sv / live;
        out->volume_var = sv2 / live - out->volume_mean * out->volume_mean;
        out->perimeter_mean = sa / live;
        out->perimeter_var = sa2 / live - out->perimeter_mean * out->perimeter_mean;
    }
    return CPM_OK;
}

int cpm_verify(cpm_handle *h, int64_t *n_mismatch)
{
    if (bad(h)) return CPM_E_HANDLE;
    if (!n_mismatch) return fail(h, CPM_E_INVALID, "n_mismatch is NULL");
    int rc = recount(h, V_buf(h, 2), A_buf(h, 2));
    if (rc) return rc;
    const int cur = (int)(h->g & 1);
    CUDA_TRY(h, cudaMemsetAsync(h->counters + 1, 0, sizeof(unsigned long long), h->stream));
    CUDA_TRY(h, launch_compare(V_buf(h, cur), A_buf(h, cur), V_buf(h, 2), A_buf(h, 2), h->n_cells + 1,
                               h->counters + 1, h->stream));
    h->launches += 1;
    unsigned long long bad_cells = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&bad_cells, h->counters + 1, sizeof bad_cells, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    *n_mismatch = (int64_t)bad_cells;
    return CPM_OK;
}

int64_t cpm_kernel_launches(const cpm_handle *h) { return h ? h->launches : 0; }

const char *cpm_last_error(const cpm_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

void cpm_destroy(cpm_handle *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"

// ===========================================================================
// Batched ensembles: many independent lattices advanced by shared launches.
// Each lattice is a full handle (its own buffers, tables, position); a batch
// step runs round q of every lattice that still has rounds left in the call,
// with one kernel launch for all of them.
// ===========================================================================
struct cpm_batch {
    std::vector<cpm_handle *> hs;
    int dim = 2;
    bool perim = false, act = false;
    cudaStream_t stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    std::vector<BatchLattice> lats;      // in batch order
    std::vector<uint32_t> order;         // lattice indices by rounds per MCS, descending
    std::vector<uint32_t> items_upto;    // round items of the first k lattices in that order
    uint32_t n_clamp_items = 0;
    uint32_t brick[3] = {8, 4, 4};       // active blocks per CTA (x, y, z)
    BatchLattice *d_lats = nullptr;
    int2 *d_items = nullptr;
    int2 *d_clamp = nullptr;
    ObserveItem *d_obs = nullptr;        // observation items, built on first use
    TableCache *tables = nullptr;        // LN / EXPQ / THR shared by the members
    int64_t obs_max_sites = 0;
    int64_t obs_rows = 0;
    int32_t obs_max_cells = 0;
    double *traj = nullptr;              // centroid tracks of cpm_batch_summarize
    size_t traj_cap = 0;
    cudaGraphExec_t graph = nullptr;     // one MCS of every member
    int64_t graph_launches = 0;          // kernels in one replay
    // the persistent loop (cpm_batch_set_persistent)
    bool persistent = false;
    bool test_absent = false;            // cpm_batch_set_persistent(b, 2, ...): timeout-path test
    long long max_polls = 1ll << 24;     // bound of each grid-barrier wait (polls about 100 ns apart)
    uint32_t *d_upto_q = nullptr;        // round items per round q
    uint32_t r_max_items = 0;            // items of the fullest round
    unsigned long long *d_bar = nullptr; // barrier counter
    unsigned *d_next = nullptr;          // per-round item counters of the persistent loop
    int *d_err = nullptr;                // barrier timeout flag
    uint32_t loop_grid = 0;              // CTAs of the last persistent launch
    bool track = false;                  // composite variable tracking in every member
    bool descriptors_dirty = true;
    int64_t launches = 0;
    std::string err;
};

namespace {
thread_local std::string g_batch_create_error;  // per calling thread, as g_create_error

int bfail(cpm_batch *b, int code, const std::string &msg)
{
    if (b) b->err = msg; else g_batch_create_error = msg;
    return code;
}

void batch_drop_graph(cpm_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

void batch_free(cpm_batch *b)
{
    batch_drop_graph(b);
    for (cpm_handle *h : b->hs) cpm_destroy(h);
    delete b->tables;
    b->tables = nullptr;
    cudaFree(b->d_lats);
    cudaFree(b->d_items);
    cudaFree(b->d_clamp);
    cudaFree(b->d_obs);
    cudaFree(b->traj);
    cudaFree(b->d_upto_q);
    cudaFree(b->d_bar);
    cudaFree(b->d_next);
    cudaFree(b->d_err);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
}

uint32_t batch_threads(const cpm_batch *b) { return b->brick[0] * b->brick[1] * (b->dim == 3 ? b->brick[2] : 1); }

// round items (member, brick) for the current brick shape, members in order of
// rounds per MCS (descending), and the Act clamp items (member, 65,536 sites)
int batch_build_items(cpm_batch *b)
{
    std::vector<int2> items;
    b->items_upto.assign(1, 0);
    const uint32_t bz = b->dim == 3 ? b->brick[2] : 1;
    for (uint32_t l : b->order) {
        const cpm_handle *h = b->hs[l];
        const uint32_t nax = h->nbx / h->cfg.c, nay = h->nby / h->cfg.c;
        const uint32_t naz = h->n_active / (nax * nay);
        const uint32_t nb = ((nax + b->brick[0] - 1) / b->brick[0]) * ((nay + b->brick[1] - 1) / b->brick[1]) *
                            ((naz + bz - 1) / bz);
        for (uint32_t c = 0; c < nb; c++) items.push_back(make_int2((int)l, (int)c));
        b->items_upto.push_back((uint32_t)items.size());
        b->lats[l].base.brick_x = b->brick[0];
        b->lats[l].base.brick_y = b->brick[1];
        b->lats[l].base.brick_z = bz;
    }
    std::vector<int2> clamp;
    for (size_t l = 0; l < b->hs.size(); l++) {
        if (!b->hs[l]->act) continue;
        const uint64_t chunks = (b->hs[l]->n_sites + 65535) / 65536;
        for (uint64_t c = 0; c < chunks; c++) clamp.push_back(make_int2((int)l, (int)c));
    }
    b->n_clamp_items = (uint32_t)clamp.size();
    // items of round q for the persistent loop: those of the members with more than q rounds per MCS
    const uint32_t r_max = b->lats[b->order[0]].R;
    std::vector<uint32_t> upto_q(r_max);
    size_t active = b->order.size();
    for (uint32_t q = 0; q < r_max; q++) {
        while (active > 0 && b->lats[b->order[active - 1]].R <= q) active--;
        upto_q[q] = b->items_upto[active];
    }
    b->r_max_items = r_max > 0 ? upto_q[0] : 0;
    cudaFree(b->d_items);
    cudaFree(b->d_clamp);
    cudaFree(b->d_upto_q);
    b->d_items = nullptr;
    b->d_clamp = nullptr;
    b->d_upto_q = nullptr;
    cudaError_t e = cudaMalloc(&b->d_upto_q, sizeof(uint32_t) * std::max<size_t>(upto_q.size(), 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_upto_q, upto_q.data(), sizeof(uint32_t) * upto_q.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(int2) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_clamp, sizeof(int2) * std::max<size_t>(clamp.size(), 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !clamp.empty())
        e = cudaMemcpy(b->d_clamp, clamp.data(), sizeof(int2) * clamp.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
    b->descriptors_dirty = true;
    batch_drop_graph(b);
    return CPM_OK;
}

// Capture one MCS of every member as a CUDA graph: the Act clamp (members at
// a multiple of 64 MCS), R_max round launches over the members that still
// have rounds, and the advance of every member's MCS and round counters.
int batch_build_graph(cpm_batch *b)
{
    batch_drop_graph(b);
    cudaError_t e = cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
    int64_t n = 0;
    if (b->act) {
        e = launch_batch_clamp(b->d_lats, b->d_clamp, b->n_clamp_items, b->capture_stream);
        n++;
    }
    const uint32_t r_max = b->lats[b->order[0]].R;
    size_t active = b->order.size();
    for (uint32_t q = 0; q < r_max && e == cudaSuccess; q++) {
        while (active > 0 && b->lats[b->order[active - 1]].R <= q) active--;
        e = launch_batch_round(b->dim, b->perim, b->act, b->track, b->d_lats, b->d_items, b->items_upto[active], q,
                               batch_threads(b), b->capture_stream);
        n++;
    }
    if (e == cudaSuccess) {
        e = launch_batch_advance(b->d_lats, (uint32_t)b->lats.size(), b->capture_stream);
        n++;
    }
    if (e == cudaSuccess && b->track) {
        e = launch_batch_track_rewrap(b->dim, b->d_lats, (uint32_t)b->lats.size(), b->capture_stream);
        n++;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->capture_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bfail(b, CPM_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    b->graph_launches = n;
    return CPM_OK;
}
}  // namespace

extern "C" {

int cpm_batch_create(const cpm_config *cfgs, int32_t n, void *cuda_stream, cpm_batch **out)
{
    if (!out) return bfail(nullptr, CPM_E_INVALID, "out is NULL");
    *out = nullptr;
    if (!cfgs || n < 1) return bfail(nullptr, CPM_E_INVALID, "need at least one configuration");
    cpm_batch *b = new (std::nothrow) cpm_batch();
    if (!b) return bfail(nullptr, CPM_E_NOMEM, "host allocation failed");
    b->stream = (cudaStream_t)cuda_stream;
    b->dim = cfgs[0].dim;
    if (b->dim == 2) { b->brick[0] = 16; b->brick[1] = 8; b->brick[2] = 1; }
    b->tables = new (std::nothrow) TableCache();
    if (!b->tables) {
        delete b;
        return bfail(nullptr, CPM_E_NOMEM, "host allocation failed");
    }
    {
        // the threshold tables of the distinct temperatures, computed on host threads
        std::vector<double> temps;
        for (int32_t i = 0; i < n; i++) {
            const double T = cfgs[i].temperature;
            if (T > 0.0 && T <= 1e4 && !b->tables->host_thr.count(t_key(T))) {
                b->tables->host_thr[t_key(T)];
                temps.push_back(T);
            }
        }
        std::vector<std::vector<uint32_t> *> slots;
        for (double T : temps) slots.push_back(&b->tables->host_thr[t_key(T)]);
        const unsigned hw = std::thread::hardware_concurrency();
        const size_t nt = std::min<size_t>(temps.size(), std::max(1u, std::min(hw, 16u)));
        std::vector<std::thread> pool;
        for (size_t w = 0; w < nt; w++)
            pool.emplace_back([&, w]() {
                for (size_t j = w; j < temps.size(); j += nt)
                    if (!thr_table(temps[j], *slots[j])) slots[j]->clear();
            });
        for (auto &th : pool) th.join();
    }
    for (int32_t i = 0; i < n; i++) {
        bool pers = false;
        for (int a = 0; a < CPM_MAX_TYPES; a++) pers |= cfgs[i].lambda_pers[a] != 0;
        if (pers) {
            batch_free(b);
            delete b;
            return bfail(nullptr, CPM_E_INVALID, "configuration " + std::to_string(i) +
                                                     ": the persistence term needs single-lattice handles");
        }
        if (cfgs[i].dim != b->dim || cfgs[i].tile != 0) {
            batch_free(b);
            delete b;
            return bfail(nullptr, CPM_E_INVALID, "a batch needs one dimension and the global schedule (tile = 0)");
        }
        cpm_handle *h = nullptr;
        int rc = create_member(&cfgs[i], cuda_stream, b->tables, &h);
        if (rc) {
            std::string msg = "configuration " + std::to_string(i) + ": " + cpm_last_error(nullptr);
            batch_free(b);
            delete b;
            return bfail(nullptr, rc, msg);
        }
        b->hs.push_back(h);
        b->perim |= h->perim;
        b->act |= h->act;
    }
    for (cpm_handle *h : b->hs) {
        BatchLattice L;
        memset(&L, 0, sizeof L);
        RoundArgs &a = L.base;
        a.lat = h->lat;
        a.packed = h->act ? 1u : 0u;
        a.stream_loads = h->act && h->cfg.a >= 8 ? 1u : 0u;
        a.cell_type = h->cell_type;
        a.thr = h->thr;
        a.ln_tab = h->ln_tab;
        a.expq = h->expq;
        a.accepts = h->counters;
        a.L = h->L;
        a.nx = h->cfg.nx; a.ny = h->cfg.ny; a.nz = h->cfg.nz;
        a.s = h->s; a.c = h->cfg.c; a.sd = h->sd;
        a.nbx = h->nbx; a.nby = h->nby;
        a.nax = h->nbx / h->cfg.c; a.nay = h->nby / h->cfg.c;
        a.n_active = h->n_active;
        a.key0 = (uint32_t)h->cfg.seed;
        a.key1 = (uint32_t)(h->cfg.seed >> 32);
        a.tp = h->tp;
        a.chem = h->chem;
        for (int p = 0; p < 2; p++) {
            L.V[p] = V_buf(h, p);
            L.A[p] = A_buf(h, p);
            L.pend[p] = h->pend + (size_t)p * h->n_active;
            L.flag[p] = h->flags + (size_t)p * h->n_active;
        }
        L.k = h->k;
        L.C = h->C;
        L.R = h->per_sub_mcs * h->k;
        L.n_cells = h->n_cells;
        b->lats.push_back(L);
    }
    b->order.resize(n);
    for (int32_t i = 0; i < n; i++) b->order[i] = (uint32_t)i;
    std::stable_sort(b->order.begin(), b->order.end(),
                     [&](uint32_t x, uint32_t y) { return b->lats[x].R > b->lats[y].R; });
    cudaError_t e = cudaMalloc(&b->d_lats, sizeof(BatchLattice) * b->lats.size());
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return bfail(nullptr, e == cudaErrorMemoryAllocation ? CPM_E_NOMEM : CPM_E_CUDA, cudaGetErrorString(e));
    }
    int rc = batch_build_items(b);
    if (rc) {
        std::string msg = b->err;
        batch_free(b);
        delete b;
        return bfail(nullptr, rc, msg);
    }
    e = cudaStreamSynchronize(b->stream);  // the members' uploads and tally counts
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        return bfail(nullptr, CPM_E_CUDA, cudaGetErrorString(e));
    }
    *out = b;
    return CPM_OK;
}

int cpm_batch_step(cpm_batch *b, int64_t n_mcs)
{
    if (!b) return CPM_E_HANDLE;
    if (n_mcs < 0) return bfail(b, CPM_E_INVALID, "n_mcs must be >= 0");
    if (n_mcs == 0) return CPM_OK;
    if (b->descriptors_dirty) {
        for (size_t l = 0; l < b->hs.size(); l++) {
            if (b->hs[l]->sp != 0) return bfail(b, CPM_E_INVALID, "every lattice must be at an MCS boundary");
            b->lats[l].t_start = b->hs[l]->t;
            b->lats[l].g_start = b->hs[l]->g;
        }
        cudaError_t e = cudaMemcpyAsync(b->d_lats, b->lats.data(), sizeof(BatchLattice) * b->lats.size(),
                                        cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
        b->descriptors_dirty = false;
    }
    if (b->persistent) {
        // one cooperative launch runs all n_mcs MCS; its barrier waits are bounded
        for (int64_t done = 0; done < n_mcs;) {
            const uint32_t chunk = (uint32_t)std::min<int64_t>(n_mcs - done, 1 << 16);
            BatchLoopArgs p{};
            p.lats = b->d_lats;
            p.n_lats = (uint32_t)b->lats.size();
            p.items = b->d_items;
            p.upto_q = b->d_upto_q;
            p.r_max = b->lats[b->order[0]].R;
            p.clamp = b->d_clamp;
            p.n_clamp = b->act ? b->n_clamp_items : 0;
            p.n_mcs = chunk;
            p.bar = b->d_bar;
            p.max_polls = b->max_polls;
            p.err = b->d_err;
            p.max_items = b->r_max_items;
            p.test_absent = b->test_absent ? 1 : 0;
            p.next = b->d_next;
            cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned long long), b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned) * p.r_max, b->stream);
            if (e == cudaSuccess) e = launch_batch_loop(b->dim, b->perim, b->act, p, batch_threads(b), b->stream,
                                                        &b->loop_grid);
            int timed_out = 0;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&timed_out, b->d_err, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
            b->launches += 1;
            if (timed_out)
                return bfail(b, CPM_E_STATE,
                             "a grid-barrier wait of the persistent loop timed out; the lattices are in an unspecified "
                             "state");
            done += chunk;
        }
    } else {
        if (!b->graph) {
            int rc = batch_build_graph(b);
            if (rc) return rc;
        }
        for (int64_t k = 0; k < n_mcs; k++) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
        }
        b->launches += n_mcs * b->graph_launches;
    }
    for (size_t l = 0; l < b->hs.size(); l++) {
        cpm_handle *h = b->hs[l];
        h->t += n_mcs;
        h->g += (uint64_t)n_mcs * b->lats[l].R;
        h->attempts += n_mcs * (int64_t)h->n_sites;
    }
    return CPM_OK;
}

int cpm_batch_set_persistent(cpm_batch *b, int32_t on, int64_t max_polls)
{
    if (!b) return CPM_E_HANDLE;
    if (on && !b->d_bar) {
        cudaError_t e = cudaMalloc(&b->d_bar, sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_next, sizeof(unsigned) * std::max<uint32_t>(1u, b->lats[b->order[0]].R));
        if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(int));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(int), b->stream);
        if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
    }
    if (on < 0 || on > 2) return bfail(b, CPM_E_INVALID, "on must be 0, 1 or 2");
    if (on != 0 && b->track) return bfail(b, CPM_E_INVALID, "the persistent loop does not track centroids");
    b->persistent = on != 0;
    b->test_absent = on == 2;
    b->max_polls = max_polls >= 0 ? (long long)max_polls : (1ll << 24);
    return CPM_OK;
}

int cpm_batch_track_centroids(cpm_batch *b, int32_t on)
{
    if (!b) return CPM_E_HANDLE;
    if (on != 0 && on != 1) return bfail(b, CPM_E_INVALID, "on must be 0 or 1");
    if (on && b->persistent) return bfail(b, CPM_E_INVALID, "the persistent loop does not track centroids");
    for (size_t l = 0; l < b->hs.size(); l++) {
        cpm_handle *h = b->hs[l];
        if (int rc = cpm_track_centroids(h, on))
            return bfail(b, rc, "lattice " + std::to_string(l) + ": " + cpm_last_error(h));
        for (int p = 0; p < 2; p++) {
            b->lats[l].S[p] = on ? S_buf(h, p) : nullptr;
            b->lats[l].tpend[p] = on ? h->tpend + (size_t)p * h->n_active : nullptr;
        }
    }
    b->track = on != 0;
    b->descriptors_dirty = true;
    batch_drop_graph(b);
    return CPM_OK;
}

int cpm_batch_read_centroid_sums(cpm_batch *b, int32_t idx, int64_t *S, int dst_is_device)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "idx out of range");
    if (int rc = cpm_read_centroid_sums(b->hs[idx], S, dst_is_device)) return bfail(b, rc, cpm_last_error(b->hs[idx]));
    return CPM_OK;
}

int cpm_batch_autotune(cpm_batch *b, int32_t n_mcs_each, int32_t *choice)
{
    if (!b) return CPM_E_HANDLE;
    if (n_mcs_each < 1) return bfail(b, CPM_E_INVALID, "n_mcs_each must be >= 1");
    static const uint32_t cand3[][3] = {{8, 4, 4}, {4, 4, 4}, {8, 8, 4}, {16, 4, 2}, {32, 4, 1}, {128, 1, 1}, {8, 8, 2}};
    static const uint32_t cand2[][3] = {{16, 8, 1}, {16, 16, 1}, {8, 8, 1}, {32, 4, 1}, {128, 1, 1}, {64, 4, 1}};
    const int nc = b->dim == 3 ? 7 : 6;
    std::vector<float> total(nc, 0.0f);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = CPM_OK;
    // passes interleave the candidates, so that each is timed on a similar
    // spread of simulation states (the cost of an MCS drifts as cells grow)
    for (int pass = 0; pass < 1 + n_mcs_each && rc == CPM_OK; pass++) {
        for (int k = 0; k < nc && rc == CPM_OK; k++) {
            const uint32_t *cb = b->dim == 3 ? cand3[k] : cand2[k];
            b->brick[0] = cb[0]; b->brick[1] = cb[1]; b->brick[2] = cb[2];
            rc = batch_build_items(b);
            if (!rc) rc = cpm_batch_step(b, 0);
            if (!rc && !b->graph) rc = batch_build_graph(b);
            if (rc) break;
            // a freshly built graph is uploaded on its first launch: pass 0 only warms up
            cudaEventRecord(e0, b->stream);
            rc = cpm_batch_step(b, 1);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (pass > 0) total[k] += ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    int best_k = 0;
    for (int k = 1; k < nc; k++)
        if (total[k] < total[best_k]) best_k = k;
    const uint32_t *cb = b->dim == 3 ? cand3[best_k] : cand2[best_k];
    b->brick[0] = cb[0]; b->brick[1] = cb[1]; b->brick[2] = cb[2];
    rc = batch_build_items(b);
    if (rc) return rc;
    if (choice) *choice = best_k;
    return CPM_OK;
}

int32_t cpm_batch_size(const cpm_batch *b) { return b ? (int32_t)b->hs.size() : 0; }

int cpm_batch_read_lattice(cpm_batch *b, int32_t idx, int32_t *dst, int dst_is_device)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "lattice index out of range");
    int rc = cpm_read_lattice(b->hs[idx], dst, dst_is_device);
    if (rc) b->err = cpm_last_error(b->hs[idx]);
    return rc;
}

int cpm_batch_load_lattice(cpm_batch *b, int32_t idx, const int32_t *src, int src_is_device)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "lattice index out of range");
    int rc = cpm_load_lattice(b->hs[idx], src, src_is_device);
    if (rc) b->err = cpm_last_error(b->hs[idx]);
    return rc;
}

int cpm_batch_read_tallies(cpm_batch *b, int32_t idx, int32_t *V, int32_t *A, int dst_is_device)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "lattice index out of range");
    int rc = cpm_read_tallies(b->hs[idx], V, A, dst_is_device);
    if (rc) b->err = cpm_last_error(b->hs[idx]);
    return rc;
}

int cpm_batch_read_act(cpm_batch *b, int32_t idx, uint8_t *dst, int dst_is_device)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "lattice index out of range");
    int rc = cpm_read_act(b->hs[idx], dst, dst_is_device);
    if (rc) b->err = cpm_last_error(b->hs[idx]);
    return rc;
}

int cpm_batch_stats(cpm_batch *b, int32_t idx, cpm_stats_t *out)
{
    if (!b) return CPM_E_HANDLE;
    if (idx < 0 || idx >= (int32_t)b->hs.size()) return bfail(b, CPM_E_INVALID, "lattice index out of range");
    int rc = cpm_stats(b->hs[idx], out);
    if (rc) b->err = cpm_last_error(b->hs[idx]);
    return rc;
}

int64_t cpm_batch_kernel_launches(const cpm_batch *b)
{
    if (!b) return 0;
    int64_t n = b->launches;
    for (const cpm_handle *h : b->hs) n += h->launches;
    return n;
}

const char *cpm_batch_last_error(const cpm_batch *b) { return b ? b->err.c_str() : g_batch_create_error.c_str(); }

namespace {
int batch_obs_items(cpm_batch *b)
{
    if (!b->d_obs) {
        std::vector<ObserveItem> items(b->hs.size());
        int64_t row = 0;
        for (size_t l = 0; l < b->hs.size(); l++) {
            const cpm_handle *h = b->hs[l];
            ObserveItem &it = items[l];
            it.lat = h->lat;
            it.accepts = h->counters;
            it.nx = (uint32_t)h->cfg.nx;
            it.ny = (uint32_t)h->cfg.ny;
            it.nz = (uint32_t)(h->dim == 3 ? h->cfg.nz : 1);
            it.dim = (uint32_t)h->dim;
            it.row0 = row;
            it.n_cells = h->n_cells;
            it.pad_ = 0;
            it.v_ref = h->v_ref;
            it.a_ref = h->a_ref;
            row += (int64_t)h->n_cells + 1;
            b->obs_max_sites = std::max<int64_t>(b->obs_max_sites, (int64_t)h->n_sites);
            b->obs_max_cells = std::max<int32_t>(b->obs_max_cells, h->n_cells);
        }
        b->obs_rows = row;
        cudaError_t e = cudaMalloc(&b->d_obs, sizeof(ObserveItem) * items.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_obs, items.data(), sizeof(ObserveItem) * items.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) {
            cudaFree(b->d_obs);
    cudaFree(b->traj);
            b->d_obs = nullptr;
            return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
        }
    }
    return CPM_OK;
}
}  // namespace

int cpm_batch_observe(cpm_batch *b, int64_t *cells_out, int64_t *member_out)
{
    if (!b) return CPM_E_HANDLE;
    if (!cells_out || !member_out) return bfail(b, CPM_E_INVALID, "cells_out and member_out are required");
    if (int rc = batch_obs_items(b)) return rc;
    cudaError_t e = launch_observe(b->dim, b->d_obs, (uint32_t)b->hs.size(), b->obs_max_sites, cells_out, member_out,
                                   b->stream);
    if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
    b->launches += 3;
    return CPM_OK;
}

int cpm_batch_summarize(cpm_batch *b, const int64_t *cells_hist, const int64_t *member_hist, int32_t n_snap,
                        int32_t every, double *out)
{
    if (!b) return CPM_E_HANDLE;
    if (!cells_hist || !member_hist || !out) return bfail(b, CPM_E_INVALID, "null buffer");
    if (b->dim != 2) return bfail(b, CPM_E_INVALID, "summary statistics are defined for 2D lattices");
    if (n_snap < 1 || n_snap > kSummaryMaxSnap) return bfail(b, CPM_E_INVALID, "n_snap must be in 1..1024");
    if (every < 1) return bfail(b, CPM_E_INVALID, "every must be >= 1");
    if (int rc = batch_obs_items(b)) return rc;
    const size_t need = (size_t)b->obs_rows * 2 * (size_t)n_snap;
    if (need > b->traj_cap) {
        cudaFree(b->traj);
        b->traj = nullptr;
        b->traj_cap = 0;
        cudaError_t e = cudaMalloc(&b->traj, sizeof(double) * need);
        if (e != cudaSuccess) return bfail(b, CPM_E_NOMEM, cudaGetErrorString(e));
        b->traj_cap = need;
    }
    cudaError_t e = launch_summarize(b->d_obs, (uint32_t)b->hs.size(), b->obs_max_cells, cells_hist, b->obs_rows,
                                     member_hist, n_snap, every, b->traj, out, b->stream);
    if (e != cudaSuccess) return bfail(b, CPM_E_CUDA, cudaGetErrorString(e));
    b->launches += 1;
    return CPM_OK;
}

void cpm_batch_destroy(cpm_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

}  // extern "C"
