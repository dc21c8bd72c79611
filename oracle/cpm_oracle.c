/*
 * CPU oracle for the cellular Potts model (CPM) copy-attempt sweep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The CUDA library
 * neither links, calls nor includes anything here, and nothing here is
 * derived from it.
 *
 * Two oracles, written plainly and without any blocking or fusion:
 *
 *  (a) orc_serial_run: the serial CPM Markov chain of the paper's Methods
 *      ("Cellular Potts model and model variants", Eq. 1 and Eq. 2): one MCS
 *      is N copy attempts; each attempt picks a target site j uniformly and a
 *      source i uniformly among j's Moore neighbours, computes the energy
 *      change of copying sigma_i into j in double precision and accepts with
 *      probability min(1, exp(-dH/T)).  Its own RNG is xoshiro256**
 *      (Blackman and Vigna, "Scrambled linear pseudorandom number
 *      generators", 2021), which the paper's CPU code also uses ("Optimized
 *      CPU implementation").
 *
 *  (b) orc_replay_run / orc_replay_subpass: a sequential replay of the
 *      parallel checkerboard scheme (Results, "Designing a parallel execution
 *      scheme", Fig. 2A/B and Fig. 3A/B): per MCS, P cycles over c^d colours
 *      in a random order; in each sub-pass every block of the active colour
 *      makes k = s^d/P copy attempts, one per round; every attempt of a round
 *      reads the tallies as they stood when the round began.
 *      Random numbers come from Philox4x32-10 (Salmon et al., "Parallel
 *      random numbers: as easy as 1, 2, 3", SC'11) keyed by the seed and
 *      counted by (block, attempt, MCS, sub-pass), so the replay draws exactly
 *      what any parallel execution of the scheme draws.  Energies are exact
 *      integers (Act in Q4 fixed point) and acceptance compares a uint32 draw
 *      with an integer threshold table.  With params.csum set the replay also
 *      keeps every cell's coordinate sums (composite variable tracking,
 *      Methods, Eq. 10 and Eq. 11; orc_track_init, orc_track_rewrap).
 *
 * Conventions (data, identical for every consumer): lattice x-fastest; id 0
 * is the medium (type 0), ids > 0 are cells, id -1 is a frozen obstacle of
 * type obstacle_type; the Moore neighbourhood is listed in lexicographic
 * (dz, dy, dx) order over {-1,0,1}^d without the centre.  Boundaries are
 * periodic.  Medium tallies are not tracked.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXT 8

typedef struct {
    int32_t dim, nx, ny, nz;
    int32_t J[ORC_MAXT][ORC_MAXT];
    int32_t lambda_v[ORC_MAXT], v_target[ORC_MAXT];
    int32_t lambda_p[ORC_MAXT], a_target[ORC_MAXT];
    int32_t lambda_act[ORC_MAXT], max_act[ORC_MAXT];
    double T;
    int32_t obstacle_type;
    int32_t a, c, P;
    uint64_t seed;
    int32_t n_cells;
    const uint8_t *cell_type; /* n_cells + 1 entries, [0] = medium */
    int32_t tile;             /* 0: global rounds; T > 0: tiled epochs of edge T */
    int32_t tile_cycles;      /* P_T: tile cycles per MCS (divides P) */
    /* motility terms (Eq. 4 to Eq. 7); zero / NULL when unused */
    const int16_t *chem_field;  /* [site][dim] components of the field C in Q14 (16384 = 1) */
    int32_t lambda_chem[ORC_MAXT];
    int32_t lambda_pers[ORC_MAXT];
    double mu_pers[ORC_MAXT];
    int32_t dt_pers[ORC_MAXT];  /* look-back of the persistence update, MCS (>= 1 where lambda_pers != 0) */
    double *pers_dir;           /* state: [n_cells + 1][3] persistence directions p_hat */
    double *pers_hist;          /* state: [pers_hist_len][n_cells + 1][3] centroids, NaN for absent cells */
    int32_t pers_hist_len;      /* > max dt_pers */
    int64_t pers_t0;            /* MCS of the first recorded centroids */
    /* composite variable tracking (Eq. 11); NULL when off (global schedule only) */
    int64_t *csum;              /* state: [n_cells + 1][3] coordinate sums of each cell's sites */
} orc_params;

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3):          */
/* a round multiplies words 0 and 2 by the two round constants, takes  */
/* the 64-bit products apart, and mixes the high halves with the other */
/* two words and the round key; the key is bumped by the Weyl          */
/* constants between rounds.                                           */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* index in [0, n) from a uint32 draw: high half of the 64-bit product */
static uint32_t scale_draw(uint32_t w, uint32_t n) { return (uint32_t)(((uint64_t)w * n) >> 32); }

/* ------------------------------------------------------------------ */
/* xoshiro256** with splitmix64 seeding (Blackman & Vigna 2021)        */
/* ------------------------------------------------------------------ */
static uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static uint64_t xoshiro_next(uint64_t s[4])
{
    uint64_t result = rotl64(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return result;
}

void orc_xoshiro_seed(uint64_t seed, uint64_t s[4])
{
    uint64_t z = seed;
    for (int i = 0; i < 4; i++) {
        z += 0x9E3779B97F4A7C15ull;
        uint64_t x = z;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        s[i] = x ^ (x >> 31);
    }
}

static uint64_t rand_below(uint64_t s[4], uint64_t n) { return ((xoshiro_next(s) >> 32) * n) >> 32; }
static double rand_unit(uint64_t s[4]) { return (double)(xoshiro_next(s) >> 11) * 0x1.0p-53; }

/* ------------------------------------------------------------------ */
/* lattice geometry                                                    */
/* ------------------------------------------------------------------ */
int orc_neighbour_offsets(int dim, int32_t off[26][3])
{
    int n = 0;
    int zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                off[n][0] = dx; off[n][1] = dy; off[n][2] = dz;
                n++;
            }
    return n;
}

static int64_t wrap(int64_t v, int64_t n) { v %= n; return v < 0 ? v + n : v; }

static int64_t neighbour(const orc_params *p, int64_t site, const int32_t o[3])
{
    int64_t x = site % p->nx, y = (site / p->nx) % p->ny, z = site / ((int64_t)p->nx * p->ny);
    x = wrap(x + o[0], p->nx);
    y = wrap(y + o[1], p->ny);
    z = wrap(z + o[2], p->nz);
    return x + (int64_t)p->nx * (y + (int64_t)p->ny * z);
}

static int type_of(const orc_params *p, int32_t sigma)
{
    if (sigma < 0) return p->obstacle_type;
    return p->cell_type[sigma];
}

static int act_enabled(const orc_params *p)
{
    for (int t = 0; t < ORC_MAXT; t++)
        if (p->lambda_act[t] != 0) return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* tallies: V = number of sites, A = number of (site, neighbour) pairs */
/* with the site in the cell and the neighbour not (Eq. 3 and its      */
/* definition of A)                                                    */
/* ------------------------------------------------------------------ */
void orc_recount(const orc_params *p, const int32_t *lat, int32_t *V, int32_t *A)
{
    int32_t off[26][3];
    int nb = orc_neighbour_offsets(p->dim, off);
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    memset(V, 0, sizeof(int32_t) * (size_t)(p->n_cells + 1));
    memset(A, 0, sizeof(int32_t) * (size_t)(p->n_cells + 1));
    for (int64_t x = 0; x < N; x++) {
        int32_t s = lat[x];
        if (s <= 0) continue;
        V[s] += 1;
        for (int n = 0; n < nb; n++)
            if (lat[neighbour(p, x, off[n])] != s) A[s] += 1;
    }
}

/* ------------------------------------------------------------------ */
/* Integer energy change of copying sigma_i into site j (Eq. 1 with     */
/* each unordered neighbour pair counted once, plus Eq. 3).  Vi, Vj,    */
/* Ai, Aj are the tallies the attempt sees.  Returns dH; m_i and m_j    */
/* are the numbers of j's neighbours that belong to sigma_i, sigma_j.   */
/* ------------------------------------------------------------------ */
static int64_t delta_h_int(const orc_params *p, const int32_t *lat, int64_t j, int32_t si, int32_t sj,
                           int64_t Vi, int64_t Vj, int64_t Ai, int64_t Aj, int nb,
                           int32_t off[26][3], int *m_i, int *m_j)
{
    int ti = type_of(p, si), tj = type_of(p, sj);
    int64_t adhesion = 0;
    int mi = 0, mj = 0;
    for (int n = 0; n < nb; n++) {
        int32_t sn = lat[neighbour(p, j, off[n])];
        int tn = type_of(p, sn);
        if (sn != si) adhesion += p->J[ti][tn]; else mi++;
        if (sn != sj) adhesion -= p->J[tj][tn]; else mj++;
    }
    int64_t volume = 0, perimeter = 0;
    int64_t dAi = nb - 2 * mi, dAj = 2 * mj - nb;
    if (si > 0) {
        volume += (int64_t)p->lambda_v[ti] * (2 * (Vi - p->v_target[ti]) + 1);
        perimeter += (int64_t)p->lambda_p[ti] * dAi * (2 * (Ai - p->a_target[ti]) + dAi);
    }
    if (sj > 0) {
        volume += (int64_t)p->lambda_v[tj] * (1 - 2 * (Vj - p->v_target[tj]));
        perimeter += (int64_t)p->lambda_p[tj] * dAj * (2 * (Aj - p->a_target[tj]) + dAj);
    }
    *m_i = mi;
    *m_j = mj;
    return adhesion + volume + perimeter;
}

/* ------------------------------------------------------------------ */
/* Motility terms (Eq. 4 chemotaxis, Eq. 5 persistence).  A copy from the */
/* source i into the target j moves the cell sigma_i (or, when sigma_i is */
/* the medium, sigma_j) along d = j - i; the term is -lambda(tau) x.v     */
/* with x = d / |d| and v the field at i (Eq. 4) or the cell's direction  */
/* p_hat (Eq. 5): copies along v become more likely, as the paper         */
/* describes (the printed sign would make them less likely).  In Q4       */
/* units it is floor(e), e formed by exactly this sequence of rounded     */
/* double operations: chemotaxis e = ((double)(-16 lambda (d.C_q)) /      */
/* 16384) * (1/sqrt(|d|^2)); persistence s = d_x p_x + d_y p_y + d_z p_z  */
/* (left to right), e = (s * (double)(-16 lambda)) * (1/sqrt(|d|^2)).      */
/* ------------------------------------------------------------------ */
static int motility_enabled(const orc_params *p)
{
    for (int t = 0; t < ORC_MAXT; t++)
        if ((p->chem_field && p->lambda_chem[t] != 0) || (p->pers_dir && p->lambda_pers[t] != 0)) return 1;
    return 0;
}

static int pers_enabled(const orc_params *p)
{
    if (!p->pers_dir || !p->pers_hist) return 0;
    for (int t = 0; t < ORC_MAXT; t++)
        if (p->lambda_pers[t] != 0) return 1;
    return 0;
}

static double inv_len(int k) { return 1.0 / sqrt((double)k); }

/* copy direction d = j - i for source i = j + off (the neighbour offset) */
static void copy_dir(const int32_t o[3], int d[3], int *k)
{
    d[0] = -o[0];
    d[1] = -o[1];
    d[2] = -o[2];
    *k = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
}

static int64_t motility_q(const orc_params *p, int64_t i, int32_t si, int32_t sj, const int32_t o[3])
{
    int32_t m = si > 0 ? si : sj;
    int tp = type_of(p, m);
    int d[3], k;
    copy_dir(o, d, &k);
    int64_t dh = 0;
    if (p->chem_field && p->lambda_chem[tp] != 0) {
        const int16_t *c = p->chem_field + i * p->dim;
        int64_t dc = (int64_t)d[0] * c[0] + (int64_t)d[1] * c[1] + (p->dim == 3 ? (int64_t)d[2] * c[2] : 0);
        double e = (double)(-16 * (int64_t)p->lambda_chem[tp] * dc) / 16384.0;
        e = e * inv_len(k);
        dh += (int64_t)floor(e);
    }
    if (p->pers_dir && p->lambda_pers[tp] != 0 && m > 0) {
        const double *ph = p->pers_dir + 3 * (int64_t)m;
        double sdot = (double)d[0] * ph[0];
        sdot = sdot + (double)d[1] * ph[1];
        sdot = sdot + (double)d[2] * ph[2];
        double e = sdot * (double)(-16 * (int64_t)p->lambda_pers[tp]);
        e = e * inv_len(k);
        dh += (int64_t)floor(e);
    }
    return dh;
}

static double motility_real(const orc_params *p, int64_t i, int32_t si, int32_t sj, const int32_t o[3])
{
    int32_t m = si > 0 ? si : sj;
    int tp = type_of(p, m);
    int d[3], k;
    copy_dir(o, d, &k);
    double len = sqrt((double)k), dh = 0.0;
    if (p->chem_field && p->lambda_chem[tp] != 0) {
        const int16_t *c = p->chem_field + i * p->dim;
        double dc = d[0] * (c[0] / 16384.0) + d[1] * (c[1] / 16384.0) + (p->dim == 3 ? d[2] * (c[2] / 16384.0) : 0.0);
        dh -= p->lambda_chem[tp] * dc / len;
    }
    if (p->pers_dir && p->lambda_pers[tp] != 0 && m > 0) {
        const double *ph = p->pers_dir + 3 * (int64_t)m;
        dh -= p->lambda_pers[tp] * (d[0] * ph[0] + d[1] * ph[1] + d[2] * ph[2]) / len;
    }
    return dh;
}

/* Centroids of every cell (Eq. 10) in one periodic image: the cell's first
 * site in raster order plus the mean minimal-image offset from it; NaN for
 * a cell without sites.  X has (n_cells + 1) x 3 entries. */
void orc_centroids(const orc_params *p, const int32_t *lat, double *X)
{
    int64_t nc = p->n_cells + 1, N = (int64_t)p->nx * p->ny * p->nz, plane = (int64_t)p->nx * p->ny;
    int64_t *anchor = (int64_t *)malloc(sizeof(int64_t) * nc);
    int64_t *sums = (int64_t *)calloc((size_t)(4 * nc), sizeof(int64_t));
    int64_t L[3] = {p->nx, p->ny, p->nz};
    for (int64_t c = 0; c < nc; c++) anchor[c] = -1;
    for (int64_t x = 0; x < N; x++) {
        int32_t s = lat[x];
        if (s <= 0) continue;
        if (anchor[s] < 0) anchor[s] = x;
        int64_t a = anchor[s];
        int64_t pc[3] = {x % p->nx, (x / p->nx) % p->ny, x / plane};
        int64_t ac[3] = {a % p->nx, (a / p->nx) % p->ny, a / plane};
        for (int d = 0; d < 3; d++) {
            int64_t o = wrap(pc[d] - ac[d] + L[d] / 2, L[d]) - L[d] / 2;
            sums[4 * s + d] += o;
        }
        sums[4 * s + 3] += 1;
    }
    for (int64_t c = 0; c < nc; c++) {
        if (anchor[c] < 0 || c == 0) {
            X[3 * c] = X[3 * c + 1] = X[3 * c + 2] = NAN;
            continue;
        }
        int64_t a = anchor[c];
        int64_t ac[3] = {a % p->nx, (a / p->nx) % p->ny, a / plane};
        double v = (double)sums[4 * c + 3];
        for (int d = 0; d < 3; d++) X[3 * c + d] = (double)ac[d] + (double)sums[4 * c + d] / v;
    }
    free(anchor);
    free(sums);
}

/* Persistence update (Eq. 6 and Eq. 7) at the end of an MCS, time t: record
 * the centroids; for every cell with a look-back dt whose centroid is known
 * at t and t - dt, u = D / |D| for the minimal-image displacement D,
 * p = (1 - mu) u + mu p_hat, p_hat = p / |p| (each product and sum rounded
 * in this order, no fused operations).  A zero displacement or an unknown
 * centroid leaves p_hat unchanged. */
void orc_pers_update(const orc_params *p, const int32_t *lat, int64_t t)
{
    if (!pers_enabled(p)) return;
    int64_t nc = p->n_cells + 1;
    double *X = p->pers_hist + 3 * nc * (t % p->pers_hist_len);
    orc_centroids(p, lat, X);
    double L[3] = {p->nx, p->ny, p->nz};
    for (int64_t c = 1; c < nc; c++) {
        int tp = p->cell_type[c];
        int dt = p->dt_pers[tp];
        if (p->lambda_pers[tp] == 0 || dt < 1 || t - dt < p->pers_t0) continue;
        const double *Xo = p->pers_hist + 3 * nc * ((t - dt) % p->pers_hist_len) + 3 * c;
        const double *Xn = X + 3 * c;
        if (isnan(Xo[0]) || isnan(Xn[0])) continue;
        double D[3];
        for (int d = 0; d < 3; d++) {
            double v = Xn[d] - Xo[d];
            D[d] = v - L[d] * rint(v / L[d]);
        }
        double n2 = D[0] * D[0];
        n2 = n2 + D[1] * D[1];
        n2 = n2 + D[2] * D[2];
        if (n2 == 0.0) continue;
        double n = sqrt(n2), a = 1.0 - p->mu_pers[tp], mu = p->mu_pers[tp];
        double *ph = p->pers_dir + 3 * c, q[3];
        for (int d = 0; d < 3; d++) {
            double u = D[d] / n;
            double x = a * u, y = mu * ph[d];
            q[d] = x + y;
        }
        double m2 = q[0] * q[0];
        m2 = m2 + q[1] * q[1];
        m2 = m2 + q[2] * q[2];
        if (m2 == 0.0) {
            ph[0] = ph[1] = ph[2] = 0.0;
            continue;
        }
        double m = sqrt(m2);
        for (int d = 0; d < 3; d++) ph[d] = q[d] / m;
    }
}

/* ------------------------------------------------------------------ */
/* Act model (Eq. 8 and Eq. 9).  GM(x) is the geometric mean of Act     */
/* over x and those of its Moore neighbours that belong to the same     */
/* cell; it is 0 for medium sites and whenever one of those Act values  */
/* is 0.  The energy change is (lambda_act/Max_act)(GM(j) - GM(i)), the */
/* parameters taken from sigma_i's type, or sigma_j's when sigma_i is   */
/* the medium: copies out of active regions become more likely.         */
/* ------------------------------------------------------------------ */
static double gm_real(const orc_params *p, const int32_t *lat, const uint8_t *act, int64_t x, int nb,
                      int32_t off[26][3])
{
    int32_t s = lat[x];
    if (s <= 0 || act[x] == 0) return 0.0;
    double sum = log((double)act[x]);
    int cnt = 1;
    for (int n = 0; n < nb; n++) {
        int64_t y = neighbour(p, x, off[n]);
        if (lat[y] != s) continue;
        if (act[y] == 0) return 0.0;
        sum += log((double)act[y]);
        cnt++;
    }
    return exp(sum / cnt);
}

static int act_param_type(const orc_params *p, int32_t si, int32_t sj)
{
    return si > 0 ? type_of(p, si) : type_of(p, sj);
}

/* integer tables of oracle (b) */
#define ORC_LN_N 129
typedef struct {
    int64_t L;          /* THR has L entries; dH_q >= L is rejected */
    uint32_t *thr;
    int32_t ln[ORC_LN_N];
    int32_t expq_n;
    int32_t *expq;
} orc_tables;

/* THR[h] = min(2^32-1, floor(2^32 exp(-h/(16 T)))), h in Q4 energy units;
 * returns L (the first h with THR[h] == 0) or -1 if cap is reached first. */
int64_t orc_thr_table(double T, uint32_t *thr, int64_t cap)
{
    for (int64_t h = 0; h < cap; h++) {
        double v = floor(ldexp(exp(-(double)h / (16.0 * T)), 32));
        if (v <= 0.0) return h;
        thr[h] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
    }
    return -1;
}

/* LN[a] = round(2^16 ln a), a in 1..128 */
void orc_ln_table(int32_t *ln)
{
    ln[0] = 0;
    for (int a = 1; a < ORC_LN_N; a++) ln[a] = (int32_t)llround(ldexp(log((double)a), 16));
}

/* EXPQ[m] = round(2^16 exp(m/1024)), m in 0..(LN[128]>>6) */
int32_t orc_expq_size(void)
{
    int32_t ln[ORC_LN_N];
    orc_ln_table(ln);
    return (ln[ORC_LN_N - 1] >> 6) + 1;
}

void orc_expq_table(int32_t *expq, int32_t n)
{
    for (int m = 0; m < n; m++) expq[m] = (int32_t)llround(ldexp(exp((double)m / 1024.0), 16));
}

static int tables_init(const orc_params *p, orc_tables *tb)
{
    int64_t cap = (int64_t)(16.0 * p->T * 32.0 * 0.6931471805599453) + 64;
    tb->thr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cap);
    if (!tb->thr) return -1;
    tb->L = orc_thr_table(p->T, tb->thr, cap);
    if (tb->L < 0) return -1;
    orc_ln_table(tb->ln);
    tb->expq_n = orc_expq_size();
    tb->expq = (int32_t *)malloc(sizeof(int32_t) * (size_t)tb->expq_n);
    if (!tb->expq) return -1;
    orc_expq_table(tb->expq, tb->expq_n);
    return 0;
}

static void tables_free(orc_tables *tb)
{
    free(tb->thr);
    free(tb->expq);
}

/* integer geometric mean in Q16: EXPQ[(sum LN / count) >> 6] */
static int64_t gm_q(const orc_params *p, const orc_tables *tb, const int32_t *lat, const uint8_t *act,
                    int64_t x, int nb, int32_t off[26][3])
{
    int32_t s = lat[x];
    if (s <= 0 || act[x] == 0) return 0;
    int64_t sum = tb->ln[act[x]];
    int64_t cnt = 1;
    for (int n = 0; n < nb; n++) {
        int64_t y = neighbour(p, x, off[n]);
        if (lat[y] != s) continue;
        if (act[y] == 0) return 0;
        sum += tb->ln[act[y]];
        cnt++;
    }
    return tb->expq[(sum / cnt) >> 6];
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

/* ------------------------------------------------------------------ */
/* Composite variable tracking (Methods, "Composite variable tracking",  */
/* Eq. 10 and Eq. 11).  Beside its size V (the volume tally), each cell  */
/* keeps the integer sums S of its sites' coordinates, so that its       */
/* centroid is S / V.  Under periodic boundaries a site is counted at    */
/* the periodic image nearest a reference point of the cell: at the     */
/* start, the cell's first site in raster order; when a copy adds or     */
/* removes a site, the cell's centroid as the round began (the tallies   */
/* every attempt of a round reads are those of the round's start).  The  */
/* sums are moved by multiples of n V, so that the centroid lies in      */
/* [0, n) on each axis, at the start and after every MCS.                */
/* ------------------------------------------------------------------ */

/* image shift k of coordinate x nearest the point S / V on an axis of
 * extent n: x + k n is within n / 2 of S / V, k = floor((S - x V) / (n V) + 1/2) */
static int64_t image_shift(int64_t x, int64_t S, int64_t V, int64_t n)
{
    return floor_div(2 * (S - x * V) + n * V, 2 * n * V);
}

static void site_coords(const orc_params *p, int64_t x, int64_t c[3])
{
    c[0] = x % p->nx;
    c[1] = (x / p->nx) % p->ny;
    c[2] = x / ((int64_t)p->nx * p->ny);
}

/* centroid of every live cell into [0, n) per axis: S -= floor(S / (n V)) n V */
void orc_track_rewrap(const orc_params *p, const int32_t *V, int64_t *S)
{
    int64_t n[3] = {p->nx, p->ny, p->nz};
    for (int64_t c = 1; c <= p->n_cells; c++) {
        if (V[c] <= 0) continue;
        for (int d = 0; d < p->dim; d++) {
            int64_t nv = n[d] * V[c];
            S[3 * c + d] -= floor_div(S[3 * c + d], nv) * nv;
        }
    }
}

/* sums of the lattice's cells: each site at its image nearest the cell's
 * first site in raster order, then moved into bounds; V is the volume
 * tally of the same lattice */
void orc_track_init(const orc_params *p, const int32_t *lat, const int32_t *V, int64_t *S)
{
    int64_t nc = p->n_cells + 1, N = (int64_t)p->nx * p->ny * p->nz;
    int64_t n[3] = {p->nx, p->ny, p->nz};
    int64_t *anchor = (int64_t *)malloc(sizeof(int64_t) * nc);
    for (int64_t c = 0; c < nc; c++) anchor[c] = -1;
    memset(S, 0, sizeof(int64_t) * 3 * nc);
    for (int64_t x = 0; x < N; x++) {
        int32_t s = lat[x];
        if (s <= 0) continue;
        if (anchor[s] < 0) anchor[s] = x;
        int64_t pc[3], ac[3];
        site_coords(p, x, pc);
        site_coords(p, anchor[s], ac);
        for (int d = 0; d < p->dim; d++) S[3 * s + d] += pc[d] + n[d] * image_shift(pc[d], ac[d], 1, n[d]);
    }
    free(anchor);
    orc_track_rewrap(p, V, S);
}

/* Act energy change in Q4 (1/16 energy units), rounded towards -inf */
static int64_t delta_h_act_q(const orc_params *p, const orc_tables *tb, const int32_t *lat,
                             const uint8_t *act, int64_t i, int64_t j, int32_t si, int32_t sj, int nb,
                             int32_t off[26][3])
{
    int tp = act_param_type(p, si, sj);
    int64_t lam = p->lambda_act[tp], mx = p->max_act[tp];
    if (lam == 0 || mx == 0) return 0;
    int64_t gi = gm_q(p, tb, lat, act, i, nb, off);
    int64_t gj = gm_q(p, tb, lat, act, j, nb, off);
    return floor_div(lam * (gj - gi), mx * 4096);
}

static double delta_h_act_real(const orc_params *p, const int32_t *lat, const uint8_t *act, int64_t i,
                               int64_t j, int32_t si, int32_t sj, int nb, int32_t off[26][3])
{
    int tp = act_param_type(p, si, sj);
    double lam = p->lambda_act[tp], mx = p->max_act[tp];
    if (lam == 0 || mx == 0) return 0.0;
    return lam / mx * (gm_real(p, lat, act, j, nb, off) - gm_real(p, lat, act, i, nb, off));
}

static void decay_act(const orc_params *p, uint8_t *act)
{
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int64_t x = 0; x < N; x++)
        if (act[x] > 0) act[x] -= 1;
}

/* Exposed for tests: the motility terms of the copy from neighbour n_idx of
 * j into j, in Q4 (as the replay applies them) and in real units (as the
 * serial chain does). */
int orc_motility(const orc_params *p, const int32_t *lat, int64_t j, int n_idx, int64_t *dh_q, double *dh_real)
{
    int32_t off[26][3];
    orc_neighbour_offsets(p->dim, off);
    int64_t i = neighbour(p, j, off[n_idx]);
    *dh_q = motility_q(p, i, lat[i], lat[j], off[n_idx]);
    *dh_real = motility_real(p, i, lat[i], lat[j], off[n_idx]);
    return 0;
}

/* Exposed for tests: every energy term of one attempt, target j, source its
 * neighbour number n_idx.  Tallies are read from V and A.  */
int orc_delta_h(const orc_params *p, const int32_t *lat, const uint8_t *act, const int32_t *V,
                const int32_t *A, int64_t j, int n_idx, int64_t *dh_int, int64_t *dh_act_q,
                double *dh_act_real, int64_t *gm_i_q, int64_t *gm_j_q, double *gm_i, double *gm_j)
{
    int32_t off[26][3];
    int nb = orc_neighbour_offsets(p->dim, off);
    int64_t i = neighbour(p, j, off[n_idx]);
    int32_t si = lat[i], sj = lat[j];
    int mi, mj;
    *dh_int = delta_h_int(p, lat, j, si, sj, si > 0 ? V[si] : 0, sj > 0 ? V[sj] : 0,
                          si > 0 ? A[si] : 0, sj > 0 ? A[sj] : 0, nb, off, &mi, &mj);
    *dh_act_q = 0;
    *dh_act_real = 0.0;
    *gm_i_q = *gm_j_q = 0;
    *gm_i = *gm_j = 0.0;
    if (act) {
        orc_tables tb;
        if (tables_init(p, &tb) != 0) return -1;
        *dh_act_q = delta_h_act_q(p, &tb, lat, act, i, j, si, sj, nb, off);
        *gm_i_q = gm_q(p, &tb, lat, act, i, nb, off);
        *gm_j_q = gm_q(p, &tb, lat, act, j, nb, off);
        tables_free(&tb);
        *dh_act_real = delta_h_act_real(p, lat, act, i, j, si, sj, nb, off);
        *gm_i = gm_real(p, lat, act, i, nb, off);
        *gm_j = gm_real(p, lat, act, j, nb, off);
    }
    return 0;
}

/* ================================================================== */
/* (a) the serial CPM                                                  */
/* ================================================================== */
int orc_serial_run(const orc_params *p, int32_t *lat, uint8_t *act, int32_t *V, int32_t *A,
                   int64_t n_mcs, uint64_t rng[4], int64_t *t_io, int64_t *accepts)
{
    int32_t off[26][3];
    int nb = orc_neighbour_offsets(p->dim, off);
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    int use_act = act_enabled(p) && act != NULL;
    int use_mot = motility_enabled(p);
    int64_t acc = 0;
    for (int64_t t = 0; t < n_mcs; t++) {
        if (use_act) decay_act(p, act);
        for (int64_t it = 0; it < N; it++) {
            int64_t j = (int64_t)rand_below(rng, (uint64_t)N);
            int n = (int)rand_below(rng, (uint64_t)nb);
            int64_t i = neighbour(p, j, off[n]);
            int32_t si = lat[i], sj = lat[j];
            if (si == sj || si < 0 || sj < 0) continue;
            if (sj > 0 && V[sj] <= 1) continue; /* a cell never loses its last site */
            int mi, mj;
            double dh = (double)delta_h_int(p, lat, j, si, sj, si > 0 ? V[si] : 0, sj > 0 ? V[sj] : 0,
                                            si > 0 ? A[si] : 0, sj > 0 ? A[sj] : 0, nb, off, &mi, &mj);
            if (use_act) dh += delta_h_act_real(p, lat, act, i, j, si, sj, nb, off);
            if (use_mot) dh += motility_real(p, i, si, sj, off[n]);
            if (!(dh <= 0.0 || rand_unit(rng) < exp(-dh / p->T))) continue;
            lat[j] = si;
            if (si > 0) { V[si] += 1; A[si] += nb - 2 * mi; }
            if (sj > 0) { V[sj] -= 1; A[sj] += 2 * mj - nb; }
            if (use_act) act[j] = si > 0 ? (uint8_t)p->max_act[type_of(p, si)] : 0;
            acc++;
        }
        if (pers_enabled(p)) orc_pers_update(p, lat, (t_io ? *t_io : 0) + t + 1);
    }
    if (t_io) *t_io += n_mcs;
    if (accepts) *accepts = acc;
    return 0;
}

/* ================================================================== */
/* (b) replay of the parallel checkerboard scheme                      */
/* ================================================================== */

static int ipow(int b, int e) { int r = 1; while (e-- > 0) r *= b; return r; }

/* Colour order of cycle pc of MCS t: Fisher-Yates over the c^d colours,
 * swap number i (from C-1 down to 1) drawn from Philox counter
 * (i, pc, t, 1<<24). */
int orc_colour_perm(const orc_params *p, int64_t t, int pc, int32_t *perm)
{
    int C = ipow(p->c, p->dim);
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    for (int q = 0; q < C; q++) perm[q] = q;
    for (int i = C - 1; i >= 1; i--) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)pc, (uint32_t)t, 1u << 24};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        int jj = (int)scale_draw(w[0], (uint32_t)(i + 1));
        int32_t tmp = perm[i]; perm[i] = perm[jj]; perm[jj] = tmp;
    }
    return C;
}

/* Target j, neighbour number n and the acceptance draw of attempt r of block
 * b in sub-pass sp of MCS t: Philox counter (b, r, t, sp) gives four words;
 * word 0 picks j uniformly inside the block, word 1 the neighbour, word 2 is
 * compared with the threshold table. */
static void attempt_draw(const orc_params *p, int64_t b, int r, int64_t t, int32_t sp, int64_t *j_out,
                         int *n_out, uint32_t *w2_out)
{
    int s = p->a / p->c;
    int sd = ipow(s, p->dim);
    int nb = p->dim == 3 ? 26 : 8;
    int64_t nbx = p->nx / s, nby = p->ny / s;
    int64_t bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t ctr[4] = {(uint32_t)b, (uint32_t)r, (uint32_t)t, (uint32_t)sp};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int64_t jl = scale_draw(w[0], (uint32_t)sd);
    int64_t jx = bx * s + jl % s;
    int64_t jy = by * s + (jl / s) % s;
    int64_t jz = p->dim == 3 ? bz * s + jl / ((int64_t)s * s) : 0;
    *j_out = jx + (int64_t)p->nx * (jy + (int64_t)p->ny * jz);
    *n_out = (int)scale_draw(w[1], (uint32_t)nb);
    *w2_out = w[2];
}

/* Active colour of sub-pass sp of MCS t, and the target site of every
 * attempt of that sub-pass in (block, round) order; returns the count. */
int64_t orc_subpass_targets(const orc_params *p, int64_t t, int32_t sp, int64_t *targets)
{
    int s = p->a / p->c;
    int C = ipow(p->c, p->dim);
    int k = ipow(s, p->dim) / p->P;
    int32_t perm[27];
    orc_colour_perm(p, t, sp / C, perm);
    int col = perm[sp % C];
    int64_t nbx = p->nx / s, nby = p->ny / s, nbz = p->nz / (p->dim == 3 ? s : 1);
    int64_t cnt = 0;
    for (int64_t b = 0; b < nbx * nby * nbz; b++) {
        int64_t bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        int colour = (int)(bx % p->c) + p->c * (int)(by % p->c) + p->c * p->c * (int)(bz % p->c);
        if (colour != col) continue;
        for (int r = 0; r < k; r++) {
            int n;
            uint32_t w2;
            attempt_draw(p, b, r, t, sp, &targets[cnt], &n, &w2);
            cnt++;
        }
    }
    return cnt;
}

/* Optional record of the target site of every attempt, in the order the
 * replay makes them (early rejects included); used by the schedule pins. */
typedef struct {
    int64_t *j;
    int64_t n, cap;
} orc_trace;

static void trace_target(orc_trace *tr, int64_t j)
{
    if (tr && tr->n < tr->cap) tr->j[tr->n] = j;
    if (tr) tr->n++;
}

/* Round r of sub-pass sp of MCS t over the listed blocks (all blocks of the
 * active colour when blocks == NULL).  Every attempt of the round reads the
 * tallies as they stood when the round began: the changes of all earlier
 * rounds are seen, those of the same round are not (they are "in flight",
 * Results, "Designing a parallel execution scheme", and the barrier after
 * every attempt of Fig. 3A).  Lattice reads need no snapshot: blocks of one
 * colour are at least two sites apart and a copy only writes inside its
 * block, so no attempt reads a site another attempt of the round writes. */
static int replay_round(const orc_params *p, const orc_tables *tb, int32_t *lat, uint8_t *act,
                        int32_t *V, int32_t *A, int64_t t, int32_t sp, int r, const int64_t *blocks,
                        int64_t n_blocks, int64_t *accepts, orc_trace *tr)
{
    int32_t off[26][3];
    int nb = orc_neighbour_offsets(p->dim, off);
    int use_act = act_enabled(p) && act != NULL;
    int use_mot = motility_enabled(p);
    int s = p->a / p->c;
    int C = ipow(p->c, p->dim);
    int32_t perm[27];
    orc_colour_perm(p, t, sp / C, perm);
    int col = perm[sp % C];
    int64_t nbx = p->nx / s, nby = p->ny / s, nbz = p->nz / (p->dim == 3 ? s : 1);
    int64_t nblk = nbx * nby * nbz;

    size_t nv = (size_t)(p->n_cells + 1);
    int32_t *Vs = (int32_t *)malloc(sizeof(int32_t) * nv);
    int32_t *As = (int32_t *)malloc(sizeof(int32_t) * nv);
    int64_t *Ss = p->csum ? (int64_t *)malloc(sizeof(int64_t) * 3 * nv) : NULL;
    if (!Vs || !As || (p->csum && !Ss)) { free(Vs); free(As); free(Ss); return -1; }
    memcpy(Vs, V, sizeof(int32_t) * nv);
    memcpy(As, A, sizeof(int32_t) * nv);
    if (Ss) memcpy(Ss, p->csum, sizeof(int64_t) * 3 * nv);
    int64_t ext[3] = {p->nx, p->ny, p->nz};

    int64_t acc = 0;
    int64_t count = blocks ? n_blocks : nblk;
    for (int64_t bi = 0; bi < count; bi++) {
        int64_t b = blocks ? blocks[bi] : bi;
        int64_t bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
        int colour = (int)(bx % p->c) + p->c * (int)(by % p->c) + p->c * p->c * (int)(bz % p->c);
        if (colour != col) continue;
        int64_t j;
        int n;
        uint32_t w2;
        attempt_draw(p, b, r, t, sp, &j, &n, &w2);
        trace_target(tr, j);
        int64_t i = neighbour(p, j, off[n]);
        int32_t si = lat[i], sj = lat[j];
        if (si == sj || si < 0 || sj < 0) continue;
        if (sj > 0 && Vs[sj] <= 1) continue; /* a cell never loses its last site */
        int mi, mj;
        int64_t dhq = 16 * delta_h_int(p, lat, j, si, sj, si > 0 ? Vs[si] : 0, sj > 0 ? Vs[sj] : 0,
                                       si > 0 ? As[si] : 0, sj > 0 ? As[sj] : 0, nb, off, &mi, &mj);
        if (use_act) dhq += delta_h_act_q(p, tb, lat, act, i, j, si, sj, nb, off);
        if (use_mot) dhq += motility_q(p, i, si, sj, off[n]);
        int ok = dhq <= 0 || (dhq < tb->L && w2 < tb->thr[dhq]);
        if (!ok) continue;
        lat[j] = si;
        if (si > 0) { V[si] += 1; A[si] += nb - 2 * mi; }
        if (sj > 0) { V[sj] -= 1; A[sj] += 2 * mj - nb; }
        if (use_act) act[j] = si > 0 ? (uint8_t)p->max_act[type_of(p, si)] : 0;
        if (Ss) { /* site j joins sigma_i and leaves sigma_j, each at its image nearest that cell */
            int64_t pc[3];
            site_coords(p, j, pc);
            for (int d = 0; d < p->dim; d++) {
                if (si > 0) p->csum[3 * si + d] += pc[d] + ext[d] * image_shift(pc[d], Ss[3 * si + d], Vs[si], ext[d]);
                if (sj > 0) p->csum[3 * sj + d] -= pc[d] + ext[d] * image_shift(pc[d], Ss[3 * sj + d], Vs[sj], ext[d]);
            }
        }
        acc++;
    }
    free(Vs);
    free(As);
    free(Ss);
    if (accepts) *accepts += acc;
    return 0;
}

/* all k = s^d / P rounds of one sub-pass */
static int replay_subpass(const orc_params *p, const orc_tables *tb, int32_t *lat, uint8_t *act,
                          int32_t *V, int32_t *A, int64_t t, int32_t sp, int64_t *accepts, orc_trace *tr)
{
    int k = ipow(p->a / p->c, p->dim) / p->P;
    for (int r = 0; r < k; r++)
        if (replay_round(p, tb, lat, act, V, A, t, sp, r, NULL, 0, accepts, tr) != 0) return -1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Tiled schedule.  Tiles of edge T (a multiple of a) on a grid shifted  */
/* per MCS by a Philox offset (a multiple of a per axis, counter         */
/* (0, 0, t, 2<<24), words 0..2 for x, y, z); tile colour = parity of    */
/* its tile coordinates.  Per MCS, P_T tile cycles visit the 2^d tile    */
/* colours in a Philox order (swap i from counter (i, cycle, t, 3<<24)). */
/* In an epoch the tiles of one colour are active; each runs, in order,  */
/* its 1/P_T share of the MCS's sub-passes (all rounds of each) on the   */
/* blocks inside it, while the tiles around it are dormant.  Tallies     */
/* read by a tile are those at the epoch start plus the tile's own       */
/* changes of earlier rounds.                                            */
/* ------------------------------------------------------------------ */
static void tile_offset(const orc_params *p, int64_t t, int64_t off[3])
{
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    uint32_t ctr[4] = {0u, 0u, (uint32_t)t, 2u << 24};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    int units = p->tile / p->a;
    off[0] = (int64_t)p->a * scale_draw(w[0], (uint32_t)units);
    off[1] = (int64_t)p->a * scale_draw(w[1], (uint32_t)units);
    off[2] = p->dim == 3 ? (int64_t)p->a * scale_draw(w[2], (uint32_t)units) : 0;
}

int orc_tile_colour_perm(const orc_params *p, int64_t t, int cycle, int32_t *perm)
{
    int C = p->dim == 3 ? 8 : 4;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    for (int q = 0; q < C; q++) perm[q] = q;
    for (int i = C - 1; i >= 1; i--) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)cycle, (uint32_t)t, 3u << 24};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        int jj = (int)scale_draw(w[0], (uint32_t)(i + 1));
        int32_t tmp = perm[i]; perm[i] = perm[jj]; perm[jj] = tmp;
    }
    return C;
}

/* tile coordinate of block coordinate bc along an axis (block edge s) */
static int64_t tile_of(int64_t bc, int s, int64_t off, int64_t n, int T)
{
    int64_t x = bc * s;               /* first site of the block */
    int64_t u = wrap(x - off, n);     /* shifted coordinate */
    return u / T;
}

typedef struct {
    int32_t si, sj, dAi, dAj;
} orc_change;

/* One epoch (tile cycle pc_t, tile colour number qt) of MCS t. */
static int replay_epoch(const orc_params *p, const orc_tables *tb, int32_t *lat, uint8_t *act, int32_t *V,
                        int32_t *A, int64_t t, int pc_t, int qt, int64_t *accepts, orc_trace *tr)
{
    int32_t off[26][3];
    int nb = orc_neighbour_offsets(p->dim, off);
    int use_act = act_enabled(p) && act != NULL;
    int s = p->a / p->c;
    int C = ipow(p->c, p->dim);
    int k = ipow(s, p->dim) / p->P;
    int T = p->tile;
    int64_t toff[3];
    tile_offset(p, t, toff);
    int32_t tperm[8];
    orc_tile_colour_perm(p, t, pc_t, tperm);
    int tcol = tperm[qt];
    int sub_per_epoch = p->P * C / p->tile_cycles;
    int sp0 = pc_t * sub_per_epoch;
    int64_t nbx = p->nx / s, nby = p->ny / s, nbz = p->nz / (p->dim == 3 ? s : 1);
    int64_t ntx = p->nx / T, nty = p->ny / T, ntz = p->dim == 3 ? p->nz / T : 1;
    int64_t bpt = T / s; /* blocks per tile per axis */

    size_t nv = (size_t)(p->n_cells + 1);
    int32_t *Vs = (int32_t *)malloc(sizeof(int32_t) * nv);
    int32_t *As = (int32_t *)malloc(sizeof(int32_t) * nv);
    int32_t *dV = (int32_t *)calloc(nv, sizeof(int32_t));
    int32_t *dA = (int32_t *)calloc(nv, sizeof(int32_t));
    int64_t max_round = 1;
    for (int d = 0; d < p->dim; d++) max_round *= bpt;
    orc_change *chg = (orc_change *)malloc(sizeof(orc_change) * (size_t)max_round);
    int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * max_round * k * sub_per_epoch + 1));
    if (!Vs || !As || !dV || !dA || !chg || !touched) {
        free(Vs); free(As); free(dV); free(dA); free(chg); free(touched);
        return -1;
    }
    memcpy(Vs, V, sizeof(int32_t) * nv);
    memcpy(As, A, sizeof(int32_t) * nv);
    int64_t acc = 0;
    for (int64_t tz = 0; tz < ntz; tz++)
        for (int64_t ty = 0; ty < nty; ty++)
            for (int64_t tx = 0; tx < ntx; tx++) {
                int colour = (int)(tx % 2) + 2 * (int)(ty % 2) + 4 * (int)(tz % 2);
                if (colour != tcol) continue;
                int64_t ntouched = 0;
                for (int sp = sp0; sp < sp0 + sub_per_epoch; sp++) {
                    int32_t perm[27];
                    orc_colour_perm(p, t, sp / C, perm);
                    int col = perm[sp % C];
                    for (int r = 0; r < k; r++) {
                        int64_t nchg = 0;
                        /* blocks of this tile, in tile-local order */
                        for (int64_t lz = 0; lz < (p->dim == 3 ? bpt : 1); lz++)
                            for (int64_t ly = 0; ly < bpt; ly++)
                                for (int64_t lx = 0; lx < bpt; lx++) {
                                    int64_t bx = wrap(toff[0] / s + tx * bpt + lx, nbx);
                                    int64_t by = wrap(toff[1] / s + ty * bpt + ly, nby);
                                    int64_t bz = p->dim == 3 ? wrap(toff[2] / s + tz * bpt + lz, nbz) : 0;
                                    int bcol = (int)(bx % p->c) + p->c * (int)(by % p->c) +
                                               p->c * p->c * (int)(bz % p->c);
                                    if (bcol != col) continue;
                                    (void)tile_of;
                                    int64_t b = bx + nbx * (by + nby * bz);
                                    int64_t j;
                                    int n;
                                    uint32_t w2;
                                    attempt_draw(p, b, r, t, sp, &j, &n, &w2);
                                    trace_target(tr, j);
                                    int64_t i = neighbour(p, j, off[n]);
                                    int32_t si = lat[i], sj = lat[j];
                                    if (si == sj || si < 0 || sj < 0) continue;
                                    int64_t Vi = si > 0 ? (int64_t)Vs[si] + dV[si] : 0;
                                    int64_t Vj = sj > 0 ? (int64_t)Vs[sj] + dV[sj] : 0;
                                    int64_t Ai = si > 0 ? (int64_t)As[si] + dA[si] : 0;
                                    int64_t Aj = sj > 0 ? (int64_t)As[sj] + dA[sj] : 0;
                                    if (sj > 0 && Vj <= 1) continue;
                                    int mi, mj;
                                    int64_t dhq = 16 * delta_h_int(p, lat, j, si, sj, Vi, Vj, Ai, Aj, nb, off, &mi, &mj);
                                    if (use_act) dhq += delta_h_act_q(p, tb, lat, act, i, j, si, sj, nb, off);
                                    int ok = dhq <= 0 || (dhq < tb->L && w2 < tb->thr[dhq]);
                                    if (!ok) continue;
                                    lat[j] = si;
                                    if (use_act) act[j] = si > 0 ? (uint8_t)p->max_act[type_of(p, si)] : 0;
                                    chg[nchg].si = si;
                                    chg[nchg].sj = sj;
                                    chg[nchg].dAi = nb - 2 * mi;
                                    chg[nchg].dAj = 2 * mj - nb;
                                    nchg++;
                                    acc++;
                                }
                        /* the round's changes become visible to the tile's next round */
                        for (int64_t e = 0; e < nchg; e++) {
                            if (chg[e].si > 0) {
                                dV[chg[e].si] += 1; dA[chg[e].si] += chg[e].dAi;
                                touched[ntouched++] = chg[e].si;
                            }
                            if (chg[e].sj > 0) {
                                dV[chg[e].sj] -= 1; dA[chg[e].sj] += chg[e].dAj;
                                touched[ntouched++] = chg[e].sj;
                            }
                        }
                    }
                }
                /* the tile's changes go into the global tallies; reset its deltas */
                for (int64_t e = 0; e < ntouched; e++) {
                    int32_t c = touched[e];
                    V[c] += dV[c]; A[c] += dA[c];
                    dV[c] = 0; dA[c] = 0;
                }
            }
    free(Vs); free(As); free(dV); free(dA); free(chg); free(touched);
    if (accepts) *accepts += acc;
    return 0;
}

static int check_params(const orc_params *p)
{
    if (p->dim != 2 && p->dim != 3) return -1;
    if (p->dim == 2 && p->nz != 1) return -1;
    if (p->c < 1 || p->a % p->c != 0) return -1;
    if (p->nx % p->a || p->ny % p->a || (p->dim == 3 && p->nz % p->a)) return -1;
    int s = p->a / p->c;
    if (p->a - s < 2) return -1;
    if (ipow(s, p->dim) % p->P) return -1;
    if (p->tile) {
        int T = p->tile;
        if (T % p->a || p->nx % (2 * T) || p->ny % (2 * T) || (p->dim == 3 && p->nz % (2 * T))) return -1;
        if (p->tile_cycles < 1 || p->P % p->tile_cycles) return -1;
        if (motility_enabled(p)) return -1; /* the tiled schedule has no motility terms */
        if (p->csum) return -1;             /* nor composite variable tracking */
    }
    if (pers_enabled(p)) {
        for (int t = 0; t < ORC_MAXT; t++)
            if (p->lambda_pers[t] != 0 && (p->dt_pers[t] < 1 || p->dt_pers[t] >= p->pers_hist_len)) return -1;
    }
    return 0;
}

/* Advance by n_sub schedule units (sub-passes of the global schedule,
 * epochs of the tiled one) from position (t, sp); Act decays at the start
 * of every MCS (sp == 0).  Position is updated in place. */
static int replay_units(const orc_params *p, int32_t *lat, uint8_t *act, int32_t *V, int32_t *A,
                        int64_t *t_io, int32_t *sp_io, int64_t n_sub, int64_t *accepts, orc_trace *tr)
{
    if (check_params(p)) return -2;
    orc_tables tb;
    if (tables_init(p, &tb) != 0) return -1;
    int use_act = act_enabled(p) && act != NULL;
    int CT = p->dim == 3 ? 8 : 4;
    int per_mcs = p->tile ? p->tile_cycles * CT : p->P * ipow(p->c, p->dim);
    int64_t t = *t_io;
    int32_t sp = *sp_io;
    if (accepts) *accepts = 0;
    for (int64_t it = 0; it < n_sub; it++) {
        if (sp == 0 && use_act) decay_act(p, act);
        int rc = p->tile ? replay_epoch(p, &tb, lat, act, V, A, t, sp / CT, sp % CT, accepts, tr)
                         : replay_subpass(p, &tb, lat, act, V, A, t, sp, accepts, tr);
        if (rc != 0) {
            tables_free(&tb);
            return -1;
        }
        if (++sp == per_mcs) {
            sp = 0;
            t++;
            if (p->csum) orc_track_rewrap(p, V, p->csum);
            if (pers_enabled(p)) orc_pers_update(p, lat, t);
        }
    }
    *t_io = t;
    *sp_io = sp;
    tables_free(&tb);
    return 0;
}

int orc_replay_run(const orc_params *p, int32_t *lat, uint8_t *act, int32_t *V, int32_t *A,
                   int64_t *t_io, int32_t *sp_io, int64_t n_sub, int64_t *accepts)
{
    return replay_units(p, lat, act, V, A, t_io, sp_io, n_sub, accepts, NULL);
}

/* As orc_replay_run, also writing the target site of every attempt, in
 * replay order, to targets[0 .. cap-1]; *n_targets receives the number of
 * attempts made (which may exceed cap). */
int orc_replay_trace(const orc_params *p, int32_t *lat, uint8_t *act, int32_t *V, int32_t *A,
                     int64_t *t_io, int32_t *sp_io, int64_t n_sub, int64_t *accepts, int64_t *targets,
                     int64_t cap, int64_t *n_targets)
{
    orc_trace tr = {targets, 0, cap};
    int rc = replay_units(p, lat, act, V, A, t_io, sp_io, n_sub, accepts, &tr);
    *n_targets = tr.n;
    return rc;
}

/* Offset of the tile grid in MCS t (tiled schedule), per axis. */
void orc_tile_offset_of(const orc_params *p, int64_t t, int64_t off[3]) { tile_offset(p, t, off); }

/* Round r of sub-pass sp of MCS t restricted to the given block indices
 * (others untouched); tallies are read from V and A as given; no Act decay
 * is applied here.  Used for sampled checks at full size. */
int orc_replay_round(const orc_params *p, int32_t *lat, uint8_t *act, int32_t *V, int32_t *A,
                     int64_t t, int32_t sp, int32_t r, const int64_t *blocks, int64_t n_blocks,
                     int64_t *accepts)
{
    if (check_params(p)) return -2;
    orc_tables tb;
    if (tables_init(p, &tb) != 0) return -1;
    if (accepts) *accepts = 0;
    int rc = replay_round(p, &tb, lat, act, V, A, t, sp, r, blocks, n_blocks, accepts, NULL);
    tables_free(&tb);
    return rc;
}
