/*
 * cpm.h -- C ABI of the GB300 cellular Potts model (CPM) sweep library
 * (libcpm_gb300.so).
 *
 * The library runs the parallel Metropolis copy-attempt sweep of the CPM
 * (Sultan, Devi, Mueller, Textor, "A parallelized cellular Potts model that
 * enables simulations at tissue scale", arXiv 2312.09317) on one GPU:
 *
 *   Hamiltonian     Methods, Eq. 1 (adhesion J over Moore-neighbour pairs,
 *                   each unordered pair counted once; volume term) and Eq. 3
 *                   (perimeter term, A = interfaces with other ids);
 *   acceptance      Methods, Eq. 2: min(1, exp(-dH/T));
 *   Act motility    Methods, Eq. 8 and Eq. 9 (geometric mean of Act over the
 *                   site and its same-cell Moore neighbours; Act set to
 *                   Max_act on update, decays by 1 per MCS);
 *   parallel scheme Results, "Designing a parallel execution scheme" and
 *                   "Aligning the lattice update statistics" (Fig. 2A/B,
 *                   Fig. 3A/B): a checkerboard of blocks, atomic tally
 *                   updates, a barrier after every copy attempt.
 *
 * Semantics fixed by this library (the paper leaves them open):
 *   - The lattice is split into areas of edge a; each area into c^d blocks
 *     of edge s = a/c; block (bx,by,bz) has colour (bx%c) + c(by%c) +
 *     c^2(bz%c).  One MCS is P cycles; each cycle visits the c^d colours in
 *     an order drawn from Philox; a visit (a "sub-pass") runs k = s^d/P
 *     rounds; in a round every block of the active colour makes one copy
 *     attempt into a target site of its own block from a uniformly chosen
 *     Moore neighbour.  So each MCS makes exactly one attempt per site.
 *   - All attempts of a round read the tallies (volume V, interface count A
 *     per cell) as they stood when the round began; the round's own changes
 *     become visible in the next round.  Blocks of one colour are >= 2 sites
 *     apart (a - s >= 2), so their lattice reads and writes never overlap.
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = seed,
 *     counter = (block index, round, MCS, sub-pass) for attempts (word 0
 *     picks the target in the block, word 1 the neighbour, word 2 is the
 *     acceptance draw) and (i, cycle, MCS, 1<<24) for the colour shuffle.
 *   - Energies are integers (the caller scales J and the lambdas by an
 *     integer S and passes T scaled by S); the Act term is added in Q4 fixed
 *     point through integer tables; acceptance compares the uint32 draw with
 *     THR[dH] = min(2^32-1, floor(2^32 exp(-dH/(16T)))).
 *   - A copy that would remove a cell's last site is rejected.
 *   - Tiled schedule (tile = T > 0): the same sub-passes, rounds and Philox
 *     counters, executed tile by tile.  Tiles of edge T (a multiple of a;
 *     every extent a multiple of 2T) sit on a grid shifted per MCS by a
 *     Philox offset (counter (0, 0, MCS, 2<<24), words 0..2 -> a multiple
 *     of a below T per axis); a tile's colour is the parity of its tile
 *     coordinates.  Per MCS, P_T tile cycles visit the 2^d tile colours in
 *     a Philox order (swap i from counter (i, cycle, MCS, 3<<24)); in such
 *     an epoch every tile of the colour runs, on its own blocks, the
 *     epoch's P*c^d/P_T sub-passes with all their rounds, while the tiles
 *     around it are dormant.  Tallies read by a tile are those at the start
 *     of the epoch plus the tile's own changes of earlier rounds.  A tile
 *     and its 2-site halo may hold at most 510 distinct cells; beyond that
 *     the epoch is invalid and the next reading call returns CPM_E_STATE.
 *   The result is a deterministic function of (config, seed, number of
 *   sub-passes run): cpm_step(h, a) then cpm_step(h, b) equals
 *   cpm_step(h, a + b), on any GPU.
 *
 * Data conventions: lattice int32, x fastest (idx = x + nx*(y + ny*z));
 * id 0 = medium (type 0, no tallies), ids 1..n_cells = cells, id -1 = frozen
 * obstacle of type obstacle_type.  Boundaries are periodic.
 *
 * Ownership: the library allocates and owns every device buffer of a
 * handle; pointers passed in are borrowed for the duration of the call.
 * Host pointers must be readable/writable for the stated sizes; device
 * pointers must be device memory of the handle's GPU.
 *
 * Errors: every int-returning call returns CPM_OK (0) or a negative
 * CPM_E_* code and records a message readable with cpm_last_error.  No call
 * aborts the process.  After CPM_E_CUDA the handle should be destroyed.
 *
 * Streams: all work of a handle is issued on the stream given to
 * cpm_create (0 = the legacy default stream).  Calls that return data to the
 * host synchronise that stream.
 */
#ifndef CPM_GB300_H
#define CPM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPM_MAX_TYPES 8

enum {
    CPM_OK = 0,
    CPM_E_INVALID = -1,   /* bad argument or configuration */
    CPM_E_NOMEM = -2,     /* device or host allocation failed */
    CPM_E_CUDA = -3,      /* a CUDA runtime call failed */
    CPM_E_HANDLE = -4,    /* NULL or destroyed handle */
    CPM_E_STATE = -5,     /* device-side consistency check failed */
    CPM_E_LIMIT = -6      /* a size exceeds the fixed scratch of cpm_step_noalloc */
};

typedef struct cpm_config {
    int32_t dim;                 /* 2 or 3 */
    int32_t nx, ny, nz;          /* extents; nz = 1 when dim = 2; multiples of a */
    int32_t J[CPM_MAX_TYPES][CPM_MAX_TYPES];   /* adhesion, symmetric, scaled */
    int32_t lambda_v[CPM_MAX_TYPES];           /* volume weight per type, scaled */
    int32_t v_target[CPM_MAX_TYPES];
    int32_t lambda_p[CPM_MAX_TYPES];           /* perimeter weight, scaled */
    int32_t a_target[CPM_MAX_TYPES];
    int32_t lambda_act[CPM_MAX_TYPES];         /* Act weight, scaled (all 0: Act off) */
    int32_t max_act[CPM_MAX_TYPES];            /* Max_act, 0..127 */
    double temperature;          /* T in the same scaled energy units, > 0 */
    int32_t obstacle_type;       /* type of id -1 sites, 1..CPM_MAX_TYPES-1 */
    int32_t a, c, P;             /* area edge, divisions per axis, cycles per MCS */
    uint64_t seed;
    int32_t n_cells;             /* cells have ids 1..n_cells; n_cells <= 2^23 - 1 */
    const uint8_t *cell_type;    /* host, n_cells + 1 entries; [0] must be 0 */
    const int32_t *init_lattice; /* host, nx*ny*nz ids in -1..n_cells */
    const uint8_t *init_act;     /* host, nx*ny*nz Act values or NULL (all 0) */
    int64_t t0;                  /* MCS index of the first MCS to run (>= 0) */
    int32_t tile;                /* 0: global rounds; T > 0: tiled schedule with tiles of edge T */
    int32_t tile_cycles;         /* tiled schedule: tile cycles per MCS (P_T, divides P) */
    /* Motility terms (Methods Eq. 4 to Eq. 7), global schedule only; all zero /
     * NULL = off.  A copy from source i into target j moves the cell sigma_i
     * (sigma_j when sigma_i is the medium) along d = j - i and adds
     * floor(-16 lambda (d . v) / |d|) in 1/16 energy units, v being the field
     * at i (chemotaxis) or the moving cell's persistence direction p_hat;
     * copies along v become more likely. */
    const int16_t *chem_field;   /* host, nx*ny*nz*dim int16: the field C per site (components innermost)
                                    in Q14 (16384 = 1), or NULL */
    int32_t lambda_chem[CPM_MAX_TYPES];        /* chemotaxis weight per type, scaled */
    int32_t lambda_pers[CPM_MAX_TYPES];        /* persistence weight per type, scaled */
    double mu_pers[CPM_MAX_TYPES];             /* persistence memory mu in [0, 1] (Eq. 6) */
    int32_t dt_pers[CPM_MAX_TYPES];            /* look-back in MCS, 1..255 where lambda_pers != 0 */
} cpm_config;

typedef struct cpm_stats_t {
    int64_t mcs;            /* MCS index of the next unit (completed MCS if subpass == 0) */
    int32_t subpass;        /* next schedule unit (sub-pass or epoch) within that MCS */
    int32_t n_live_cells;   /* cells with V > 0 */
    int64_t attempts;       /* copy attempts made by this handle */
    int64_t accepts;        /* accepted copies made by this handle */
    double volume_mean, volume_var;        /* over live cells */
    double perimeter_mean, perimeter_var;  /* over live cells */
} cpm_stats_t;

typedef struct cpm_handle cpm_handle;

/* Validate cfg, allocate device state, upload the initial lattice, compute
 * the tallies and the threshold/log/exp tables.  cuda_stream is a
 * cudaStream_t (or NULL).  On success *out receives a handle.
 * Errors: CPM_E_INVALID (message says which field), CPM_E_NOMEM, CPM_E_CUDA. */
int cpm_create(const cpm_config *cfg, void *cuda_stream, cpm_handle **out);

/* Run n_mcs Monte Carlo steps (n_mcs * P * c^d sub-passes).  Asynchronous on
 * the handle's stream.  n_mcs >= 0. */
int cpm_step(cpm_handle *h, int64_t n_mcs);

/* Run n schedule units: sub-passes (colour visits) of the global schedule,
 * epochs of the tiled one; cpm_step(h, m) = cpm_step_subpasses(h, m * P * c^d)
 * (global) or (h, m * P_T * 2^d) (tiled).  Used for finer-grained checks. */
int cpm_step_subpasses(cpm_handle *h, int64_t n);

/* Copy the lattice (nx*ny*nz int32) to dst (host if dst_is_device == 0,
 * device otherwise).  Synchronises the handle's stream. */
int cpm_read_lattice(cpm_handle *h, int32_t *dst, int dst_is_device);

/* Copy the tallies: V and A, n_cells + 1 int32 each (entry 0 unused, 0).
 * Either pointer may be NULL.  Synchronises the stream. */
int cpm_read_tallies(cpm_handle *h, int32_t *V, int32_t *A, int dst_is_device);

/* Copy the Act values (nx*ny*nz uint8) as seen after the last completed
 * sub-pass (all 0 when Act is off).  Synchronises the stream. */
int cpm_read_act(cpm_handle *h, uint8_t *dst, int dst_is_device);

/* Replace the lattice with src (host or device, nx*ny*nz int32 in
 * -1..n_cells; obstacle sites must stay where they are) and recompute the
 * tallies on the device.  Act values and the position are kept. */
int cpm_load_lattice(cpm_handle *h, const int32_t *src, int src_is_device);

/* Copy the persistence directions p_hat, (n_cells + 1) x 3 doubles (x, y,
 * z; zeros before the first update, for absent cells and without the
 * persistence term) to a host array.  p_hat is updated at the end of every
 * MCS (Eq. 6, Eq. 7) from the cell centroids (Eq. 10) dt_pers MCS apart:
 * u = D / |D| for the minimal-image displacement D, p = (1 - mu) u +
 * mu p_hat, p_hat = p / |p|, every product, sum, quotient and root rounded
 * once in that order; a zero displacement or an absent cell leaves p_hat.
 * Synchronises the stream. */
int cpm_read_persistence(cpm_handle *h, double *dir);

/* Composite variable tracking (Methods, "Composite variable tracking",
 * Eq. 10 and Eq. 11): beside each cell's size V (the volume tally), the
 * integer sums S of its sites' coordinates, so that its centroid is S / V,
 * kept up to date by the sweep itself on every accepted copy.  Under
 * periodic boundaries each site counts at its periodic image nearest a
 * reference point of its cell: when tracking starts (and after
 * cpm_load_lattice), the cell's first site in raster order; when a copy adds
 * or removes a site, the cell's centroid as the round began (the tallies
 * every attempt of a round reads).  At the start and after every MCS each
 * live cell's sums are moved by a multiple of n x V so that its centroid lies
 * in [0, n) on each axis (the paper's re-wrap); between MCS ends a centroid
 * may leave [0, n) by the distance its cell moved.  Sums are int64 (the
 * paper's are 32-bit, interleaved with the size for a 64-bit
 * compare-and-swap; here size and sums are round-synchronous tallies that the
 * round boundary keeps consistent).  The image shift of a copy must be within
 * +-3 lattice lengths, which holds for any cell smaller than half the lattice.
 *
 * on = 1 allocates 48 (n_cells + 1) + 16 n_active bytes on the device,
 * recomputes the tallies from the lattice (pending changes of the last round
 * are folded in) and starts the sums; on = 0 frees them.  Tracking changes
 * no lattice update.  Global schedule only: CPM_E_INVALID on a tiled handle. */
int cpm_track_centroids(cpm_handle *h, int32_t on);

/* Copy the tracked sums, (n_cells + 1) x 3 int64 (x, y, z; z is 0 in 2D;
 * row 0, the medium, is 0) as of the last completed round, to host or device
 * memory.  Centroid of cell c: S[c] / V[c] with V from cpm_read_tallies.
 * CPM_E_INVALID when tracking is off.  Synchronises the stream. */
int cpm_read_centroid_sums(cpm_handle *h, int64_t *S, int dst_is_device);

/* Counters and moments of the tallies.  Synchronises the stream. */
int cpm_stats(cpm_handle *h, cpm_stats_t *out);

/* Recount V and A from the lattice on the device and compare with the
 * tallies; *n_mismatch receives the number of cells that differ (0 when the
 * bookkeeping is exact).  Synchronises the stream. */
int cpm_verify(cpm_handle *h, int64_t *n_mismatch);

/* Number of kernel launches the library has issued for this handle. */
int64_t cpm_kernel_launches(const cpm_handle *h);

/* Message of the last failed call on h (or, when h is NULL, of the calling
 * thread's last failed cpm_create).  The string stays valid until the next
 * call on h (with NULL: the thread's next cpm_create). */
const char *cpm_last_error(const cpm_handle *h);

/* Free every resource of h (NULL is ignored).  Synchronises the stream. */
void cpm_destroy(cpm_handle *h);

/* Batched ensembles (many independent lattices, e.g. replicates or a
 * parameter sweep, advanced together; the paper runs ensembles as
 * independent simulations, Results, "Serial Cellular Potts Models are
 * limited", Fig. 1B).  Every lattice of a batch is a full simulation with its
 * own configuration and seed; after cpm_batch_step(b, n) lattice i is
 * exactly what cpm_step(h_i, n) gives for a handle created from cfgs[i].  A
 * batch step launches one kernel per round for all lattices that still have
 * rounds in the call (lattices with fewer rounds per MCS finish earlier).
 * All configurations of a batch must share dim and use the global schedule
 * (tile = 0).  The library owns all device memory; cfgs is borrowed for the
 * duration of cpm_batch_create. */
typedef struct cpm_batch cpm_batch;

/* Create n lattices from cfgs[0..n-1] on cuda_stream.  Errors as cpm_create
 * (the message names the offending configuration). */
int cpm_batch_create(const cpm_config *cfgs, int32_t n, void *cuda_stream, cpm_batch **out);

/* Advance every lattice by n_mcs MCS (asynchronous on the batch's stream).
 * One MCS of the whole batch is a CUDA graph, captured on first use: the Act
 * stamp clamp, one launch per round over the members that still have
 * rounds, and a device-side advance of every member's MCS counter. */
int cpm_batch_step(cpm_batch *b, int64_t n_mcs);

/* Choose how cpm_batch_step runs the MCS loop.
 *   on = 0 (the default): one CUDA graph per MCS, replayed: the Act clamp,
 *          one kernel per round, and the advance of the members' counters.
 *   on = 1: one persistent, cooperative launch per call runs all n_mcs MCS:
 *          the same phases, separated by grid-wide barriers instead of
 *          kernel boundaries (every CTA of the launch is resident; the grid
 *          is at most what the device holds at once).  Same results bit for
 *          bit.  cpm_batch_step then waits for its launch to finish.
 * Every barrier wait is bounded: after max_polls polls (about 100 ns apart;
 * max_polls < 0 selects the default, 2^24) the waiting CTA records a timeout
 * and ends, and cpm_batch_step returns CPM_E_STATE ("grid-barrier wait ...
 * timed out"); the lattices are then in an unspecified state and the batch
 * should be destroyed.  A healthy launch never times out.
 *   on = 2: a test of that path: as on = 1, but the launch's first CTA leaves
 *          before its first barrier, so the other CTAs' waits run out (use a
 *          small max_polls); the step returns CPM_E_STATE.
 * Errors: CPM_E_HANDLE, CPM_E_INVALID (on not 0..2, or on != 0 while the
 * batch tracks centroids), CPM_E_CUDA. */
int cpm_batch_set_persistent(cpm_batch *b, int32_t on, int64_t max_polls);

/* Composite variable tracking (as cpm_track_centroids) in every lattice of
 * the batch: on = 1 starts it (tallies recomputed from each lattice, pending
 * changes folded in), on = 0 stops it.  The batch graph then runs the
 * tracking variant of the round kernel and, after each MCS, moves every
 * member's centroids into [0, n).  Graph loop only: CPM_E_INVALID while the
 * persistent loop is on.  cpm_batch_read_centroid_sums copies lattice idx's
 * sums as cpm_read_centroid_sums does (CPM_E_INVALID when tracking is off or
 * idx is out of range). */
int cpm_batch_track_centroids(cpm_batch *b, int32_t on);
int cpm_batch_read_centroid_sums(cpm_batch *b, int32_t idx, int64_t *S, int dst_is_device);

/* Pick the CTA brick shape (active blocks per CTA along x, y, z) for this
 * batch by timing: in 1 + n_mcs_each passes every candidate shape runs one
 * MCS of the batch itself (the first pass only warms up) and the shape
 * with the least total time is kept.  The shape changes only how the work
 * is split over CTAs, never the result, so the batch simply advances by
 * candidates * (1 + n_mcs_each) MCS (7 candidates in 3D, 6 in 2D).
 * *choice (if not NULL) receives the chosen candidate's number. */
int cpm_batch_autotune(cpm_batch *b, int32_t n_mcs_each, int32_t *choice);

/* Number of lattices in b (0 for NULL). */
int32_t cpm_batch_size(const cpm_batch *b);

/* Per-lattice access, as cpm_read_lattice, cpm_load_lattice, cpm_read_tallies,
 * cpm_read_act and cpm_stats for lattice idx (0 <= idx < n). */
int cpm_batch_read_lattice(cpm_batch *b, int32_t idx, int32_t *dst, int dst_is_device);
int cpm_batch_load_lattice(cpm_batch *b, int32_t idx, const int32_t *src, int src_is_device);
int cpm_batch_read_tallies(cpm_batch *b, int32_t idx, int32_t *V, int32_t *A, int dst_is_device);
int cpm_batch_read_act(cpm_batch *b, int32_t idx, uint8_t *dst, int dst_is_device);
int cpm_batch_stats(cpm_batch *b, int32_t idx, cpm_stats_t *out);

/* Observations of every lattice of b in its current state, for summary
 * statistics (asynchronous on the batch's stream; call between steps).
 * cells_out: DEVICE int64 array of rows of 12, one row per cell id 0..n_cells
 * of each lattice, lattice k's rows starting at sum_{j<k} (n_cells_j + 1);
 * row 0 of a lattice (the medium) is unused.  Per cell:
 *   [0] anchor: linear index z*ny*nx + y*nx + x of the cell's first site in
 *       raster order, -1 when the cell has no site;
 *   [1] volume (sites);
 *   [2..4] sums over the cell's sites of the minimal-image offsets
 *       ((p - anchor + n/2) mod n) - n/2 from the anchor along x, y, z, so the
 *       centroid (Methods, "Composite variable tracking", Eq. 10) is
 *       anchor + sums / volume, modulo the lattice, for any cell shorter than
 *       half the lattice along each axis;
 *   [5] interface count: neighbour pairs with a different id (Eq. 3);
 *   [6..11] sums of the offset products xx, yy, zz, xy, xz, yz (the cell's
 *       second moments about the anchor; z terms are 0 in 2D).
 * member_out: DEVICE int64 [n][2]: unordered (cell, medium) neighbour pairs
 * over the model's neighbourhood, and accepted copies since creation.
 * Three kernel launches; the first call uploads one descriptor per lattice. */
int cpm_batch_observe(cpm_batch *b, int64_t *cells_out, int64_t *member_out);

/* Summary statistics of every lattice of a 2D batch from n_snap
 * observations taken every `every` MCS (cpm_batch_observe outputs stacked
 * on the device: cells_hist [n_snap][rows][12], member_hist [n_snap][n][2]).
 * out: DEVICE double [n][16], NaN where a statistic is undefined:
 *   0 mean cell volume / V_t, 1 std of the volume over cells / V_t (root
 *   of the per-snapshot variance averaged over snapshots), 2 mean interface
 *   count / A_t, 3 its std / A_t (V_t, A_t of cell 1's type);
 *   4..6 mean squared centroid displacement over 10, 50 and 200 MCS;
 *   7, 8 mean and std of the centroid speed over `every`-MCS steps;
 *   9 mean cosine between successive 50-MCS displacements;
 *   10 persistence time: every * (1/2 + sum of the step-direction
 *      autocorrelation over lags 1..20 up to its first value <= 0);
 *   11 arrest coefficient: share of 50-MCS sub-tracks slower than 0.05
 *      sites / MCS;
 *   12 acceptance rate over the window; 13 cell-cell share of the cells'
 *      interface pairs; 14 net displacement / path length;
 *   15 elongation: sqrt of the ratio of the principal second moments.
 * Centroids follow Methods, "Composite variable tracking" (Eq. 10); a cell
 * absent at some snapshot counts for 0..3, 13 and 15 only.  One kernel
 * launch; the batch keeps a scratch track buffer of n_snap * 2 * rows
 * doubles.  Asynchronous on the batch's stream. */
int cpm_batch_summarize(cpm_batch *b, const int64_t *cells_hist, const int64_t *member_hist, int32_t n_snap,
                        int32_t every, double *out);

/* Kernel launches issued for b (set-up included). */
int64_t cpm_batch_kernel_launches(const cpm_batch *b);

/* Message of the last failed call on b (of the calling thread's last failed
 * cpm_batch_create when b is NULL). */
const char *cpm_batch_last_error(const cpm_batch *b);

/* Free b and all its lattices (NULL is ignored).  Synchronises the stream. */
void cpm_batch_destroy(cpm_batch *b);

/* cpm_step_noalloc -- the sweep without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc, e.g. a host framework or plug-in that owns the
 * GPU's memory budget and only hands out fixed buffers, or code that must not
 * allocate while it runs because an allocation could block, fail half way or
 * escape the caller's memory accounting.  It runs n_subpasses sub-passes of
 * the same round kernel as cpm_step, from position (t, sp) (MCS index and
 * sub-pass within it), directly on the caller's device buffers:
 *   lattice    device, nx*ny*nz int32, read and updated in place;
 *   V, A       device, n_cells + 1 int32 each: the exact volume and interface
 *              tallies of that lattice on entry (e.g. from cpm_read_tallies),
 *              updated in place;
 *   cell_type  device, n_cells + 1 uint8.
 * cfg gives the model and schedule (its host pointer fields are ignored;
 * only the global schedule, tile = 0; at most 2^31 sites).  The result
 * equals what a handle at the same position would produce with
 * cpm_step_subpasses.
 * Precondition, not checked (cpm_create checks it for handles): every
 * lattice value lies in -1..n_cells and every cell_type entry is below
 * CPM_MAX_TYPES.  A violation is undefined behaviour: the kernel would index
 * the tallies and the type tables out of bounds.
 *
 * It allocates nothing: all scratch (second tally buffer, pending-change
 * buffers, threshold/log/exp tables, accept counter) lives in one fixed
 * file-scope device array of about 9.2 MiB, present on every GPU that loads
 * the library until the process exits.  Limits, beyond which the call
 * returns CPM_E_LIMIT without doing anything: at most 262,144 active blocks
 * per round (nx*ny*nz / a^d), at most 65,535 cells, a threshold table of at
 * most 32,768 entries (temperature up to about 92 in scaled units), and no
 * Act term.
 * The first call on a device looks up the array's device address with that
 * device current (a one-time set-up); make that first call before any stream
 * capture.  A call on a stream that is capturing returns CPM_E_INVALID: its
 * table uploads read host memory that the next call rewrites.  The tables
 * are built in static host buffers (not on the caller's stack) under a lock.
 * Every call shares the array and finds the previous call's
 * contents there; the call re-initialises everything it reads, but calls
 * that overlap on the GPU (other streams, other threads) race on it and must
 * be serialised by the caller.  Work is queued on cuda_stream; when accepts
 * is not NULL the call waits for it and stores the number of accepted copies
 * of this call there.  Returns CPM_OK, CPM_E_LIMIT, CPM_E_INVALID or
 * CPM_E_CUDA (cpm_last_error does not report on this call). */
int cpm_step_noalloc(const cpm_config *cfg, int32_t *lattice, int32_t *V, int32_t *A,
                     const uint8_t *cell_type, int64_t t, int32_t sp, int64_t n_subpasses,
                     void *cuda_stream, int64_t *accepts);

#ifdef __cplusplus
}
#endif

#endif /* CPM_GB300_H */
