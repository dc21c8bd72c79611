// cpm_step_noalloc: the sweep for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc: code running inside a host that owns
// the device memory budget (a simulation framework or plug-in that hands out
// fixed buffers), code that runs where an allocation could block or fail
// mid-run, and code whose memory must all be accounted for up front.  This
// entry point runs the same round kernel as cpm_step on buffers the caller
// passes in, and keeps every scratch buffer it needs (the second tally buffer,
// the pending-change buffers, the threshold/log/exp tables, the accept
// counter) in one file-scope device array of fixed size.  That array exists on
// every GPU that loads the library, from load until the process exits.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "../../include/cpm.h"
#include "cpm_internal.h"

using namespace cpmgb;

namespace {

// Limits of the static scratch (see include/cpm.h).
constexpr uint32_t kNaMaxActive = 262144;   // active blocks per round
constexpr int32_t kNaMaxCells = 65535;      // cell ids 1..65535
constexpr int32_t kNaMaxThr = 32768;        // threshold table entries (T <= 92)
constexpr int32_t kNaMaxExpq = 5120;

constexpr size_t kPendBytes = sizeof(int4) * 2 * (size_t)kNaMaxActive;
constexpr size_t kFlagBytes = 2 * (size_t)kNaMaxActive;
constexpr size_t kTallyBytes = sizeof(int32_t) * 2 * ((size_t)kNaMaxCells + 1);
constexpr size_t kThrBytes = sizeof(uint32_t) * (size_t)kNaMaxThr;
constexpr size_t kLnBytes = 1024;
constexpr size_t kExpqBytes = sizeof(int32_t) * (size_t)kNaMaxExpq;
constexpr size_t kOffPend = 0;
constexpr size_t kOffFlag = kOffPend + kPendBytes;
constexpr size_t kOffTally = kOffFlag + kFlagBytes;
constexpr size_t kOffThr = kOffTally + kTallyBytes;
constexpr size_t kOffLn = kOffThr + kThrBytes;
constexpr size_t kOffExpq = kOffLn + kLnBytes;
constexpr size_t kOffCount = kOffExpq + kExpqBytes;
constexpr size_t kScratchBytes = kOffCount + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {nullptr};

// Host copies of the integer tables, built by each call under g_table_mutex
// and uploaded from here (kept off the caller's stack: about 150 KiB, more
// than some worker threads have).  A host-to-device cudaMemcpyAsync from
// pageable memory returns once the source has been staged, so the next call
// may rebuild them as soon as this call has issued its copies.
std::mutex g_table_mutex;
uint32_t g_thr[kNaMaxThr];
int32_t g_ln[kLnEntries];
int32_t g_expq[kNaMaxExpq];
// Failures are reported by return code only (the message strings below are
// for the reader): CPM_E_LIMIT when a size exceeds the static scratch,
// CPM_E_INVALID for other bad arguments, CPM_E_CUDA for runtime errors.
int na_fail(int code, const char *) { return code; }

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is asked for
// once per device with that device current.
int scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return na_fail(CPM_E_CUDA, "cudaGetDevice failed");
    if (dev < 0 || dev >= kMaxDevices) return na_fail(CPM_E_INVALID, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) return na_fail(CPM_E_CUDA, "cudaGetSymbolAddress of the scratch failed");
        g_scratch_addr[dev] = (unsigned char *)p;
    }
    *out = g_scratch_addr[dev];
    return CPM_OK;
}

uint32_t na_ipow(uint32_t b, int e)
{
    uint32_t r = 1;
    while (e-- > 0) r *= b;
    return r;
}

}  // namespace

extern "C" int cpm_step_noalloc(const cpm_config *cfg, int32_t *lattice, int32_t *V, int32_t *A,
                                const uint8_t *cell_type, int64_t t, int32_t sp, int64_t n_subpasses,
                                void *cuda_stream, int64_t *accepts)
{
    if (!cfg || !lattice || !V || !A || !cell_type) return na_fail(CPM_E_INVALID, "NULL argument");
    const cpm_config &c = *cfg;
    if (c.dim != 2 && c.dim != 3) return na_fail(CPM_E_INVALID, "dim must be 2 or 3");
    if (c.nx < 3 || c.ny < 3 || (c.dim == 3 && c.nz < 3) || (c.dim == 2 && c.nz != 1))
        return na_fail(CPM_E_INVALID, "extents must be >= 3 (nz = 1 in 2D)");
    if (c.c < 2 || c.a < 2 || c.a % c.c) return na_fail(CPM_E_INVALID, "need c >= 2 and c | a");
    const uint32_t s = (uint32_t)(c.a / c.c);
    if ((uint32_t)c.a - s < 2) return na_fail(CPM_E_INVALID, "blocks of one colour must be >= 2 sites apart");
    if (c.nx % c.a || c.ny % c.a || (c.dim == 3 && c.nz % c.a))
        return na_fail(CPM_E_INVALID, "extents must be multiples of a");
    // the round kernel indexes sites with 32-bit integers
    if ((uint64_t)c.nx * (uint64_t)c.ny * (uint64_t)c.nz > (1ull << 31))
        return na_fail(CPM_E_INVALID, "more than 2^31 sites");
    const uint32_t C = na_ipow((uint32_t)c.c, c.dim);
    if (C > 27) return na_fail(CPM_E_INVALID, "at most 27 colours");
    const uint32_t sd = na_ipow(s, c.dim);
    if (c.P < 1 || sd % (uint32_t)c.P) return na_fail(CPM_E_INVALID, "P must divide s^d");
    if (c.obstacle_type < 1 || c.obstacle_type >= CPM_MAX_TYPES) return na_fail(CPM_E_INVALID, "bad obstacle_type");
    for (int a = 0; a < CPM_MAX_TYPES; a++) {
        for (int b = 0; b < CPM_MAX_TYPES; b++)
            if (c.J[a][b] != c.J[b][a]) return na_fail(CPM_E_INVALID, "J must be symmetric");
        if (c.lambda_act[a] != 0) return na_fail(CPM_E_LIMIT, "the Act term is not available here");
        if (c.lambda_v[a] < 0 || c.lambda_p[a] < 0) return na_fail(CPM_E_INVALID, "lambdas must be >= 0");
    }
    if (c.n_cells < 0 || c.n_cells > kNaMaxCells) return na_fail(c.n_cells < 0 ? CPM_E_INVALID : CPM_E_LIMIT, "n_cells above the limit");
    const uint32_t nbx = (uint32_t)c.nx / s, nby = (uint32_t)c.ny / s, nbz = c.dim == 3 ? (uint32_t)c.nz / s : 1;
    const uint64_t n_active = (uint64_t)nbx * nby * nbz / C;
    if (n_active > kNaMaxActive) return na_fail(CPM_E_LIMIT, "too many active blocks per round for the scratch");
    if (t < 0 || sp < 0 || sp >= (int32_t)(C * (uint32_t)c.P) || n_subpasses < 0)
        return na_fail(CPM_E_INVALID, "bad position or count");
    if (!(c.temperature > 0.0)) return na_fail(CPM_E_INVALID, "temperature must be > 0");
    if (c.tile != 0) return na_fail(CPM_E_INVALID, "only the global schedule (tile = 0) runs here");
    bool motility = c.chem_field != nullptr;
    for (int a = 0; a < CPM_MAX_TYPES; a++) motility |= c.lambda_chem[a] != 0 || c.lambda_pers[a] != 0;
    if (motility) return na_fail(CPM_E_INVALID, "no motility terms here");

    // the threshold table must fit the scratch: L is the first h with THR[h] = 0
    int32_t L = 0;
    while (std::floor(std::ldexp(std::exp(-(double)L / (16.0 * c.temperature)), 32)) > 0.0)
        if (++L > kNaMaxThr) return na_fail(CPM_E_LIMIT, "temperature too high for the scratch table");

    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the table uploads below read host memory that this call rebuilds next
    // time, so a copy recorded into a graph would not keep its contents
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return na_fail(CPM_E_CUDA, "cudaStreamIsCapturing failed");
    if (cap != cudaStreamCaptureStatusNone) return na_fail(CPM_E_INVALID, "the stream is capturing");

    unsigned char *scr = nullptr;
    int rc = scratch_for_current_device(&scr);
    if (rc) return rc;
    int4 *pend = (int4 *)(scr + kOffPend);
    uint8_t *flags = scr + kOffFlag;
    int32_t *V1 = (int32_t *)(scr + kOffTally);
    int32_t *A1 = V1 + (kNaMaxCells + 1);
    uint32_t *d_thr = (uint32_t *)(scr + kOffThr);
    int32_t *d_ln = (int32_t *)(scr + kOffLn);
    int32_t *d_expq = (int32_t *)(scr + kOffExpq);
    unsigned long long *d_count = (unsigned long long *)(scr + kOffCount);
    const size_t tb = sizeof(int32_t) * ((size_t)c.n_cells + 1);

#define NA_TRY(expr)                                                            \
    do {                                                                        \
        if ((expr) != cudaSuccess) return na_fail(CPM_E_CUDA, #expr " failed"); \
    } while (0)
    // the scratch keeps the previous call's contents: set everything this call reads
    {
        std::lock_guard<std::mutex> lock(g_table_mutex);
        for (int32_t h = 0; h < L; h++) {
            const double v = std::floor(std::ldexp(std::exp(-(double)h / (16.0 * c.temperature)), 32));
            g_thr[h] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
        }
        g_ln[0] = 0;
        for (int a = 1; a < kLnEntries; a++) g_ln[a] = (int32_t)std::llround(std::ldexp(std::log((double)a), 16));
        const int32_t ne = (g_ln[kLnEntries - 1] >> 6) + 1;
        if (ne > kNaMaxExpq) return na_fail(CPM_E_INVALID, "exp table too long");
        for (int m = 0; m < ne; m++)
            g_expq[m] = (int32_t)std::llround(std::ldexp(std::exp((double)m / 1024.0), 16));
        NA_TRY(cudaMemcpyAsync(d_thr, g_thr, sizeof(uint32_t) * (size_t)L, cudaMemcpyHostToDevice, st));
        NA_TRY(cudaMemcpyAsync(d_ln, g_ln, sizeof g_ln, cudaMemcpyHostToDevice, st));
        NA_TRY(cudaMemcpyAsync(d_expq, g_expq, sizeof(int32_t) * (size_t)ne, cudaMemcpyHostToDevice, st));
    }
    NA_TRY(cudaMemsetAsync(flags, 0, 2 * (size_t)n_active, st));
    NA_TRY(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st));
    NA_TRY(cudaMemcpyAsync(V1, V, tb, cudaMemcpyDeviceToDevice, st));
    NA_TRY(cudaMemcpyAsync(A1, A, tb, cudaMemcpyDeviceToDevice, st));

    RoundArgs a;
    memset(&a, 0, sizeof a);
    a.lat = lattice;
    a.packed = 0;  // no Act term here: the words are plain ids
    a.pdl = 1;     // each round overlaps its set-up with the previous round's tail
    a.cell_type = cell_type;
    a.thr = d_thr;
    a.ln_tab = d_ln;
    a.expq = d_expq;
    a.accepts = d_count;
    a.L = L;
    a.nx = (uint32_t)c.nx; a.ny = (uint32_t)c.ny; a.nz = (uint32_t)c.nz;
    a.s = s; a.c = (uint32_t)c.c; a.sd = sd;
    a.nbx = nbx; a.nby = nby;
    a.nax = nbx / (uint32_t)c.c; a.nay = nby / (uint32_t)c.c;
    a.n_active = (uint32_t)n_active;
    a.key0 = (uint32_t)c.seed;
    a.key1 = (uint32_t)(c.seed >> 32);
    pick_bricks(c.dim, a.nax, a.nay, a);
    memcpy(a.tp.J, c.J, sizeof a.tp.J);
    memcpy(a.tp.lambda_v, c.lambda_v, sizeof a.tp.lambda_v);
    memcpy(a.tp.v_target, c.v_target, sizeof a.tp.v_target);
    memcpy(a.tp.lambda_p, c.lambda_p, sizeof a.tp.lambda_p);
    memcpy(a.tp.a_target, c.a_target, sizeof a.tp.a_target);
    memcpy(a.tp.lambda_act, c.lambda_act, sizeof a.tp.lambda_act);
    memcpy(a.tp.max_act, c.max_act, sizeof a.tp.max_act);
    a.tp.obstacle_type = c.obstacle_type;
    bool perim = false;
    for (int k = 0; k < CPM_MAX_TYPES; k++)
        if (c.lambda_p[k]) perim = true;

    int32_t *Vb[2] = {V, V1}, *Ab[2] = {A, A1};
    const uint32_t k_rounds = sd / (uint32_t)c.P;
    const uint32_t per_mcs = C * (uint32_t)c.P;
    uint64_t g = 0;
    for (int64_t it = 0; it < n_subpasses; it++) {
        // colour of this sub-pass: Fisher-Yates over the colours of its cycle
        uint32_t perm[27];
        for (uint32_t q = 0; q < C; q++) perm[q] = q;
        for (uint32_t i = C - 1; i >= 1; i--) {
            const Philox4 w = philox4x32_10(i, (uint32_t)sp / C, (uint32_t)t, 1u << 24, a.key0, a.key1);
            const uint32_t j = draw_below(w.v[0], i + 1);
            const uint32_t tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
        const uint32_t col = perm[(uint32_t)sp % C];
        a.cx = col % (uint32_t)c.c;
        a.cy = (col / (uint32_t)c.c) % (uint32_t)c.c;
        a.cz = col / ((uint32_t)c.c * (uint32_t)c.c);
        a.t = (uint32_t)t;
        a.sp = (uint32_t)sp;
        for (uint32_t r = 0; r < k_rounds; r++, g++) {
            const int cur = (int)(g & 1);
            a.r = r;
            a.Vc = Vb[cur];
            a.Ac = Ab[cur];
            a.Vn = Vb[cur ^ 1];
            a.An = Ab[cur ^ 1];
            a.pend_prev = pend + (size_t)(cur ^ 1) * n_active;
            a.pend_cur = pend + (size_t)cur * n_active;
            a.flag_prev = flags + (size_t)(cur ^ 1) * n_active;
            a.flag_cur = flags + (size_t)cur * n_active;
            NA_TRY(launch_round(c.dim, perim, false, a, st));
        }
        if (++sp == (int32_t)per_mcs) {
            sp = 0;
            t++;
        }
    }
    // the current tallies are in buffer g & 1; hand them back in V and A
    if (g & 1) {
        NA_TRY(cudaMemcpyAsync(V, V1, tb, cudaMemcpyDeviceToDevice, st));
        NA_TRY(cudaMemcpyAsync(A, A1, tb, cudaMemcpyDeviceToDevice, st));
    }
    if (accepts) {
        unsigned long long n = 0;
        NA_TRY(cudaMemcpyAsync(&n, d_count, sizeof n, cudaMemcpyDeviceToHost, st));
        NA_TRY(cudaStreamSynchronize(st));
        *accepts = (int64_t)n;
    }
#undef NA_TRY
    return CPM_OK;
}

