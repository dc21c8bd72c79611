// The emulator: an ensemble of small MLPs mapping the seven swept CPM
// parameters to summary statistics of a run.  BF16 weights and activations,
// FP32 accumulation, FP32 master weights and Adam moments.
//
// Member e of the ensemble is the network
//     Z_l = H_{l-1} W_l^T + b_l,  H_l = GELU(Z_l)  (hidden layers),
//     P   = H_{L-1} W_L^T + b_L                    (linear output),
// with GELU(z) = z Phi(z) (Hendrycks & Gimpel 2016), trained on the mean
// squared error with Adam (Kingma & Ba 2015, Algorithm 1).  Every kernel
// runs all members in one launch (grid.z = member), each member reading its
// own slice of the flat parameter buffer.
//
// The forward layers (A [M][K] times W^T, N <= 256, K <= 256) run on the
// fifth-generation tensor cores (tcgen05.mma into TMEM, gemm_tc_kernel).  The
// backward GEMMs (transposed operands) use mma.sync m16n8k16 (bf16 x bf16 ->
// f32) on 64 x 64 CTA tiles with a 32-deep K slab, double-buffered in shared
// memory.  Bias, GELU and GELU' are fused into the epilogues.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>

#include "../../include/cpm_emulator.h"

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32, kLds = kBK + 8;  // smem row stride (halves): 80 B, conflict-free
constexpr int kGemmThreads = 128;                             // 4 warps, 2 x 2, each 32 x 32 of the tile

// Standard normal CDF Phi(z) = (1 + erf(z / sqrt 2)) / 2 and the density
// term exp(-z^2 / 2), with erf from the rational approximation of
// Abramowitz & Stegun, Handbook of Mathematical Functions, formula 7.1.26
// (after Hastings): for x >= 0,
//   erf(x) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) exp(-x^2) + e(x),
//   t = 1 / (1 + p x),  |e(x)| <= 1.5e-7,
// p = 0.3275911, a1..a5 = 0.254829592, -0.284496736, 1.421413741,
// -1.453152027, 1.061405429.  The reciprocal and the exponential are the
// fast hardware approximations.  With float32 rounding the |Phi error| stays
// below 4e-7 (the tests pin it on a dense grid against float64), far under
// the bf16 rounding (2^-9) of the activations that the epilogue stores.  The
// GELU epilogue is issue-bound, and this form is shorter than erff.
__device__ __forceinline__ float phi_f(float z, float &dens)
{
    const float x = fabsf(z) * 0.70710678118654752f;
    dens = __expf(-x * x);  // exp(-z^2 / 2)
    const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
    float poly = 1.061405429f;
    poly = fmaf(poly, t, -1.453152027f);
    poly = fmaf(poly, t, 1.421413741f);
    poly = fmaf(poly, t, -0.284496736f);
    poly = fmaf(poly, t, 0.254829592f);
    const float half_tail = 0.5f * poly * t * dens;  // (1 - erf(x)) / 2
    return z >= 0.0f ? 1.0f - half_tail : half_tail;
}

__device__ __forceinline__ float gelu_f(float z)
{
    float dens;
    return z * phi_f(z, dens);
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    float dens;
    const float cdf = phi_f(z, dens);
    return cdf + z * 0.39894228040143268f * dens;
}

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16 *A;
    int64_t lda, sa;
    const __nv_bfloat16 *B;
    int64_t ldb, sb;
    const float *bias;
    int64_t sbias;
    void *C;
    int64_t ldc, sc;
    float *Z;  // EPI_GELU: pre-activation out (may be null); EPI_DGELU: pre-activation in
    int64_t ldz, sz;
    int epi, c_f32, vec_a, vec_b;
};

// Loads one 64 x 32 slab of an operand whose shared-memory image is S[row][k].
// Non-transposed: X[row * ld + k] (k contiguous); transposed: X[k * ld + row].
template <bool TRANS>
struct SlabLoader {
    uint4 v[2];
    __device__ __forceinline__ void load(const __nv_bfloat16 *X, int64_t ld, int rows, int K, int r0, int k0, bool vec)
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = tid + i * kGemmThreads;  // 256 vectors of 8 halves
            int row, k;
            if (!TRANS) {
                row = e >> 2;
                k = (e & 3) * 8;
            } else {
                k = e >> 3;
                row = (e & 7) * 8;
            }
            const int gr = r0 + row, gk = k0 + k;
            __align__(16) __nv_bfloat16 h[8];
            if (!TRANS) {
                if (vec && gr < rows && gk + 8 <= K) {
                    v[i] = *reinterpret_cast<const uint4 *>(X + (int64_t)gr * ld + gk);
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    h[j] = (gr < rows && gk + j < K) ? X[(int64_t)gr * ld + gk + j] : __float2bfloat16(0.0f);
            } else {
                if (vec && gk < K && gr + 8 <= rows) {
                    v[i] = *reinterpret_cast<const uint4 *>(X + (int64_t)gk * ld + gr);
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    h[j] = (gk < K && gr + j < rows) ? X[(int64_t)gk * ld + gr + j] : __float2bfloat16(0.0f);
            }
            v[i] = *reinterpret_cast<const uint4 *>(h);
        }
    }
    __device__ __forceinline__ void store(__nv_bfloat16 (*S)[kLds]) const
    {
        const int tid = threadIdx.x;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = tid + i * kGemmThreads;
            if (!TRANS) {
                *reinterpret_cast<uint4 *>(&S[e >> 2][(e & 3) * 8]) = v[i];
            } else {
                const int k = e >> 3, row = (e & 7) * 8;
                const __nv_bfloat16 *h = reinterpret_cast<const __nv_bfloat16 *>(&v[i]);
#pragma unroll
                for (int j = 0; j < 8; ++j) S[row + j][k] = h[j];
            }
        }
    }
};

// C[m][n] = sum_k op(A)[m][k] op(B)[k][n], op(A)[m][k] = TA ? A[k][m] : A[m][k],
// op(B)[k][n] = TB ? B[n][k] : B[k][n]; then the epilogue.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(const GemmArgs p)
{
    __shared__ __align__(16) __nv_bfloat16 As[2][kBM][kLds];
    __shared__ __align__(16) __nv_bfloat16 Bs[2][kBN][kLds];
    const int z = blockIdx.z;
    const __nv_bfloat16 *A = p.A + z * p.sa;
    const __nv_bfloat16 *B = p.B + z * p.sb;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tq = lane & 3;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    SlabLoader<TA> la;
    SlabLoader<!TB> lb;  // B's image is Bs[n][k]: a plain row load when B is stored [n][k]
    const int nk = (p.K + kBK - 1) / kBK;
    la.load(A, p.lda, p.M, p.K, m0, 0, p.vec_a);
    lb.load(B, p.ldb, p.N, p.K, n0, 0, p.vec_b);
    la.store(As[0]);
    lb.store(Bs[0]);
    __syncthreads();
    for (int t = 0; t < nk; ++t) {
        const int cur = t & 1;
        if (t + 1 < nk) {
            la.load(A, p.lda, p.M, p.K, m0, (t + 1) * kBK, p.vec_a);
            lb.load(B, p.ldb, p.N, p.K, n0, (t + 1) * kBK, p.vec_b);
        }
#pragma unroll
        for (int ks = 0; ks < kBK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[cur][r][ks + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[cur][r + 8][ks + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[cur][r][ks + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[cur][r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bfr[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[cur][c][ks + 2 * tq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[cur][c][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bfr[j][0]),
                          "r"(bfr[j][1]));
        }
        if (t + 1 < nk) {
            la.store(As[cur ^ 1]);
            lb.store(Bs[cur ^ 1]);
        }
        __syncthreads();
    }

    // epilogue: accumulator element r of fragment (i, j) sits at row g (+8 for r >= 2), column 2 tq + (r & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int gm = m0 + wm + i * 16 + g + (r >= 2 ? 8 : 0);
                const int gn = n0 + wn + j * 8 + 2 * tq + (r & 1);
                if (gm >= p.M || gn >= p.N) continue;
                float v = acc[i][j][r];
                if (p.bias) v += p.bias[z * p.sbias + gn];
                if (p.epi == CPM_MLP_EPI_GELU) {
                    if (p.Z) p.Z[z * p.sz + (int64_t)gm * p.ldz + gn] = v;
                    v = gelu_f(v);
                } else if (p.epi == CPM_MLP_EPI_DGELU) {
                    v *= gelu_grad_f(p.Z[z * p.sz + (int64_t)gm * p.ldz + gn]);
                }
                const int64_t o = z * p.sc + (int64_t)gm * p.ldc + gn;
                if (p.c_f32) static_cast<float *>(p.C)[o] = v;
                else static_cast<__nv_bfloat16 *>(p.C)[o] = __float2bfloat16(v);
            }
}

// db[z][n] = sum over rows of dZ[z][row][n]; one CTA per 32 columns and member,
// 8 row groups reduced through shared memory in a fixed order (deterministic).
__global__ void __launch_bounds__(256) bias_grad_kernel(int rows, int N, const __nv_bfloat16 *dZ, int64_t ld,
                                                        int64_t sdz, float *db, int64_t sdb)
{
    __shared__ float part[8][33];
    const int z = blockIdx.z;
    const int col = threadIdx.x & 31, rg = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + col;
    float s = 0.0f;
    if (n < N)
        for (int r = rg; r < rows; r += 8) s += __bfloat162float(dZ[z * sdz + (int64_t)r * ld + n]);
    part[rg][col] = s;
    __syncthreads();
    if (rg == 0 && n < N) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += part[k][col];
        db[z * sdb + n] = t;
    }
}

// per member: loss[z] += mean (P - Y)^2 over count elements; dP = 2 (P - Y) / count in bf16
__global__ void mse_kernel(int64_t count, const float *P, int64_t sp, const float *Y, int64_t sy, __nv_bfloat16 *dP,
                           float *loss)
{
    const int z = blockIdx.y;
    float s = 0.0f;
    const float inv = 1.0f / (float)count;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const float d = P[z * sp + e] - Y[z * sy + e];
        if (dP) dP[z * sp + e] = __float2bfloat16(2.0f * d * inv);
        s += d * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss + z, s * inv);
}

__global__ void adam_kernel(int64_t n, float *w, __nv_bfloat16 *wb, const float *grad, float *m, float *v, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gr = grad[e];
        const float mm = b1 * m[e] + (1.0f - b1) * gr;
        const float vv = b2 * v[e] + (1.0f - b2) * gr * gr;
        m[e] = mm;
        v[e] = vv;
        const float wn = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        w[e] = wn;
        if (wb) wb[e] = __float2bfloat16(wn);
    }
}

__global__ void cast_kernel(int64_t n, const float *x, __nv_bfloat16 *y)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(x[e]);
}

// xb[r][:] = bf16(X[src][:]), yb[r][:] = Y[src][:], src = order ? order[off + r] : off + r
__global__ void gather_kernel(int rows, int n_in, int n_out, const float *X, const float *Y, const int32_t *order,
                              int64_t off, int64_t n_total, __nv_bfloat16 *xb, float *yb, int *bad)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const int64_t src = order ? (int64_t)order[off + r] : off + r;
    if (src < 0 || src >= n_total) {
        atomicExch(bad, 1);
        return;
    }
    for (int i = 0; i < n_in; ++i) xb[(int64_t)r * n_in + i] = __float2bfloat16(X[src * n_in + i]);
    if (Y)
        for (int k = 0; k < n_out; ++k) yb[(int64_t)r * n_out + k] = Y[src * n_out + k];
}

// Ensemble mean / std over members for each (row, statistic); the mean is
// mapped back to the statistic's units (y = mean * scale + shift, then exp
// where log_mask is set); fallback[row] = 1 when any statistic's std (in the
// network's standardised units) exceeds factor * rmse.
__global__ void predict_kernel(int rows, int n_members, int n_out, const float *out, int64_t s_member,
                               const float *shift, const float *scale, const uint8_t *log_mask, const float *rmse,
                               float factor, float *mean_out, float *std_out, uint8_t *fallback)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    int fb = 0;
    for (int k = 0; k < n_out; ++k) {
        float s = 0.0f;
        for (int e = 0; e < n_members; ++e) s += out[e * s_member + (int64_t)r * n_out + k];
        const float mu = s / (float)n_members;
        float q = 0.0f;
        for (int e = 0; e < n_members; ++e) {
            const float d = out[e * s_member + (int64_t)r * n_out + k] - mu;
            q += d * d;
        }
        const float sd = sqrtf(q / (float)n_members);
        float y = mu * scale[k] + shift[k];
        if (log_mask[k]) y = expf(y);
        if (mean_out) mean_out[(int64_t)r * n_out + k] = y;
        if (std_out) std_out[(int64_t)r * n_out + k] = sd;
        if (rmse && sd > factor * rmse[k]) fb = 1;
    }
    if (fallback) fallback[r] = (uint8_t)fb;
}

// ---------------------------------------------------------------------------
// Forward GEMM on the fifth-generation tensor cores: C = epi(A W^T + b) with
// A [M][K] and W [N][K] both K-major (the layout of every forward layer).
// Persistent CTAs take contiguous ranges of 128-row tiles (members outer), so
// a member's weights are staged once per CTA.  The weight slab (N x Kp) and
// the activation tile (128 x Kp) sit in shared memory in the canonical
// no-swizzle K-major layout: 8-row x 16-byte core matrices, K-adjacent core
// matrices 128 B apart (leading byte offset), 8-row groups Kp/8 x 128 B apart
// (stride byte offset).  One thread issues Kp/16 tcgen05.mma (bf16 x bf16 ->
// f32, M = 128, N <= 256) into a TMEM accumulator and commits them to an
// mbarrier; after a bounded wait the 32 warps read the accumulator with
// tcgen05.ld (warp w owns TMEM lanes 32 (w % 4) .. + 31 and every eighth
// 16-column chunk) and apply the bias / GELU epilogue.  The epilogue is what
// bounds the kernel, so it gets the most warps a CTA can have (1M-point
// prediction: 85.7 M points/s against 82.0 with 16 warps).
constexpr int kTcThreads = 1024;
constexpr int kTcM = 128;
constexpr uint32_t kTcSpinLimit = 1u << 22;
constexpr int kTcNotApplicable = 1;  // launch_gemm_tc: use the mma.sync kernel instead

struct TcArgs {
    int M, N, K, Kp, ncols;
    const __nv_bfloat16 *A;
    int64_t lda, sa;
    const __nv_bfloat16 *B;
    int64_t ldb, sb;
    const float *bias;
    int64_t sbias;
    void *C;
    int64_t ldc, sc;
    float *Z;
    int64_t ldz, sz;
    int epi, c_f32, vec_a, vec_b, vec_c;
    int mtiles, tiles;
    int *err;
    int report_timeout;  // test hook: report the first accumulator wait as timed out once it has completed
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ bool tc_wait(uint64_t *mbar, uint32_t parity)
{
    const uint32_t addr = smem_u32(mbar);
    for (uint32_t it = 0; it < kTcSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// rows [r0, r0 + rows_tile) x [0, Kp) of X into the core-matrix layout, zero outside [0, rows) x [0, K);
// element e of the layout is core matrix e / 8 (8-row group outer, K chunk inner), row e % 8
__device__ __forceinline__ void tc_stage(unsigned char *S, const __nv_bfloat16 *X, int64_t ld, int rows, int K, int r0,
                                         int rows_tile, int Kp, bool vec)
{
    const int kc = Kp / 8;
    const int n = rows_tile * kc;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int rr = e & 7, k8 = (e >> 3) % kc, r8 = (e >> 3) / kc;
        const int gr = r0 + r8 * 8 + rr, gk = k8 * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < rows) {
            if (vec && gk + 8 <= K) {
                v = *reinterpret_cast<const uint4 *>(X + (int64_t)gr * ld + gk);
            } else {
                __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = gk + j < K ? X[(int64_t)gr * ld + gk + j] : __float2bfloat16(0.0f);
                v = *reinterpret_cast<const uint4 *>(h);
            }
        }
        *reinterpret_cast<uint4 *>(S + (size_t)e * 16) = v;
    }
}

// As tc_stage for 16-byte aligned rows with K a multiple of 8, issued as
// cp.async copies (rows past `rows` are zero-filled without reading);
// completion: cp.async.wait_all, then fence.proxy.async before the MMAs read.
__device__ __forceinline__ void tc_stage_async(unsigned char *S, const __nv_bfloat16 *X, int64_t ld, int rows, int r0,
                                               int rows_tile, int Kp)
{
    const int kc = Kp / 8;
    const int n = rows_tile * kc;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int rr = e & 7, k8 = (e >> 3) % kc, r8 = (e >> 3) / kc;
        const int gr = r0 + r8 * 8 + rr;
        const bool in = gr < rows;
        const __nv_bfloat16 *src = X + (in ? (int64_t)gr * ld + k8 * 8 : 0);
        const unsigned dst = (unsigned)__cvta_generic_to_shared(S + (size_t)e * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__global__ void __launch_bounds__(kTcThreads, 1) gemm_tc_kernel(const TcArgs p)
{
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    unsigned char *Bs = tc_smem;                                          // N x Kp
    unsigned char *As = tc_smem + (size_t)p.N * p.Kp * 2;                 // 128 x Kp
    float *bias_s = reinterpret_cast<float *>(tc_smem + (size_t)(p.N + kTcM) * p.Kp * 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"((uint32_t)p.ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    const int t0 = (int)((int64_t)p.tiles * blockIdx.x / gridDim.x);
    const int t1 = (int)((int64_t)p.tiles * (blockIdx.x + 1) / gridDim.x);
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(p.N >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t sbo = (uint32_t)(p.Kp / 8) * 128u;
    const int q = warp & 3, part = warp >> 2, nparts = kTcThreads / 128, nchunk = p.N / 16;
    int cur_z = -1;
    uint32_t phase = 0;
    bool aborted = false;
    // the activation tile of the first tile; later tiles are prefetched during the previous epilogue
    const bool async_a = p.vec_a && p.K % 8 == 0;
    if (t0 < t1) {
        const int z = t0 / p.mtiles, m0 = (t0 % p.mtiles) * kTcM;
        if (async_a) {
            tc_stage_async(As, p.A + z * p.sa, p.lda, p.M, m0, kTcM, p.Kp);
            asm volatile("cp.async.wait_all;\n" ::: "memory");
        } else {
            tc_stage(As, p.A + z * p.sa, p.lda, p.M, p.K, m0, kTcM, p.Kp, p.vec_a);
        }
    }
    for (int t = t0; t < t1; ++t) {
        const int z = t / p.mtiles, m0 = (t % p.mtiles) * kTcM;
        if (z != cur_z) {
            tc_stage(Bs, p.B + z * p.sb, p.ldb, p.N, p.K, 0, p.N, p.Kp, p.vec_b);
            for (int n = threadIdx.x; n < p.N; n += blockDim.x) bias_s[n] = p.bias ? p.bias[z * p.sbias + n] : 0.0f;
            cur_z = z;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
            for (int ks = 0; ks < p.Kp / 16; ++ks) {
                const uint64_t ad = tc_desc(a0 + ks * 256u, 128u, sbo), bd = tc_desc(b0 + ks * 256u, 128u, sbo);
                asm volatile("{\n .reg .pred acc;\n setp.ne.b32 acc, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, acc;\n}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(ks > 0 ? 1 : 0)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        // (with report_timeout the wait still completes: the MMAs are done before the failure path runs)
        const bool ok = tc_wait(&mbar, phase) && !p.report_timeout;
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        // the MMAs are done with the activation tile: fetch the next one behind the epilogue
        const bool next = t + 1 < t1;
        int z1 = 0, m1 = 0;
        if (next) {
            z1 = (t + 1) / p.mtiles;
            m1 = ((t + 1) % p.mtiles) * kTcM;
            if (async_a) tc_stage_async(As, p.A + z1 * p.sa, p.lda, p.M, m1, kTcM, p.Kp);
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = m0 + q * 32 + lane;
        for (int ch = part; ch < nchunk; ch += nparts) {
            uint32_t r[16];
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 16);
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
                         "%12, %13, %14, %15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < p.M) {
                const int n0 = ch * 16;
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]) + bias_s[n0 + j];
                if (p.epi == CPM_MLP_EPI_GELU) {
                    if (p.Z) {
                        float *zr = p.Z + z * p.sz + (int64_t)row * p.ldz + n0;
                        if (p.vec_c) {
#pragma unroll
                            for (int j = 0; j < 16; j += 4)
                                *reinterpret_cast<float4 *>(zr + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) zr[j] = v[j];
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = gelu_f(v[j]);
                }
                const int64_t o = z * p.sc + (int64_t)row * p.ldc + n0;
                if (p.c_f32) {
                    float *cr = static_cast<float *>(p.C) + o;
                    if (p.vec_c) {
#pragma unroll
                        for (int j = 0; j < 16; j += 4)
                            *reinterpret_cast<float4 *>(cr + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) cr[j] = v[j];
                    }
                } else {
                    __nv_bfloat16 *cr = static_cast<__nv_bfloat16 *>(p.C) + o;
                    __align__(16) __nv_bfloat16 hb[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) hb[j] = __float2bfloat16(v[j]);
                    if (p.vec_c) {
                        reinterpret_cast<uint4 *>(cr)[0] = reinterpret_cast<const uint4 *>(hb)[0];
                        reinterpret_cast<uint4 *>(cr)[1] = reinterpret_cast<const uint4 *>(hb)[1];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) cr[j] = hb[j];
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (next) {
            if (async_a) asm volatile("cp.async.wait_all;\n" ::: "memory");
            else {
                __syncthreads();  // every warp is done with the tile before it is overwritten
                tc_stage(As, p.A + z1 * p.sa, p.lda, p.M, p.K, m1, kTcM, p.Kp, p.vec_a);
            }
        }
        __syncthreads();
    }
    if (aborted) {
        // record the timeout, then give the issued MMAs another bounded wait before freeing TMEM
        if (threadIdx.x == 0 && p.err) atomicExch(p.err, 1);
        tc_wait(&mbar, phase ^ 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)p.ncols)
                     : "memory");
}

unsigned grid1(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The tensor-core path takes the forward layout (A [M][K], W [N][K]) with
// N a multiple of 16 up to 256 and K up to 256.
bool tc_eligible(int ta, int tb, const GemmArgs &a)
{
    return ta == 0 && tb == 1 && a.epi != CPM_MLP_EPI_DGELU && a.N >= 16 && a.N <= 256 && a.N % 16 == 0 &&
           a.K >= 1 && a.K <= 256;
}

int launch_gemm_tc(const GemmArgs &a, int batch, int *err, cudaStream_t st, int report_timeout)
{
    TcArgs p{};
    p.report_timeout = report_timeout;
    p.M = a.M;
    p.N = a.N;
    p.K = a.K;
    p.Kp = (a.K + 15) / 16 * 16;
    p.ncols = 32;
    while (p.ncols < a.N) p.ncols *= 2;
    p.A = a.A;
    p.lda = a.lda;
    p.sa = a.sa;
    p.B = a.B;
    p.ldb = a.ldb;
    p.sb = a.sb;
    p.bias = a.bias;
    p.sbias = a.sbias;
    p.C = a.C;
    p.ldc = a.ldc;
    p.sc = a.sc;
    p.Z = a.Z;
    p.ldz = a.ldz;
    p.sz = a.sz;
    p.epi = a.epi;
    p.c_f32 = a.c_f32;
    p.vec_a = a.vec_a;
    p.vec_b = a.vec_b;
    // 16-element runs of C (and Z) start 16-byte aligned
    p.vec_c = aligned16(a.C) && a.ldc % 8 == 0 && a.sc % 8 == 0 && (!a.Z || (aligned16(a.Z) && a.ldz % 4 == 0 && a.sz % 4 == 0));
    p.mtiles = (a.M + kTcM - 1) / kTcM;
    p.tiles = p.mtiles * batch;
    p.err = err;
    size_t smem = (size_t)(a.N + kTcM) * p.Kp * 2 + (size_t)a.N * 4;
    // at most 512 / ncols CTAs may hold TMEM on one SM: pad the shared memory so that no more are resident
    const int per_sm_tmem = 512 / p.ncols;
    const size_t floor_smem = per_sm_tmem >= 8 ? 0 : (size_t)(228 * 1024) / (size_t)(per_sm_tmem + 1) + 1024;
    if (smem < floor_smem) smem = floor_smem;
    static int sms = 0, max_dyn = 0;
    if (sms == 0) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, gemm_tc_kernel);
        max_dyn = optin - (int)fa.sharedSizeBytes;
        if (cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dyn) != cudaSuccess)
            max_dyn = 48 * 1024 - (int)fa.sharedSizeBytes;
        cudaGetLastError();
    }
    if (smem > (size_t)max_dyn) return kTcNotApplicable;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_tc_kernel, kTcThreads, smem);
    if (per_sm < 1) per_sm = 1;
    int grid = sms * per_sm;
    if (grid > p.tiles) grid = p.tiles;
    gemm_tc_kernel<<<grid, kTcThreads, smem, st>>>(p);
    return cudaPeekAtLastError() == cudaSuccess ? CPM_MLP_OK : CPM_MLP_E_CUDA;
}

int launch_gemm(int ta, int tb, GemmArgs &a, int batch, cudaStream_t st, int *tc_err = nullptr,
                bool allow_tc = true, int *report_timeout = nullptr)
{
    if (a.M == 0 || a.N == 0) return CPM_MLP_OK;
    // vector loads need 16-byte aligned rows: base, leading dimension and member stride
    a.vec_a = aligned16(a.A) && a.lda % 8 == 0 && a.sa % 8 == 0;
    a.vec_b = aligned16(a.B) && a.ldb % 8 == 0 && a.sb % 8 == 0;
    if (allow_tc && tc_eligible(ta, tb, a)) {
        const int rc = launch_gemm_tc(a, batch, tc_err, st, report_timeout ? *report_timeout : 0);
        if (rc != kTcNotApplicable) {
            if (report_timeout) *report_timeout = 0;  // armed for one launch
            return rc;
        }
    }
    const dim3 grid((a.N + kBN - 1) / kBN, (a.M + kBM - 1) / kBM, batch);
    if (grid.y > 65535u || batch > 65535) return CPM_MLP_E_INVALID;
    if (ta) {
        if (tb) gemm_kernel<true, true><<<grid, kGemmThreads, 0, st>>>(a);
        else gemm_kernel<true, false><<<grid, kGemmThreads, 0, st>>>(a);
    } else {
        if (tb) gemm_kernel<false, true><<<grid, kGemmThreads, 0, st>>>(a);
        else gemm_kernel<false, false><<<grid, kGemmThreads, 0, st>>>(a);
    }
    return cudaPeekAtLastError() == cudaSuccess ? CPM_MLP_OK : CPM_MLP_E_CUDA;
}

}  // namespace

struct cpm_mlp {
    cpm_mlp_shape sh{};
    int n_layers = 0;
    int in_dim[CPM_MLP_MAX_LAYERS]{}, out_dim[CPM_MLP_MAX_LAYERS]{};
    int64_t off_w[CPM_MLP_MAX_LAYERS]{}, off_b[CPM_MLP_MAX_LAYERS]{};
    int64_t P = 0;  // parameters per member
    cudaStream_t st = nullptr;
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    __nv_bfloat16 *wb = nullptr;
    __nv_bfloat16 *xb = nullptr;
    float *yb = nullptr;
    __nv_bfloat16 *H[CPM_MLP_MAX_LAYERS]{};
    float *Z[CPM_MLP_MAX_LAYERS]{};
    float *out = nullptr;
    __nv_bfloat16 *dP = nullptr, *dZ[2]{};
    float *loss = nullptr;
    int *bad = nullptr;
    float *shift = nullptr, *scale = nullptr, *rmse = nullptr;
    uint8_t *logm = nullptr;
    float factor = 3.0f;
    int have_transform = 0, have_rmse = 0;
    int64_t t = 0;
    uint64_t launches = 0;
    int report_tc_timeout = 0;  // cpm_mlp_report_next_tc_timeout
    char err[256]{};
};

namespace {

int fail(cpm_mlp *h, int code, const char *msg)
{
    if (h) snprintf(h->err, sizeof h->err, "%s", msg);
    return code;
}

// Message of the calling thread's last failed cpm_mlp_create (no handle exists then).
thread_local char g_create_err[256] = "";

int create_fail(int code, const char *msg)
{
    snprintf(g_create_err, sizeof g_create_err, "%s", msg);
    return code;
}

int cuda_check(cpm_mlp *h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CPM_MLP_OK;
    if (h) snprintf(h->err, sizeof h->err, "%s: %s", what, cudaGetErrorString(e));
    return CPM_MLP_E_CUDA;
}

template <typename T>
int dalloc(cpm_mlp *h, T **p, int64_t n)
{
    if (n <= 0) n = 1;
    return cuda_check(h, cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * (size_t)n), "cudaMalloc");
}

void release(cpm_mlp *h)
{
    void *ptrs[] = {h->w,     h->g,     h->m,    h->v,    h->wb,    h->xb,    h->yb,   h->out,  h->dP,
                    h->dZ[0], h->dZ[1], h->loss, h->bad, h->shift, h->scale, h->rmse, h->logm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < CPM_MLP_MAX_LAYERS; ++l) {
        if (h->H[l]) cudaFree(h->H[l]);
        if (h->Z[l]) cudaFree(h->Z[l]);
    }
}

// forward over `rows` gathered rows (xb); keep_z stores pre-activations for the backward pass
int forward(cpm_mlp *h, int rows, bool keep_z)
{
    const int L = h->n_layers;
    for (int l = 0; l < L; ++l) {
        GemmArgs a{};
        a.M = rows;
        a.N = h->out_dim[l];
        a.K = h->in_dim[l];
        a.A = l == 0 ? h->xb : h->H[l - 1];
        a.lda = h->in_dim[l];
        a.sa = l == 0 ? 0 : (int64_t)rows * h->in_dim[l];
        a.B = h->wb + h->off_w[l];
        a.ldb = h->in_dim[l];
        a.sb = h->P;
        a.bias = h->w + h->off_b[l];
        a.sbias = h->P;
        a.ldc = h->out_dim[l];
        a.sc = (int64_t)rows * h->out_dim[l];
        if (l < L - 1) {
            a.C = h->H[l];
            a.c_f32 = 0;
            a.epi = CPM_MLP_EPI_GELU;
            a.Z = keep_z ? h->Z[l] : nullptr;
            a.ldz = a.ldc;
            a.sz = a.sc;
        } else {
            a.C = h->out;
            a.c_f32 = 1;
            a.epi = CPM_MLP_EPI_NONE;
        }
        const int rc = launch_gemm(0, 1, a, h->sh.n_members, h->st, h->bad + 1, true, &h->report_tc_timeout);
        if (rc) return fail(h, rc, "forward gemm launch failed");
        ++h->launches;
    }
    return CPM_MLP_OK;
}

// loss and gradients of the gathered batch (xb, yb) into h->g and h->loss
int grads(cpm_mlp *h, int rows)
{
    const int L = h->n_layers, E = h->sh.n_members, no = h->sh.n_out;
    int rc = forward(h, rows, true);
    if (rc) return rc;
    if ((rc = cuda_check(h, cudaMemsetAsync(h->loss, 0, sizeof(float) * E, h->st), "memset loss"))) return rc;
    const int64_t count = (int64_t)rows * no;
    const unsigned gx = (unsigned)((count + 255) / 256 < 128 ? (count + 255) / 256 : 128);
    mse_kernel<<<dim3(gx, E), 256, 0, h->st>>>(count, h->out, count, h->yb, 0, h->dP, h->loss);
    ++h->launches;
    const __nv_bfloat16 *dz = h->dP;
    int cur = 0;
    for (int l = L - 1; l >= 0; --l) {
        const int fo = h->out_dim[l], fi = h->in_dim[l];
        // dW_l = dZ_l^T In_l
        GemmArgs a{};
        a.M = fo;
        a.N = fi;
        a.K = rows;
        a.A = dz;
        a.lda = fo;
        a.sa = (int64_t)rows * fo;
        a.B = l == 0 ? h->xb : h->H[l - 1];
        a.ldb = fi;
        a.sb = l == 0 ? 0 : (int64_t)rows * fi;
        a.C = h->g + h->off_w[l];
        a.c_f32 = 1;
        a.ldc = fi;
        a.sc = h->P;
        a.epi = CPM_MLP_EPI_NONE;
        if ((rc = launch_gemm(1, 0, a, E, h->st))) return fail(h, rc, "weight-gradient gemm launch failed");
        ++h->launches;
        bias_grad_kernel<<<dim3((fo + 31) / 32, 1, E), 256, 0, h->st>>>(rows, fo, dz, fo, (int64_t)rows * fo,
                                                                         h->g + h->off_b[l], h->P);
        ++h->launches;
        if (l > 0) {
            // dZ_{l-1} = (dZ_l W_l) * GELU'(Z_{l-1})
            GemmArgs b{};
            b.M = rows;
            b.N = fi;
            b.K = fo;
            b.A = dz;
            b.lda = fo;
            b.sa = (int64_t)rows * fo;
            b.B = h->wb + h->off_w[l];
            b.ldb = fi;
            b.sb = h->P;
            b.C = h->dZ[cur];
            b.c_f32 = 0;
            b.ldc = fi;
            b.sc = (int64_t)rows * fi;
            b.epi = CPM_MLP_EPI_DGELU;
            b.Z = h->Z[l - 1];
            b.ldz = fi;
            b.sz = (int64_t)rows * fi;
            if ((rc = launch_gemm(0, 0, b, E, h->st))) return fail(h, rc, "input-gradient gemm launch failed");
            ++h->launches;
            dz = h->dZ[cur];
            cur ^= 1;
        }
    }
    return cuda_check(h, cudaPeekAtLastError(), "gradient kernels");
}

int gather(cpm_mlp *h, const float *X, const float *Y, const int32_t *order, int64_t off, int64_t n_total, int rows)
{
    if (rows <= 0) return CPM_MLP_OK;
    gather_kernel<<<(rows + 127) / 128, 128, 0, h->st>>>(rows, h->sh.n_in, h->sh.n_out, X, Y, order, off, n_total,
                                                          h->xb, h->yb, h->bad);
    ++h->launches;
    return cuda_check(h, cudaPeekAtLastError(), "gather");
}

// flags: [0] a row index outside the data, [1] a tensor-core wait that timed out
int check_bad(cpm_mlp *h)
{
    int bad[2] = {0, 0};
    int rc = cuda_check(h, cudaMemcpyAsync(bad, h->bad, sizeof bad, cudaMemcpyDeviceToHost, h->st), "read flag");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "sync");
    if (rc) return rc;
    if (bad[0] || bad[1]) {
        cudaMemsetAsync(h->bad, 0, sizeof bad, h->st);
        if (bad[1]) return fail(h, CPM_MLP_E_CUDA, "tensor-core accumulator wait timed out");
        return fail(h, CPM_MLP_E_INVALID, "row index out of range in order[]");
    }
    return CPM_MLP_OK;
}

}  // namespace

extern "C" {

int64_t cpm_mlp_param_count(const cpm_mlp_shape *s)
{
    if (!s || s->n_in < 1 || s->width < 1 || s->n_hidden < 1 || s->n_out < 1 || s->n_hidden + 1 > CPM_MLP_MAX_LAYERS)
        return -1;
    int64_t p = (int64_t)s->width * s->n_in + s->width;
    p += (int64_t)(s->n_hidden - 1) * ((int64_t)s->width * s->width + s->width);
    p += (int64_t)s->n_out * s->width + s->n_out;
    return p;
}

int cpm_mlp_create(const cpm_mlp_shape *shape, const float *init_params, void *cuda_stream, cpm_mlp **out)
{
    if (!shape || !init_params || !out) return create_fail(CPM_MLP_E_INVALID, "shape, init_params and out are required");
    *out = nullptr;
    const int64_t P = cpm_mlp_param_count(shape);
    if (P < 0 || shape->n_members < 1 || shape->n_members > 64 || shape->max_rows < 1 || shape->width % 8 ||
        shape->max_rows > (1 << 22))
        return create_fail(CPM_MLP_E_INVALID,
                           "invalid shape (members 1..64, width a multiple of 8, hidden layers 1..15, rows 1..2^22)");
    cpm_mlp *h = new (std::nothrow) cpm_mlp();
    if (!h) return create_fail(CPM_MLP_E_NOMEM, "host allocation failed");
    h->sh = *shape;
    h->st = (cudaStream_t)cuda_stream;
    h->n_layers = shape->n_hidden + 1;
    int64_t off = 0;
    for (int l = 0; l < h->n_layers; ++l) {
        h->in_dim[l] = l == 0 ? shape->n_in : shape->width;
        h->out_dim[l] = l == h->n_layers - 1 ? shape->n_out : shape->width;
        h->off_w[l] = off;
        off += (int64_t)h->in_dim[l] * h->out_dim[l];
        h->off_b[l] = off;
        off += h->out_dim[l];
    }
    h->P = P;
    const int E = shape->n_members, R = shape->max_rows, W = shape->width;
    const int64_t nP = (int64_t)E * P;
    int rc = 0;
    rc |= dalloc(h, &h->w, nP) | dalloc(h, &h->g, nP) | dalloc(h, &h->m, nP) | dalloc(h, &h->v, nP);
    rc |= dalloc(h, &h->wb, nP) | dalloc(h, &h->xb, (int64_t)R * shape->n_in) |
          dalloc(h, &h->yb, (int64_t)R * shape->n_out);
    for (int l = 0; l < shape->n_hidden; ++l)
        rc |= dalloc(h, &h->H[l], (int64_t)E * R * W) | dalloc(h, &h->Z[l], (int64_t)E * R * W);
    rc |= dalloc(h, &h->out, (int64_t)E * R * shape->n_out) | dalloc(h, &h->dP, (int64_t)E * R * shape->n_out);
    rc |= dalloc(h, &h->dZ[0], (int64_t)E * R * W) | dalloc(h, &h->dZ[1], (int64_t)E * R * W);
    rc |= dalloc(h, &h->loss, E) | dalloc(h, &h->bad, 2);
    rc |= dalloc(h, &h->shift, shape->n_out) | dalloc(h, &h->scale, shape->n_out) | dalloc(h, &h->rmse, shape->n_out);
    rc |= dalloc(h, &h->logm, shape->n_out);
    if (rc) {
        release(h);
        delete h;
        return create_fail(CPM_MLP_E_NOMEM, "device allocation failed");
    }
    if (cpm_mlp_set_params(h, init_params) != CPM_MLP_OK ||
        cudaMemsetAsync(h->bad, 0, 2 * sizeof(int), h->st) != cudaSuccess) {
        create_fail(CPM_MLP_E_CUDA, h->err[0] ? h->err : "initial upload failed");
        release(h);
        delete h;
        return CPM_MLP_E_CUDA;
    }
    *out = h;
    return CPM_MLP_OK;
}

int cpm_mlp_set_params(cpm_mlp *h, const float *params)
{
    if (!h || !params) return CPM_MLP_E_INVALID;
    const int64_t n = (int64_t)h->sh.n_members * h->P;
    int rc = cuda_check(h, cudaMemcpyAsync(h->w, params, sizeof(float) * n, cudaMemcpyHostToDevice, h->st), "upload");
    if (!rc) rc = cuda_check(h, cudaMemsetAsync(h->m, 0, sizeof(float) * n, h->st), "memset m");
    if (!rc) rc = cuda_check(h, cudaMemsetAsync(h->v, 0, sizeof(float) * n, h->st), "memset v");
    if (rc) return rc;
    cast_kernel<<<grid1(n), 256, 0, h->st>>>(n, h->w, h->wb);
    ++h->launches;
    h->t = 0;
    rc = cuda_check(h, cudaPeekAtLastError(), "cast");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "sync");
    return rc;
}

int cpm_mlp_get_params(cpm_mlp *h, float *params)
{
    if (!h || !params) return CPM_MLP_E_INVALID;
    const int64_t n = (int64_t)h->sh.n_members * h->P;
    int rc = cuda_check(h, cudaMemcpyAsync(params, h->w, sizeof(float) * n, cudaMemcpyDeviceToHost, h->st), "download");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "sync");
    return rc;
}

int cpm_mlp_grads(cpm_mlp *h, const float *X, const float *Y, int64_t n_total, const int32_t *order, int64_t offset,
                  int32_t rows, float *grads_out, float *loss_out)
{
    if (!h || !X || !Y || rows < 1 || rows > h->sh.max_rows || offset < 0 || n_total < 1) return CPM_MLP_E_INVALID;
    if (!order && offset + rows > n_total) return fail(h, CPM_MLP_E_INVALID, "rows past the end of the data");
    int rc = gather(h, X, Y, order, offset, n_total, rows);
    if (!rc) rc = grads(h, rows);
    if (!rc && grads_out)
        rc = cuda_check(h, cudaMemcpyAsync(grads_out, h->g, sizeof(float) * h->sh.n_members * h->P,
                                           cudaMemcpyDeviceToDevice, h->st),
                        "copy grads");
    if (!rc && loss_out)
        rc = cuda_check(h, cudaMemcpyAsync(loss_out, h->loss, sizeof(float) * h->sh.n_members,
                                           cudaMemcpyDeviceToDevice, h->st),
                        "copy loss");
    if (!rc) rc = check_bad(h);
    return rc;
}

int cpm_mlp_train(cpm_mlp *h, const float *X, const float *Y, int64_t n_total, const int32_t *order, int64_t n_order,
                  int32_t batch_rows, float lr, float beta1, float beta2, float eps, float *loss_trace)
{
    if (!h || !X || !Y || batch_rows < 1 || batch_rows > h->sh.max_rows || n_total < 1 || n_order < 0 ||
        !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return CPM_MLP_E_INVALID;
    if (!order && n_order > n_total) return fail(h, CPM_MLP_E_INVALID, "n_order > n_total without an order");
    const int64_t nP = (int64_t)h->sh.n_members * h->P;
    const int64_t steps = n_order / batch_rows;
    for (int64_t s = 0; s < steps; ++s) {
        int rc = gather(h, X, Y, order, s * batch_rows, n_total, batch_rows);
        if (!rc) rc = grads(h, batch_rows);
        if (rc) return rc;
        ++h->t;
        const float c1 = 1.0f - powf(beta1, (float)h->t), c2 = 1.0f - powf(beta2, (float)h->t);
        adam_kernel<<<grid1(nP), 256, 0, h->st>>>(nP, h->w, h->wb, h->g, h->m, h->v, lr, beta1, beta2, eps, c1, c2);
        ++h->launches;
        if (loss_trace) {
            rc = cuda_check(h, cudaMemcpyAsync(loss_trace + s * h->sh.n_members, h->loss,
                                               sizeof(float) * h->sh.n_members, cudaMemcpyDeviceToDevice, h->st),
                            "copy loss");
            if (rc) return rc;
        }
    }
    if (int rc = cuda_check(h, cudaPeekAtLastError(), "train kernels")) return rc;
    return check_bad(h);
}

int cpm_mlp_forward(cpm_mlp *h, const float *X, int64_t n_rows, float *out)
{
    if (!h || n_rows < 0 || (n_rows > 0 && (!X || !out))) return CPM_MLP_E_INVALID;
    const int E = h->sh.n_members, no = h->sh.n_out;
    for (int64_t r0 = 0; r0 < n_rows; r0 += h->sh.max_rows) {
        const int rows = (int)(n_rows - r0 < h->sh.max_rows ? n_rows - r0 : h->sh.max_rows);
        int rc = gather(h, X, nullptr, nullptr, r0, n_rows, rows);
        if (!rc) rc = forward(h, rows, false);
        for (int e = 0; !rc && e < E; ++e)
            rc = cuda_check(h, cudaMemcpyAsync(out + ((int64_t)e * n_rows + r0) * no, h->out + (int64_t)e * rows * no,
                                               sizeof(float) * rows * no, cudaMemcpyDeviceToDevice, h->st),
                            "copy out");
        if (rc) return rc;
    }
    return check_bad(h);
}

int cpm_mlp_set_output_transform(cpm_mlp *h, const float *shift, const float *scale, const uint8_t *log_mask,
                                 const float *val_rmse, float factor)
{
    if (!h || !shift || !scale || !log_mask || !(factor >= 0.0f)) return CPM_MLP_E_INVALID;
    const int no = h->sh.n_out;
    int rc = cuda_check(h, cudaMemcpyAsync(h->shift, shift, sizeof(float) * no, cudaMemcpyHostToDevice, h->st), "upload");
    if (!rc)
        rc = cuda_check(h, cudaMemcpyAsync(h->scale, scale, sizeof(float) * no, cudaMemcpyHostToDevice, h->st), "upload");
    if (!rc) rc = cuda_check(h, cudaMemcpyAsync(h->logm, log_mask, no, cudaMemcpyHostToDevice, h->st), "upload");
    if (!rc && val_rmse)
        rc = cuda_check(h, cudaMemcpyAsync(h->rmse, val_rmse, sizeof(float) * no, cudaMemcpyHostToDevice, h->st),
                        "upload");
    if (!rc) rc = cuda_check(h, cudaStreamSynchronize(h->st), "sync");
    if (rc) return rc;
    h->factor = factor;
    h->have_transform = 1;
    h->have_rmse = val_rmse != nullptr;
    return CPM_MLP_OK;
}

int cpm_mlp_predict(cpm_mlp *h, const float *X, int64_t n_rows, float *mean_out, float *std_out, uint8_t *fallback_out)
{
    if (!h || n_rows < 0 || (n_rows > 0 && !X)) return CPM_MLP_E_INVALID;
    if (!h->have_transform) return fail(h, CPM_MLP_E_STATE, "cpm_mlp_set_output_transform has not been called");
    if (fallback_out && !h->have_rmse) return fail(h, CPM_MLP_E_STATE, "no validation RMSE for the fallback rule");
    const int E = h->sh.n_members, no = h->sh.n_out;
    for (int64_t r0 = 0; r0 < n_rows; r0 += h->sh.max_rows) {
        const int rows = (int)(n_rows - r0 < h->sh.max_rows ? n_rows - r0 : h->sh.max_rows);
        int rc = gather(h, X, nullptr, nullptr, r0, n_rows, rows);
        if (!rc) rc = forward(h, rows, false);
        if (rc) return rc;
        predict_kernel<<<(rows + 127) / 128, 128, 0, h->st>>>(
            rows, E, no, h->out, (int64_t)rows * no, h->shift, h->scale, h->logm, h->have_rmse ? h->rmse : nullptr,
            h->factor, mean_out ? mean_out + r0 * no : nullptr, std_out ? std_out + r0 * no : nullptr,
            fallback_out ? fallback_out + r0 : nullptr);
        ++h->launches;
    }
    if (int rc = cuda_check(h, cudaPeekAtLastError(), "predict")) return rc;
    return check_bad(h);
}

uint64_t cpm_mlp_kernel_launches(const cpm_mlp *h) { return h ? h->launches : 0; }

const char *cpm_mlp_last_error(const cpm_mlp *h) { return h ? h->err : g_create_err; }

int cpm_mlp_report_next_tc_timeout(cpm_mlp *h)
{
    if (!h) return CPM_MLP_E_INVALID;
    h->report_tc_timeout = 1;
    return CPM_MLP_OK;
}

int cpm_mlp_destroy(cpm_mlp *h)
{
    if (!h) return CPM_MLP_E_INVALID;
    cudaStreamSynchronize(h->st);
    release(h);
    delete h;
    return CPM_MLP_OK;
}

int cpm_mlp_gemm(int trans_a, int trans_b, int m, int n, int k, int batch, const void *A, int64_t lda,
                 int64_t stride_a, const void *B, int64_t ldb, int64_t stride_b, const float *bias,
                 int64_t stride_bias, void *C, int c_is_f32, int64_t ldc, int64_t stride_c, float *Z, int64_t ldz,
                 int64_t stride_z, int epilogue, void *cuda_stream)
{
    if (m < 0 || n < 0 || k < 1 || batch < 1 || !A || !B || !C) return CPM_MLP_E_INVALID;
    if (epilogue < CPM_MLP_EPI_NONE || epilogue > CPM_MLP_EPI_DGELU || (epilogue == CPM_MLP_EPI_DGELU && !Z))
        return CPM_MLP_E_INVALID;
    GemmArgs a{};
    a.M = m;
    a.N = n;
    a.K = k;
    a.A = static_cast<const __nv_bfloat16 *>(A);
    a.lda = lda;
    a.sa = stride_a;
    a.B = static_cast<const __nv_bfloat16 *>(B);
    a.ldb = ldb;
    a.sb = stride_b;
    a.bias = bias;
    a.sbias = stride_bias;
    a.C = C;
    a.c_f32 = c_is_f32;
    a.ldc = ldc;
    a.sc = stride_c;
    a.Z = Z;
    a.ldz = ldz;
    a.sz = stride_z;
    a.epi = epilogue;
    return launch_gemm(trans_a, trans_b, a, batch, (cudaStream_t)cuda_stream);
}

}  // extern "C"
