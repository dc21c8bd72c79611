/*
 * cpm_emulator.h -- C ABI of the MLP-ensemble emulator of CPM summary
 * statistics (libcpm_gb300.so).
 *
 * The emulator maps the seven swept parameters of the cellular Potts model
 * (J cell-cell, J cell-medium, lambda_V, lambda_P, lambda_Act, Max_Act, T;
 * the energy terms of Methods Eq. 1, Eq. 3 and Eq. 8) to summary statistics
 * of a run: cell volume and interface statistics, centroid displacement
 * statistics (centroids as in Methods, "Composite variable tracking",
 * Eq. 10), acceptance rate and contact fractions.  The paper itself has no
 * emulator; the network is the project's own.
 *
 * The model is an ensemble of n_members fully connected networks, each
 *     Z_l = H_{l-1} W_l^T + b_l,  H_l = GELU(Z_l)  (n_hidden layers of `width`)
 *     P   = H_{L-1} W_L^T + b_L                    (n_out linear outputs)
 * with GELU(z) = z Phi(z) (Phi the standard normal CDF), trained on the mean
 * squared error over all outputs with Adam (Kingma & Ba 2015):
 *     m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
 *     w <- w - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
 *
 * Arithmetic: FP32 master weights and Adam moments; every GEMM reads BF16
 * operands (weights, activations and back-propagated gradients rounded to
 * BF16) on the tensor cores and accumulates in FP32; biases, GELU, GELU',
 * loss and the optimiser run in FP32.
 *
 * Parameter layout: one flat float array, member after member; within a
 * member, layer after layer, W_l row-major [out][in] followed by b_l [out].
 * cpm_mlp_param_count() gives the per-member length.
 *
 * Pointers: unless stated otherwise, data pointers (X, Y, order, outputs)
 * are DEVICE pointers on the handle's device; initial and read-back
 * parameter arrays and the output transform are HOST pointers.  All work is
 * ordered on the stream given at creation (NULL = legacy default stream);
 * functions that return host-visible results synchronise that stream.
 * The caller keeps ownership of every buffer it passes.
 *
 * Errors: every int-returning function returns CPM_MLP_OK (0) or a negative
 * code; cpm_mlp_last_error() describes the last failure on a handle.  A
 * CUDA error leaves the handle's buffers allocated; destroy it.
 */
#ifndef CPM_EMULATOR_H
#define CPM_EMULATOR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CPM_MLP_OK 0
#define CPM_MLP_E_INVALID (-1) /* bad argument (null pointer, size, range, out-of-range row index) */
#define CPM_MLP_E_NOMEM (-2)   /* device allocation failed */
#define CPM_MLP_E_CUDA (-3)    /* a CUDA call or launch failed */
#define CPM_MLP_E_STATE (-5)   /* call out of order (e.g. predict before set_output_transform) */

#define CPM_MLP_MAX_LAYERS 16

/* GEMM epilogues (cpm_mlp_gemm). */
#define CPM_MLP_EPI_NONE 0  /* C = acc (+ bias) */
#define CPM_MLP_EPI_GELU 1  /* Z = acc + bias (stored if Z != NULL); C = GELU(Z) */
#define CPM_MLP_EPI_DGELU 2 /* C = acc * GELU'(Z), Z read (pre-activation of the layer below) */

typedef struct {
    int32_t n_members; /* ensemble size, 1..64 */
    int32_t n_in;      /* inputs per row (7 swept parameters) */
    int32_t width;     /* hidden width, a multiple of 8 */
    int32_t n_hidden;  /* hidden layers, 1..CPM_MLP_MAX_LAYERS-1 */
    int32_t n_out;     /* outputs per row (16 statistics) */
    int32_t max_rows;  /* rows per internal batch: training batch limit and inference chunk */
} cpm_mlp_shape;

typedef struct cpm_mlp cpm_mlp;

/* Parameters per member, or -1 for an invalid shape. */
int64_t cpm_mlp_param_count(const cpm_mlp_shape *shape);

/* Allocates the ensemble and its work buffers (about
 * n_members * max_rows * width * 16 bytes for activations, pre-activations
 * and gradients) and uploads the initial parameters (host array of
 * n_members * param_count floats; the project draws them from its seeded
 * input generator).  Adam state starts at zero, step 0. */
int cpm_mlp_create(const cpm_mlp_shape *shape, const float *init_params_host, void *cuda_stream, cpm_mlp **out);

/* Replaces the parameters (host array) and resets Adam's moments and step. */
int cpm_mlp_set_params(cpm_mlp *h, const float *params_host);
/* Copies the FP32 master parameters to a host array. */
int cpm_mlp_get_params(cpm_mlp *h, float *params_host);

/* Loss and gradients of one batch without updating the weights.
 * X: [n_total][n_in] f32, Y: [n_total][n_out] f32 (standardised targets);
 * rows taken are order[offset .. offset+rows) (int32 row indices) or, with
 * order == NULL, offset .. offset+rows.  Every member sees the same rows.
 * grads_out (device, may be NULL): n_members * param_count floats in the
 * parameter layout, each the gradient of that member's mean squared error;
 * loss_out (device, may be NULL): n_members floats.  An index outside
 * [0, n_total) returns CPM_MLP_E_INVALID. */
int cpm_mlp_grads(cpm_mlp *h, const float *X, const float *Y, int64_t n_total, const int32_t *order, int64_t offset,
                  int32_t rows, float *grads_out, float *loss_out);

/* floor(n_order / batch_rows) Adam steps over consecutive batches of
 * order[] (or of rows 0.. when order == NULL), batch_rows <= max_rows.
 * loss_trace (device, may be NULL): per step the n_members losses of the
 * batch before its update, [steps][n_members]. */
int cpm_mlp_train(cpm_mlp *h, const float *X, const float *Y, int64_t n_total, const int32_t *order, int64_t n_order,
                  int32_t batch_rows, float lr, float beta1, float beta2, float eps, float *loss_trace);

/* Raw member outputs (standardised units): out[n_members][n_rows][n_out]. */
int cpm_mlp_forward(cpm_mlp *h, const float *X, int64_t n_rows, float *out);

/* Output transform and fallback rule (host arrays of n_out): a statistic is
 * recovered from the ensemble mean mu as y = mu * scale + shift, then
 * exp(y) where log_mask != 0.  val_rmse (may be NULL) is each output's
 * validation RMSE in standardised units; a row falls back to the CPM when
 * any output's ensemble standard deviation exceeds factor * val_rmse. */
int cpm_mlp_set_output_transform(cpm_mlp *h, const float *shift, const float *scale, const uint8_t *log_mask,
                                 const float *val_rmse, float factor);

/* Inference over n_rows query rows X [n_rows][n_in] in chunks of max_rows.
 * mean_out [n_rows][n_out] (statistics in their own units), std_out
 * [n_rows][n_out] (ensemble std, standardised units), fallback_out
 * [n_rows] (1 = ask the CPM); any output may be NULL. */
int cpm_mlp_predict(cpm_mlp *h, const float *X, int64_t n_rows, float *mean_out, float *std_out, uint8_t *fallback_out);

/* Kernels launched by this handle so far. */
uint64_t cpm_mlp_kernel_launches(const cpm_mlp *h);
/* Message of the last failed call on h; with h NULL, of the calling thread's
 * last failed cpm_mlp_create. */
const char *cpm_mlp_last_error(const cpm_mlp *h);
int cpm_mlp_destroy(cpm_mlp *h);

/* Test hook for the failure path of the tensor-core GEMM (the paper has no
 * counterpart).  The GEMM waits for its tensor-core accumulator on an
 * mbarrier with a bounded number of polls; when the bound runs out, the
 * kernel records the timeout, waits (bounded) for the MMAs it issued, frees
 * its tensor memory and returns, and the call that launched it returns
 * CPM_MLP_E_CUDA with the message "tensor-core accumulator wait timed out".
 * A healthy GPU never gets there, so this call arms the handle's next
 * tensor-core GEMM launch to take that path after its wait has completed:
 * the kernel reports the timeout and the handle stays usable for the calls
 * after it.  Returns CPM_MLP_OK, or CPM_MLP_E_INVALID for a NULL handle. */
int cpm_mlp_report_next_tc_timeout(cpm_mlp *h);

/* The batched GEMM behind the network, exposed for tests:
 *   C[z][m][n] = epilogue( sum_k op(A)[m][k] op(B)[k][n] ),  z < batch,
 *   op(A)[m][k] = trans_a ? A[z*stride_a + k*lda + m] : A[z*stride_a + m*lda + k],
 *   op(B)[k][n] = trans_b ? B[z*stride_b + n*ldb + k] : B[z*stride_b + k*ldb + n],
 * A, B bf16; bias f32 [z*stride_bias + n] (may be NULL); C bf16 or f32
 * (c_is_f32) at z*stride_c + m*ldc + n; Z f32 at z*stride_z + m*ldz + n.
 * Stride 0 shares an operand across the batch.  Asynchronous on cuda_stream. */
int cpm_mlp_gemm(int trans_a, int trans_b, int m, int n, int k, int batch, const void *A, int64_t lda,
                 int64_t stride_a, const void *B, int64_t ldb, int64_t stride_b, const float *bias,
                 int64_t stride_bias, void *C, int c_is_f32, int64_t ldc, int64_t stride_c, float *Z, int64_t ldz,
                 int64_t stride_z, int epilogue, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* CPM_EMULATOR_H */
