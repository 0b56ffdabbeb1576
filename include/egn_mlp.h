/*
 * egn_mlp.h -- C ABI of the kernels of the MLP surrogate of the integrator.
 *
 * The surrogate maps per-channel features of a link to eta [dB] with a
 * multilayer perceptron trained on the integrator's outputs (egn_nli_eta).  The
 * paper itself evaluates the model; surrogates are one of the fast alternatives
 * its introduction weighs against it.  These entry points are the device
 * kernels of its training and inference: BF16 GEMMs on the tensor cores
 * (tcgen05, accumulation in tensor memory, FP32 accumulate) with fused
 * epilogues, and the small FP32 kernels around them.
 *
 * Conventions: matrices are row-major; "BF16" buffers hold __nv_bfloat16;
 * every pointer is a device pointer; every call is asynchronous on `stream`
 * (NULL = legacy default stream) and returns EGN_E_INVALID_ARG for bad shapes
 * or pointers before launching anything.  err_dev is a device int that a
 * kernel sets non-zero if one of its bounded waits runs out (the caller clears
 * it and reads it back); the result is then undefined.
 */
#ifndef EGN_MLP_H
#define EGN_MLP_H

#include "egn.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
    EGN_MLP_EPI_BIAS_RELU = 0, /* out BF16 [m][n] = max(acc + bias[n], 0) */
    EGN_MLP_EPI_BIAS = 1,      /* out BF16 [m][n] = acc + bias[n] */
    EGN_MLP_EPI_F32 = 2,       /* out FP32 [splits][m][n] = partial acc of each k split */
    EGN_MLP_EPI_RELU_GRAD = 3, /* out BF16 [m][n] = acc where aux BF16 [m][n] > 0, else 0 */
    EGN_MLP_EPI_BIAS_GELU = 4, /* aux BF16 [m][n] = z = acc + bias[n] (written: the pre-activation,
                                  kept for the backward pass); out BF16 [m][n] = GELU(z) = z Phi(z),
                                  Phi the standard normal distribution function, of z as stored */
    EGN_MLP_EPI_GELU_GRAD = 5  /* out BF16 [m][n] = acc * GELU'(aux), aux BF16 [m][n] the stored
                                  pre-activation; GELU'(z) = Phi(z) + z phi(z) */
};

/* D = A B^T: A BF16 [m][k], B BF16 [n][k], both with k contiguous; k a
 * multiple of 64, n a multiple of 32, m >= 1; A, B, out 16-byte aligned.
 * splits > 1 divides the k range over that many CTA layers (EGN_MLP_EPI_F32
 * only; sum the slabs with egn_mlp_reduce_splits). */
egn_status egn_mlp_gemm(int m, int n, int k, int splits, const void* a, const void* b, int epilogue,
                        const float* bias, const void* aux, void* out, int* err_dev, void* stream);

/* out[i] = sum over s = 0 .. splits-1 of part[s * count + i], in that order. */
egn_status egn_mlp_reduce_splits(const float* part, int splits, long long count, float* out, void* stream);

/* out BF16 [cols][rows_pad] = in BF16 [rows][cols] transposed, zero for the
 * padding rows rows .. rows_pad-1. */
egn_status egn_mlp_transpose(const void* in, int rows, int cols, int rows_pad, void* out, void* stream);

/* out[c] = sum over r of in BF16 [rows][cols] (fixed order). */
egn_status egn_mlp_colsum(const void* in, int rows, int cols, float* out, void* stream);

/* Output layer and loss.  y[r] = sum_j h[r][j] w[j] + b (h BF16 [rows][hid],
 * hid a multiple of 32, w FP32 [hid], b FP32 [1]).  With target != NULL also:
 * loss[0] = sum_r mask[r] (y[r] - target[r])^2 / sum_r mask[r]; g[r] =
 * dloss/dy[r]; dh BF16 [rows][hid] = g[r] w[j] where h[r][j] > 0 (the ReLU of
 * the layer below), dw[j] = sum_r g[r] h[r][j], db[0] = sum_r g[r] (fixed-order
 * sums). */
egn_status egn_mlp_head(const void* h, int rows, int hid, const float* w, const float* b, float* y,
                        const float* target, const float* mask, float* loss, float* g, void* dh, float* dw,
                        float* db, void* stream);

/* Multi-output layer and loss, for a network whose last GEMM wrote acc FP32
 * [rows][n_pad] (EGN_MLP_EPI_F32) with n_out <= n_pad live columns:
 * y FP32 [rows][n_out] = acc[r][j] + b[j].  With target != NULL (FP32
 * [rows][n_out]) and mask (FP32 [rows]) also: loss[0] = sum_r mask[r] sum_j
 * (y[r][j] - target[r][j])^2 / (n_out sum_r mask[r]); g BF16 [rows_pad][n_pad] =
 * dloss/dy, zero in the padding rows (r >= rows) and columns (j >= n_out);
 * db FP32 [n_out] = sum over r of dloss/dy[r][j] (fixed-order sums). */
egn_status egn_mlp_outputs(const float* acc, int rows, int rows_pad, int n_out, int n_pad, const float* b, float* y,
                           const float* target, const float* mask, float* loss, void* g, float* db, void* stream);

/* Adam step on FP32 master weights w[n] with gradient g, moments m and v
 * (bias-corrected for step t >= 1); then w_bf16 [n] = w and, if wt_bf16 is
 * not NULL, wt_bf16 = the BF16 transpose of w viewed as [rows][cols]. */
egn_status egn_mlp_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float beta1, float beta2,
                        float eps, int t, void* w_bf16, void* wt_bf16, int rows, int cols, void* stream);

/* out BF16 [n] = in FP32 [n] rounded to nearest even. */
egn_status egn_mlp_cast(const float* in, long long n, void* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif
