/* Learned form of the fast solve: a multilayer perceptron that predicts a fast
 * stage's increment from the cell state, and whose prediction serves as the Newton
 * initial guess of the stage (the fast solve still decides every result, and falls
 * back to its plain start wherever Newton does not converge from the guess).
 *
 * The paper integrates the fast partition with plain Runge-Kutta methods and has
 * no learned component; these calls implement the learned form named for this
 * library: a network with SiLU hidden layers and a linear output,
 *   a_0 = x,  z_l = a_{l-1} W_l^T + b_l,  a_l = silu(z_l) = z_l / (1 + e^{-z_l}),
 *   y = z_L,
 * bfloat16 weights and GEMM inputs, FP32 accumulation (tensor-core tcgen05 MMA),
 * FP32 master parameters trained with Adam (Kingma & Ba 2015) on the loss
 *   L = sum_{b,j} m_j (y_bj - t_bj)^2 / (2 B).
 * All device pointers are caller-owned unless stated; all calls are stream-ordered
 * and return MRI_* codes (mri.h). */
#ifndef MRI_MLP_H
#define MRI_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "mri.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MRI_MLP_MAX_LAYERS 8

typedef struct mri_mlp mri_mlp;

/* Create a network of n_layers affine layers with sizes dims[0..n_layers]
 * (dims[0] inputs, dims[n_layers] outputs; every size a multiple of 16 in 16..256)
 * for batches of up to batch_max rows.  init_params: host FP32 parameters packed
 * layer by layer as W_l [dims[l+1]][dims[l]] row-major then b_l [dims[l+1]]
 * (mri_mlp_num_params floats), or NULL for zeros.  Allocates device memory (owned
 * by the handle until mri_mlp_free).  Returns MRI_EINVAL for bad sizes,
 * MRI_ECUDA on an allocation or copy failure. */
int mri_mlp_create(const int* dims, int n_layers, int batch_max, const float* init_params, mri_mlp** out);
void mri_mlp_free(mri_mlp* mlp);
long long mri_mlp_num_params(const mri_mlp* mlp);

/* Copy the FP32 master parameters to host_out (if not NULL), then replace them
 * with host_in (if not NULL).  Synchronous. */
int mri_mlp_params(mri_mlp* mlp, float* host_out, const float* host_in);

/* y [B][dims[L]] = network(x [B][dims[0]]), x and y FP32 device arrays, B <=
 * batch_max.  Keeps the layer activations for a following mri_mlp_grad. */
int mri_mlp_forward(mri_mlp* mlp, const float* x, int B, float* y, void* stream);

/* Forward pass on x, then the gradient of L with respect to every parameter for
 * targets t [B][dims[L]] and output weights w_out [dims[L]] (FP32 device arrays).
 * y receives the outputs; loss (device float, nullable) receives L.  The gradient
 * stays in the handle for mri_mlp_adam and mri_mlp_grad_copy. */
int mri_mlp_grad(mri_mlp* mlp, const float* x, const float* t, const float* w_out, int B, float* y, float* loss,
                 void* stream);

/* Copy the last gradient (packed like the parameters) to the device array dst. */
int mri_mlp_grad_copy(mri_mlp* mlp, float* dst, void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for step >= 1)
 * with learning rate lr on the last gradient; refreshes the bfloat16 weights. */
int mri_mlp_adam(mri_mlp* mlp, float lr, int step, void* stream);

/* MRI_ETIMEOUT if a tensor-core wait of any earlier call ran out (the results of
 * that call are then invalid), else MRI_OK.  Synchronous. */
int mri_mlp_status(mri_mlp* mlp);

/* ---- data of the learned form --------------------------------------------
 * Network inputs for ncell cells of n = Ns + 1 unknowns (y [ncell][n] FP64, T last),
 * pressure p [ncell] and the stage's forcing phi [ncell][K][n] (nullable when K = 0):
 *   raw[0..Ns)      log10(max(Y_k, 1e-30))
 *   raw[Ns]         T / 1000 K
 *   raw[Ns+1]       ln(p / 101325 Pa)
 *   raw[Ns+2]       log10(Hstage / 1 s)
 *   raw[Ns+3+e]     Hstage sum_k phi[c][k][e] / (k + 1)   (the forcing's increment
 *                   over the stage, e < n)
 * x[c][f] = (raw[f] - mean[f]) * inv_std[f] for f < 2n + 2, 0 up to ld_x (FP32). */
int mri_learned_features(const double* y, const double* p, const double* phi, int K, int ncell, int n,
                         double Hstage, const float* mean, const float* inv_std, float* x, int ld_x, void* stream);

/* Training targets: the states y_seq [ncell][G][n] at the ends of a stage's G
 * substeps relative to the stage input y_in [ncell][n], standardised per output:
 * t[c][g n + j] = ((y_seq[c][g][j] - y_in[c][j]) - tmean[g n + j]) * tinv_std[g n + j]
 * for g n + j < G n, 0 up to ld_t. */
int mri_learned_targets(const double* y_in, const double* y_seq, int G, int ncell, int n, const float* tmean,
                        const float* tinv_std, float* t, int ld_t, void* stream);

/* The predicted substep-end states for mri_stage_fast_guided from the network's
 * outputs yhat [ncell][ld_yhat]:
 * guess[c][g][j] = y_in[c][j] + tmean[g n + j] + tstd[g n + j] * yhat[c][g n + j]. */
int mri_learned_guess(const double* y_in, const float* yhat, int ld_yhat, int G, int ncell, int n,
                      const float* tmean, const float* tstd, double* guess, void* stream);

/* The network's substep-size prediction: output column col of yhat [ncell][ld_yhat]
 * holds the standardised log2 of a cell's step relative to the uniform substep;
 * step_exp[c] = round(tmean + tstd * yhat[c][col]) clamped to [kmin, kmax], the
 * first-step exponent of mri_stage_fast_guided (int8, device). */
int mri_learned_step_exp(const float* yhat, int ld_yhat, int col, int ncell, float tmean, float tstd, int kmin,
                         int kmax, int8_t* step_exp, void* stream);

/* Standardisation constants of a data matrix (the network's raw inputs or targets),
 * computed on the device: X [rows][ld] FP32, for each column f < cols the mean and the
 * population standard deviation over the rows (sums in FP64, over row chunks added in
 * a fixed order, so the result is deterministic); a deviation below floor_sd (a
 * constant column) is replaced by 1.  mean, inv_std = 1 / sd and sd (nullable) are
 * FP32 device arrays of cols values.  workspace: device buffer of
 * mri_learned_moments_workspace_size(cols) bytes (MRI_ENOMEM if smaller). */
size_t mri_learned_moments_workspace_size(int cols);
int mri_learned_moments(const float* X, long long rows, int cols, int ld, float floor_sd, float* mean,
                        float* inv_std, float* sd, void* workspace, size_t workspace_bytes, void* stream);

/* Standardised and reordered rows: out [rows_out][ld_out] with
 * out[i][f] = (X[perm[i]][f] - mean[f]) * inv_std[f] for f < used and 0 for
 * used <= f < ld_out; perm (device int32 [rows_out], nullable: identity) is the
 * shuffle of a training epoch, drawn by the caller. */
int mri_learned_standardise(const float* X, int ld, const int32_t* perm, long long rows_out, int used,
                            const float* mean, const float* inv_std, float* out, int ld_out, void* stream);

/* Targets of the substep-size network from an adaptive solve's per-cell counters:
 * k[c] = log2(n_sub / max(accepted[c * stride], 1)), the log2 of the cell's mean
 * accepted step relative to the uniform substep Hstage / n_sub (accepted: device
 * int32, e.g. cell_stats with stride 4; k: device FP32 [ncell]). */
int mri_learned_step_targets(const int32_t* accepted, int stride, int ncell, int n_sub, float* k, void* stream);

/* The GEMM the network is built on, exposed for testing:
 * C [M][ldc] (FP32) = A [M][lda] * B [N][ldb]^T over K, A and B bfloat16 bit
 * patterns (uint16) with K contiguous; N a multiple of 16 in 16..256, K, lda and
 * ldb multiples of 8.  err: device int set to 1 if a tensor-core wait ran out. */
int mri_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K, float* C, int ldc, int* err,
                  void* stream);

#ifdef __cplusplus
}
#endif

#endif
