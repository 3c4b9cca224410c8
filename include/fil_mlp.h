/*
 * C ABI of the learned warm start: a per-filament MLP that proposes the next
 * step's unknowns X = (Y_1, u, Lambda) of a 32-segment filament (the initial
 * guess of the implicit step, which the paper extrapolates from past steps,
 * Sec. 3.3). The network and its training are not part of the paper; the
 * plain solve keeps the last word: fil_step starts from whichever of the
 * prediction and the extrapolation has the smaller residual and converges to
 * the same tolerance either way.
 *
 * Network: 800 -> 256 -> 256 -> 256 -> 192, ReLU on the hidden layers, BF16
 * weights and activations on the tensor cores with FP32 accumulation, FP32
 * biases and master weights. Inputs and outputs are normalised per component
 * with stored means and standard deviations.
 *
 * Input (FIL_MLP_IN = 32 x 13 + 192 + 192) of filament i, in its own frame
 * (origin Y_1, axes R(q_1)): per segment n the position R1^T (Y_n - Y_1), the
 * quaternion q_1^* q_n, and the total force and torque R1^T F_n, R1^T T_n
 * acting at the current state (constraint + elastic + external, Sec. 2.5);
 * then, per 3-vector of the filament's unknowns, the extrapolated increment
 * R1^T (X_ex - X^j) (X^j = (Y_1^j, u = 0, Lambda^j), the current state), which
 * carries the velocities a single state does not, and the previous step's
 * correction R1^T (X*_prev - X_ex,prev) (zero until a step was committed since
 * the last fil_set_state / fil_init_straight).
 * Output (FIL_MLP_OUT = 192 = 6N): the correction R1^T (X* - X_ex) of the
 * extrapolated X_0 (X_ex), per 3-vector of the filament's unknowns (Y_1, the
 * Lie-algebra increments u_n with q^{j+1} = exp(u_n) q^j, Lambda); X* is the
 * converged solution of the step. A zero network reproduces the extrapolation.
 *
 * Arrays are FP32, row-major, device memory unless stated. Functions return a
 * fil_status (include/fil.h); they never abort.
 */
#ifndef FIL_MLP_H
#define FIL_MLP_H

#include <stdint.h>

#include "fil.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FIL_MLP_SEG 32
#define FIL_MLP_IN 800
#define FIL_MLP_HIDDEN 256
#define FIL_MLP_OUT 192
/* packed parameter vector: W1 [256 x 800], b1 [256], W2 [256 x 256], b2,
   W3 [256 x 256], b3, W4 [192 x 256], b4 [192] (W row-major, out x in) */
#define FIL_MLP_NPARAM (256 * 800 + 256 + 2 * (256 * 256 + 256) + 192 * 256 + 192)

typedef struct fil_mlp fil_mlp;

/* A network with workspace for batches of up to max_batch rows on `stream`
   (cudaStream_t, NULL = default). Parameters start at zero; normalisation at
   mean 0, std 1. FIL_ENOMEM if the device allocation fails. */
fil_status fil_mlp_create(int64_t max_batch, void *stream, fil_mlp **out);
void fil_mlp_destroy(fil_mlp *m);

/* Packed FP32 parameters (FIL_MLP_NPARAM, host or device memory). set_params
   also resets the Adam moments. */
fil_status fil_mlp_set_params(fil_mlp *m, const float *params);
fil_status fil_mlp_get_params(fil_mlp *m, float *params);

/* Per-component normalisation (host or device, FIL_MLP_IN and FIL_MLP_OUT
   entries; std must be > 0): x_hat = (x - in_mean) / in_std, and the network
   output y_hat maps to y = out_mean + out_std * y_hat. */
fil_status fil_mlp_set_norm(fil_mlp *m, const float *in_mean, const float *in_std,
                            const float *out_mean, const float *out_std);

/* y [batch x 192] = network(x [batch x 800]), raw units. */
fil_status fil_mlp_forward(fil_mlp *m, const float *x, float *y, int64_t batch);

/* Loss L = sum over rows and outputs of (y_hat - t_hat)^2 / (2 batch), with
   t_hat the normalised target, and its gradient with respect to the packed
   parameters (grad: FIL_MLP_NPARAM floats, device). loss: host scalar. */
fil_status fil_mlp_gradients(fil_mlp *m, const float *x, const float *target, int64_t batch,
                             float *grad, float *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the loss above with
   learning rate lr; loss (host, nullable) receives the loss before the step. */
fil_status fil_mlp_train_step(fil_mlp *m, const float *x, const float *target, int64_t batch,
                              float lr, float *loss);

/* ---- the network inside the implicit step ---------------------------------
   Filaments of FIL_MLP_SEG segments get a predicted X_0; others keep the
   extrapolation. */

/* Network inputs at the current state (FIL_MLP_IN floats per filament, device
   array [n_fil x FIL_MLP_IN]; rows of other lengths are zero). The loads F, T
   are those of X = (Y_1, u = 0, Lambda) of the current state. FIL_ESTATE
   inside a step. */
fil_status fil_warm_features(fil_ctx *c, float *feat);

/* Training targets of the step committed last (device [n_fil x FIL_MLP_OUT]):
   R1^T (X* - X_ex) in the frame of the state that step started from.
   FIL_ESTATE unless a step was committed since the last fil_set_state /
   fil_init_straight (and no fil_broyden_begin since). */
fil_status fil_warm_targets(fil_ctx *c, float *targ);

typedef enum {
    FIL_WARM_BEST_OF_TWO = 0,      /* evaluate f at both candidates, keep the smaller ||f||_inf */
    FIL_WARM_PREDICTION_FIRST = 1  /* start from the prediction (if f is finite there) */
} fil_warm_mode;

/* Attach a network (NULL detaches; not owned; its max_batch must be >= n_fil).
   While attached, fil_broyden_begin and fil_step take X_0 from the network's
   prediction or the extrapolation as `mode` says, and fil_step restarts from
   the extrapolation if a start from the prediction fails to converge. The
   convergence criterion is unchanged. */
fil_status fil_warm_attach(fil_ctx *c, fil_mlp *net, int32_t mode);

/* Steps started from the prediction / the extrapolation, and restarts. */
fil_status fil_warm_stats(const fil_ctx *c, int64_t *from_prediction, int64_t *from_extrapolation,
                          int64_t *restarts);

/* Tensor-core GEMM used by the network, exposed for testing:
   C [M x N] (FP32, ldc) = A [M x K] . B [N x K]^T, A and B BF16 bit patterns
   (uint16), row-major with leading dimensions lda, ldb (elements). Device
   memory; N a multiple of 32, K of 64, lda and ldb of 8, ldc of 4; rows and
   leading dimensions 16-byte aligned. Synchronises `stream`; FIL_ECUDA if a
   wait inside the kernel ran out. */
fil_status fil_tc_gemm_bf16(const uint16_t *A, int64_t lda, const uint16_t *B, int64_t ldb,
                            float *C, int64_t ldc, int64_t M, int64_t N, int64_t K,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FIL_MLP_H */
