/*
 * libelmddm: the learned interface warm start.
 *
 * A small multilayer perceptron y = W3^T g(W2^T g(W1^T x + b1) + b2) + b3 with
 * g = GELU (exact, 0.5 z (1 + erf(z / sqrt 2))), trained by the library's own forward,
 * backward and Adam kernels: FP32 parameters and activations, the layers' products on the
 * tensor cores at FP32 accuracy (three TF32 products of a hi/lo split of each operand).  It maps the coefficients of a source term to the
 * interface variable u_Gamma of the Schur system of Eq. (3.5), whose prediction starts
 * the conjugate-gradient interface solve (elm_ddm_solve_pcg).  The paper has no
 * counterpart: it is an extension of its iterative interface solve (Section 4).
 *
 * Conventions: every array is a device pointer, FP32, row-major; x [batch][d_in],
 * y and targets [batch][d_out].  Parameters are one contiguous block in the order
 * W1 [d_in][d_h], b1 [d_h], W2 [d_h][d_h], b2 [d_h], W3 [d_h][d_out], b3 [d_out];
 * gradients use the same layout.  The loss is the mean squared error
 * L = sum (y - t)^2 / (batch * d_out).  Calls are stream-ordered on the stream given
 * at creation; the handle owns all of its workspace.  Return codes are the
 * ELM_DDM_* codes of elm_ddm.h (ERR_ARG for a bad argument, ERR_CUDA, ERR_OOM).
 */
#ifndef ELM_MLP_H
#define ELM_MLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct elm_mlp elm_mlp;

/* Glorot-uniform weights from a seeded generator, zero biases; batch <= max_batch. */
int elm_mlp_create(int d_in, int d_hidden, int d_out, int max_batch, uint64_t seed, void* stream,
                   elm_mlp** out);
int elm_mlp_param_count(const elm_mlp* m, int64_t* count);
int elm_mlp_get_params(elm_mlp* m, float* dst);
int elm_mlp_set_params(elm_mlp* m, const float* src);
/* Inference: y = f(x). */
int elm_mlp_forward(elm_mlp* m, const float* x, int batch, float* y);
/* Loss (device scalar, may be NULL) and its gradient with respect to every parameter
 * (device, parameter layout, may be NULL), without an update. */
int elm_mlp_gradient(elm_mlp* m, const float* x, const float* target, int batch, float* loss,
                     float* grad);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the loss of this
 * batch; loss (device scalar, may be NULL) receives the loss before the update. */
int elm_mlp_train_step(elm_mlp* m, const float* x, const float* target, int batch, float lr,
                       float* loss);
/* Synchronises the stream; ELM_DDM_ERR_TIMEOUT when a bounded wait of a GEMM kernel gave up
 * since the previous check (the affected outputs are not valid), else ELM_DDM_OK. */
int elm_mlp_check(elm_mlp* m);
int elm_mlp_destroy(elm_mlp* m);
const char* elm_mlp_last_error(const elm_mlp* m);

#ifdef __cplusplus
}
#endif

#endif
