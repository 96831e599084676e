/*
 * liblbm warm-start network: a multilayer perceptron (SiLU hidden layers,
 * linear output) trained and evaluated on the GPU with BF16 tensor-core
 * matrix products and FP32 accumulation.  It maps the six 0D parameters of a
 * vessel (R_p, C, R_d, E_max, E_min, beat period) to a periodic-state
 * initialisation of the coupled solver.  The paper has no counterpart: the
 * network only chooses the initial state; the solver of include/lbm.h is run
 * from it unchanged and decides the result.
 *
 * Conventions: every call returns an lbm_status (include/lbm.h); host arrays
 * are FP32 and copied; nothing is retained.  Flat parameter layout (shared
 * with any checker): for each layer k = 0..L-1, its weight matrix stored
 * transposed (n_out_k rows of n_in_k values), then its bias (n_out_k).
 */
#ifndef LBM_MLP_H
#define LBM_MLP_H

#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbm_mlp lbm_mlp;

/* n_in in [1, 16] (zero-padded to 16 inside), hidden a multiple of 64,
 * n_hidden >= 1 hidden layers, n_out a multiple of 16, max_batch a multiple
 * of 64.  Parameters start at zero; set them with lbm_mlp_set_params. */
lbm_status lbm_mlp_create(int n_in, int hidden, int n_hidden, int n_out, int max_batch, int device,
                          void *stream, lbm_mlp **out);
int64_t lbm_mlp_num_params(const lbm_mlp *m);
/* FP32 master parameters, n = lbm_mlp_num_params values, flat layout above. */
lbm_status lbm_mlp_set_params(lbm_mlp *m, const float *theta, int64_t n);
lbm_status lbm_mlp_get_params(lbm_mlp *m, float *theta, int64_t n);
/* y (batch x n_out) = network(x (batch x n_in)); batch a multiple of 16, <= max_batch. */
lbm_status lbm_mlp_forward(lbm_mlp *m, const float *x, int batch, float *y);
/* g (num_params) = gradient of sum(y * dy) with respect to the parameters. */
lbm_status lbm_mlp_grad(lbm_mlp *m, const float *x, const float *dy, int batch, float *g);
/* Copies a training set (n rows of n_in inputs and n_out targets) to the device. */
lbm_status lbm_mlp_set_data(lbm_mlp *m, const float *x, const float *t, int n);
/* n_steps Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared
 * error; minibatch s uses the rows order[s*batch .. s*batch+batch) of the
 * training set (host int32 array, n_steps*batch entries, each in [0, n)).
 * losses (host, n_steps) receives the loss of every step (may be NULL). */
lbm_status lbm_mlp_train(lbm_mlp *m, const int32_t *order, int n_steps, int batch, float lr, float *losses);
void lbm_mlp_destroy(lbm_mlp *m);

#ifdef __cplusplus
}
#endif
#endif /* LBM_MLP_H */
