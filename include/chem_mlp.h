/*
 * chem_mlp.h - learned per-cell cost and initial-step model (C ABI).
 *
 * The paper balances the uneven per-cell chemistry cost across MPI ranks
 * (Methodology, "DLBFoam: Dynamic load balancing") and measures that cost per
 * process (Results, Fig. 4). It has no learned component: this model is an
 * addition. A small MLP is trained on the integrator's own per-cell logs
 * (substeps and first accepted step size, from chem_get_stats) and predicts,
 * for new cells, ln(substeps) and ln(first step). The integrator uses the
 * predictions to order its work queue heaviest-first (option "order" = 1) and to
 * seed the initial step (option "h0" = 1). Its error control judges every step,
 * so results stay within tolerance whatever the model predicts; the
 * starting-step heuristic remains the fallback for non-finite predictions.
 *
 * Network: x = [T/1000, ln p, ln(Y_k + 1e-20)] (K + 2 features, standardised by
 * training-set mean and standard deviation) -> Linear(K+2, 128) -> GELU ->
 * Linear(128, 128) -> GELU -> Linear(128, 2). GEMMs take BF16 operands and
 * accumulate in FP32 (tensor cores); master weights and Adam state are FP32.
 *
 * Pointers are device pointers unless marked host; `stream` as in chem.h.
 */
#ifndef CHEM_MLP_H_
#define CHEM_MLP_H_

#include <stdint.h>

#include "chem.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chem_mlp_s* chem_mlp;

/* New model for n_species species, weights drawn from a seeded uniform
 * (+-1/sqrt(fan_in)) initialisation; normalisation is identity until trained. */
chem_status chem_mlp_create(int32_t n_species, uint64_t seed, chem_mlp* out);
chem_status chem_mlp_destroy(chem_mlp m);

/*
 * Trains on n logged cells: states (T[n], p[n], Y[n][K]) at the START of the
 * logged step, and that step's substeps[n] (int32) and h_first[n] (s). Sets the
 * normalisation from these samples, then runs `epochs` epochs of Adam
 * (lr, beta1 0.9, beta2 0.999, eps 1e-8) over seeded shuffled minibatches of
 * `batch` samples. loss_host (nullable, host, `epochs` floats) receives the mean
 * training loss of each epoch. Synchronises `stream`.
 */
chem_status chem_mlp_train(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                           const int32_t* substeps, const double* h_first, int32_t epochs,
                           int32_t batch, double lr, uint64_t seed, float* loss_host, void* stream);

/* Predictions for n cells: ln_cost[n] and ln_h0[n] (device float, either may be NULL). */
chem_status chem_mlp_predict(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                             float* ln_cost, float* ln_h0, void* stream);

/* Attach (or detach with NULL) the model used by a handle's learned options. */
chem_status chem_mlp_attach(chem_handle h, chem_mlp m);

/*
 * Parameters as one host float vector in the order
 *   mu_x[D], sd_x[D], mu_t[2], sd_t[2], W1[128][D], b1[128], W2[128][128], b2[128],
 *   W3[2][128], b3[2]      (D = K + 2).
 * chem_mlp_get_params writes *n_floats and, when buf is not NULL, the values.
 */
chem_status chem_mlp_get_params(chem_mlp m, float* buf, int64_t* n_floats);
chem_status chem_mlp_set_params(chem_mlp m, const float* buf, int64_t n_floats);

/*
 * One forward + backward pass over n samples with the current parameters and
 * normalisation (no update): loss (host float) and the gradient with respect to
 * W1, b1, W2, b2, W3, b3 (host floats in that order). For gradient checks.
 */
chem_status chem_mlp_gradient(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                              const int32_t* substeps, const double* h_first, float* loss_host,
                              float* grad_host, void* stream);

/*
 * One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias corrections by the model's
 * own count of updates, which chem_mlp_train advances too) on the FP32 master
 * weights with a caller-supplied gradient, then the BF16 copy the kernels read is
 * refreshed. grad_host: host floats in the order and length of chem_mlp_gradient's
 * output (W1, b1, W2, b2, W3, b3), e.g. a gradient accumulated over several batches.
 * Normalisation is untouched. Synchronises `stream`. Errors: CHEM_ERR_INVALID_ARG
 * (NULL, lr not finite and > 0), CHEM_ERR_CUDA.
 */
chem_status chem_mlp_apply_gradient(chem_mlp m, const float* grad_host, double lr, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CHEM_MLP_H_ */
