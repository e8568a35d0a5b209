// Internal hooks between the integrator's scheduler and the learned cost / initial-step model.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "chem.h"

// Predicts, for each cell, the cost (float, substeps) and optionally the initial
// step (double, s) with the model attached to the handle. *cost and *h0 point
// into handle-owned buffers valid until the next call.
chem_status chem_internal_mlp_predict(chem_handle h, const double* T, const double* p, const double* Y,
                                      int64_t n, cudaStream_t st, const float** cost, const double** h0);

// Handle-owned per-cell buffers for the learned options (reused between calls):
// predicted cost, predicted initial step, and a snapshot of the previous cost.
chem_status chem_internal_learned_buffers(chem_handle h, int64_t n, float** cost, double** h0, float** snap);

// Cell indices ordered by decreasing cost.
chem_status chem_internal_cost_order(chem_handle h, const float* d_cost, int64_t n, cudaStream_t st,
                                     const int** perm_out);
