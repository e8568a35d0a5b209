// Host-side launchers of the device kernels (implemented in chem_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "chem_internal.h"

namespace chem {

size_t smem_bytes(int Kmax, int Imax, int prec, bool m0_global = false);
cudaError_t launch_integrate(const IntegrateArgs& a, int block, int prec, int grid, cudaStream_t st);
cudaError_t occupancy_integrate(int block, int prec, int K, int I, int* ctas_per_sm, bool m0_global = false);
cudaError_t launch_diag(const DevMech& m, int64_t n, const double* T, const double* p, const double* Y,
                        double* out, double dt, double rtol, double atol, int what, int prec,
                        cudaStream_t st, int jac_fd = 0, int q = 4);
cudaError_t launch_math(int op, const double* x, double* y, int64_t n, cudaStream_t st);
cudaError_t launch_lu_solve(int64_t n_mat, int dim, const double* A, const double* b, double* x,
                            int* info, int prec, int ir, cudaStream_t st);

}  // namespace chem
