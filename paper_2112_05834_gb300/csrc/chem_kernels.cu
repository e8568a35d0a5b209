// Diagnostic kernels and host launchers of the batched stiff-chemistry integrator
// (sm_103a); the device code shared with chem_kernels_w.cu is in chem_device.cuh.
// This translation unit instantiates the integration kernel with the RODAS4 stepper.

#include "chem_device.cuh"

namespace chem {

size_t smem_bytes(int Kmax, int Imax, int prec, bool m0_global) {
  return make_layout(Kmax, Imax, prec, m0_global).total;
}

// W-method instantiations (chem_kernels_w.cu)
cudaError_t launch_integrate_w(const IntegrateArgs& a, int block, int prec, int grid, cudaStream_t st);

struct DiagArgs {
  DevMech m;
  int64_t n;
  const double *T, *p, *Y;
  double* out;
  double dt, rtol, atol;
  int what;    // 0 rhs, 1 jacobian, 2 h0
  int jac_fd;  // FP64 form: forward-difference Jacobian for what = 1
  int q;       // starting-step exponent 1/q (the method's embedded order + 1)
};

template <int NW, int PREC>
__global__ void __launch_bounds__(NW * 32) k_diag(const __grid_constant__ DiagArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using A = typename Policy<PREC>::ASM;
  const Layout L = make_layout(a.m.K, a.m.I, PREC);
  Cta<NW> c;
  c.bind(smem, L);

  constexpr int NT = NW * 32;
  const int K = a.m.K, n = K + 1, ld = odd_ld(n);
  for (int64_t cell = blockIdx.x; cell < a.n; cell += gridDim.x) {
    if (c.tid == 0) c.y[0] = a.T[cell];
    for (int k = c.tid; k < K; k += NT) c.y[1 + k] = a.Y[(size_t)cell * K + k];
    __syncthreads();
    const double p = a.p[cell];
    if (a.what == 0) {
      eval_rhs<NW, false, Policy<PREC>::IR>(a.m, c, c.y, p, c.f0);
      for (int i = c.tid; i < n; i += NT) a.out[(size_t)cell * n + i] = c.f0[i];
    } else if (a.what == 1) {
      if (PREC == PREC_FP64 && a.jac_fd) {
        eval_rhs<NW, false, false>(a.m, c, c.y, p, c.f0);
        fd_matrix<NW, true>(a.m, c, p, c.y, c.f0, 0.0);
      } else {
        const Scal s = eval_rhs<NW, true, Policy<PREC>::IR>(a.m, c, c.y, p, c.f0);
        build_matrix<NW, PREC, true>(a.m, c, s, c.f0, 0.0);
      }
      const A* J = reinterpret_cast<const A*>(Policy<PREC>::IR ? c.M0 : c.M);
      for (int i = c.warp; i < n; i += NW)
        for (int j = c.lane; j < n; j += 32) a.out[(size_t)cell * n * n + i * n + j] = to_double(J[i * ld + j]);
    } else {
      eval_rhs<NW, false, Policy<PREC>::IR>(a.m, c, c.y, p, c.f0);
      const double h = starting_step<NW, Policy<PREC>::IR>(a.m, c, p, a.dt, a.rtol, a.atol, a.q);
      if (c.tid == 0) a.out[cell] = h;
    }
    __syncthreads();
  }
}

// The rate kernels' elementary functions, elementwise (diagnostic): op 0 exp, 1 log,
// 2 1/x; 3 and 4 the hi and lo parts of the float-float split (widened exactly).
__global__ void k_math(int op, const double* x, double* y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (op >= 3) {
      const ff2 s = ff_split(x[i]);
      y[i] = f32_to_f64(op == 3 ? s.hi : s.lo);
    } else {
      y[i] = op == 0 ? xexp(x[i]) : op == 1 ? xlog(x[i]) : xrcp(x[i]);
    }
  }
}

struct LuArgs {
  int64_t n_mat;
  int dim;
  const double *A, *b;
  double* x;
  int* info;
  int ir;
};

template <int NW, int PREC>
__global__ void __launch_bounds__(NW * 32) k_lu_solve(const __grid_constant__ LuArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  using P = Policy<PREC>;
  using R = typename P::LU;
  const Layout L = make_layout(a.dim - 1, 1, PREC);
  Cta<NW> c;
  c.bind(smem, L);
  constexpr int NT = NW * 32;
  const int n = a.dim, ld = odd_ld(n);
  R* M = reinterpret_cast<R*>(c.M);
  for (int64_t s = blockIdx.x; s < a.n_mat; s += gridDim.x) {
    const double* As = a.A + (size_t)s * n * n;
    for (int i = c.warp; i < n; i += NW)
      for (int j = c.lane; j < n; j += 32) {
        const double v = As[i * n + j];
        M[i * ld + j] = (R)v;
        if constexpr (P::IR) reinterpret_cast<typename P::ASM*>(c.M0)[i * ld + j] = from_double<typename P::ASM>(v);
      }
    for (int i = c.tid; i < n; i += NT) c.fv[i] = a.b[(size_t)s * n + i];
    __syncthreads();
    const int info = factor<NW, PREC>(c, n);
    if (info == 0) solve<NW, PREC>(c, n, c.fv, c.u, a.ir);
    for (int i = c.tid; i < n; i += NT) a.x[(size_t)s * n + i] = info == 0 ? c.u[i] : NAN;
    if (c.tid == 0 && a.info) a.info[s] = info;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <int NW, int PREC>
static cudaError_t launch_integrate_t(const IntegrateArgs& a, int grid, cudaStream_t st) {
  return launch_integrate_m<NW, PREC, METHOD_RODAS4>(a, grid, st);
}

cudaError_t launch_integrate(const IntegrateArgs& a, int block, int prec, int grid, cudaStream_t st) {
  if (a.tab.s == 4) return launch_integrate_w(a, block, prec, grid, st);
#define LI(P)                                                                       \
  do {                                                                              \
    if (block == 64) return launch_integrate_t<2, P>(a, grid, st);                  \
    if (block == 256) return launch_integrate_t<8, P>(a, grid, st);                 \
    return launch_integrate_t<4, P>(a, grid, st);                                   \
  } while (0)
  if (prec == PREC_FP64) LI(PREC_FP64);
  if (prec == PREC_MIXED) LI(PREC_MIXED);
  LI(PREC_FP32ASM);
#undef LI
}

cudaError_t occupancy_integrate(int block, int prec, int K, int I, int* ctas_per_sm, bool m0_global) {
  const size_t smem = smem_bytes(K, I, prec, m0_global);
  cudaError_t e;
#define OCC(NW, P)                                                                                    \
  do {                                                                                                \
    e = prep(k_integrate<NW, P, METHOD_RODAS4>, smem);                                                \
    if (e != cudaSuccess) return e;                                                                   \
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_integrate<NW, P, METHOD_RODAS4>, \
                                                         NW * 32, smem);                              \
  } while (0)
#define OCCP(P)                  \
  do {                           \
    if (block == 64) OCC(2, P);  \
    if (block == 256) OCC(8, P); \
    OCC(4, P);                   \
  } while (0)
  if (prec == PREC_FP64) OCCP(PREC_FP64);
  if (prec == PREC_MIXED) OCCP(PREC_MIXED);
  OCCP(PREC_FP32ASM);
#undef OCCP
#undef OCC
}

template <int PREC, class ArgT, class KernelT>
static cudaError_t launch_simple(KernelT k, const ArgT& a, size_t smem, int grid, cudaStream_t st) {
  cudaError_t e = prep(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 128, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_diag(const DevMech& m, int64_t n, const double* T, const double* p, const double* Y,
                        double* out, double dt, double rtol, double atol, int what, int prec,
                        cudaStream_t st, int jac_fd, int q) {
  DiagArgs a;
  a.jac_fd = jac_fd;
  a.q = q;
  a.m = m;
  a.n = n;
  a.T = T;
  a.p = p;
  a.Y = Y;
  a.out = out;
  a.dt = dt;
  a.rtol = rtol;
  a.atol = atol;
  a.what = what;
  const size_t smem = smem_bytes(m.K, m.I, prec);
  const int grid = (int)(n < 65535 ? n : 65535);
  if (prec == PREC_FP64) return launch_simple<PREC_FP64>(k_diag<4, PREC_FP64>, a, smem, grid, st);
  if (prec == PREC_MIXED) return launch_simple<PREC_MIXED>(k_diag<4, PREC_MIXED>, a, smem, grid, st);
  return launch_simple<PREC_FP32ASM>(k_diag<4, PREC_FP32ASM>, a, smem, grid, st);
}

cudaError_t launch_math(int op, const double* x, double* y, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = (n + 255) / 256;
  k_math<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(op, x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_lu_solve(int64_t n_mat, int dim, const double* A, const double* b, double* x,
                            int* info, int prec, int ir, cudaStream_t st) {
  LuArgs a;
  a.n_mat = n_mat;
  a.dim = dim;
  a.A = A;
  a.b = b;
  a.x = x;
  a.info = info;
  a.ir = ir;
  const size_t smem = smem_bytes(dim - 1, 1, prec);
  const int grid = (int)(n_mat < 65535 ? n_mat : 65535);
  if (prec == PREC_FP64) return launch_simple<PREC_FP64>(k_lu_solve<4, PREC_FP64>, a, smem, grid, st);
  if (prec == PREC_MIXED) return launch_simple<PREC_MIXED>(k_lu_solve<4, PREC_MIXED>, a, smem, grid, st);
  return launch_simple<PREC_FP32ASM>(k_lu_solve<4, PREC_FP32ASM>, a, smem, grid, st);
}

}  // namespace chem
