// Learned per-cell cost and initial-step model: BF16 tensor-core GEMMs with FP32
// accumulation (mma.sync m16n8k16), GELU MLP forward/backward, Adam on FP32
// master weights, and the predictions the scheduler consumes.
//
// The paper has no learned component: DLBFoam balances measured per-process cost
// (Methodology, "DLBFoam: Dynamic load balancing"; Results, Fig. 4). Here the
// integrator's own per-cell logs (substeps, first accepted step) train a model
// that orders the work queue heaviest-first and seeds each cell's first step.

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "chem.h"
#include "chem_capi_internal.h"
#include "chem_mlp.h"
#include "chem_mlp_internal.h"

namespace {

constexpr int kH = 128;      // hidden width
constexpr int kChunk = 65536;  // rows per inference chunk
typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ---------------------------------------------------------------------------
// features: x = [T/1000, ln p, ln(Y_k + 1e-20)], optionally standardised
// ---------------------------------------------------------------------------
__device__ __forceinline__ double feature(const double* T, const double* p, const double* Y, int K, int64_t c,
                                          int d) {
  if (d == 0) return T[c] * 1e-3;
  if (d == 1) return log(p[c]);
  return log(Y[(size_t)c * K + (d - 2)] + 1e-20);
}

__global__ void k_feature_stats(const double* T, const double* p, const double* Y, int K, int64_t n,
                                double* sums /* [2 D] */) {
  extern __shared__ double sh[];
  const int D = K + 2;
  for (int i = threadIdx.x; i < 2 * D; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x)
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
      const double x = feature(T, p, Y, K, r, d);
      sh[d] += x;
      sh[D + d] += x * x;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * D; i += blockDim.x) atomicAdd(&sums[i], sh[i]);
}

__global__ void k_target_stats(const int32_t* sub, const double* hf, int64_t n, double* sums /* [4] */) {
  double a = 0, a2 = 0, b = 0, b2 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t0 = log(fmax((double)sub[i], 1.0)), t1 = log(fmax(hf[i], 1e-300));
    a += t0;
    a2 += t0 * t0;
    b += t1;
    b2 += t1 * t1;
  }
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    b2 += __shfl_xor_sync(0xffffffffu, b2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], a2);
    atomicAdd(&sums[2], b);
    atomicAdd(&sums[3], b2);
  }
}

// Standardised BF16 features of rows [r0, r0 + rows). With zmax > 0, out[r] is set
// to 1 for a row with a standardised feature beyond +-zmax (any thread of the row may
// store it; all store the same value; the head kernel reads and clears it).
__global__ void k_features(const double* T, const double* p, const double* Y, int K, int64_t r0, int64_t rows,
                           const float* norm, bf16* X, float zmax = 0.0f, unsigned char* out = nullptr) {
  const int D = K + 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rows * D; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / D;
    const int d = (int)(e - r * D);
    const double x = feature(T, p, Y, K, r0 + r, d);
    const float z = (float)((x - norm[d]) / norm[D + d]);
    X[e] = __float2bfloat16(z);
    if (zmax > 0.0f && !(fabsf(z) <= zmax)) out[r] = 1;
  }
}

__global__ void k_targets(const int32_t* sub, const double* hf, int64_t n, const float* norm_t, float* Ts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double t0 = log(fmax((double)sub[i], 1.0)), t1 = log(fmax(hf[i], 1e-300));
    Ts[2 * i] = (float)((t0 - norm_t[0]) / norm_t[2]);
    Ts[2 * i + 1] = (float)((t1 - norm_t[1]) / norm_t[3]);
  }
}

__global__ void k_gather(const bf16* X, const float* Ts, const int* perm, int64_t b0, int rows, int D, bf16* Xb,
                         float* Tb) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * D; e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / D), d = (int)(e - (int64_t)r * D);
    Xb[e] = X[(size_t)perm[b0 + r] * D + d];
  }
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
    Tb[2 * r] = Ts[2 * (size_t)perm[b0 + r]];
    Tb[2 * r + 1] = Ts[2 * (size_t)perm[b0 + r] + 1];
  }
}

// ---------------------------------------------------------------------------
// BF16 GEMM, FP32 accumulation: C(m, n) = sum_k A(m, k) B(n, k) with general strides
// A(m, k) = A[m sam + k sak], B(n, k) = B[n sbn + k sbk]. 64 x 64 tile per CTA,
// 4 warps of 32 x 32, mma.sync.m16n8k16; split-K over blockIdx.z.
// mode 0: C[z zstride + m ldc + n] = acc
// mode 1: z = acc + bias[n]; Zout (optional) = z; Hout = bf16(GELU(z))
// mode 2: dZout = bf16(acc * GELU'(Zin))
// ---------------------------------------------------------------------------
struct GemmP {
  const bf16* A;
  long long sam, sak;
  const bf16* B;
  long long sbn, sbk;
  int M, N, K, kchunk, mode;
  float* C;
  long long ldc, zstride;
  const float* bias;
  float* Zout;
  bf16* Hout;
  const float* Zin;
  bf16* dZout;
};

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(128) k_gemm(const GemmP p) {
  __shared__ __align__(16) bf16 As[64][40];
  __shared__ __align__(16) bf16 Bs[64][40];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, t4 = lane & 3;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  const int kb = blockIdx.z * p.kchunk;
  const int ke = min(p.K, kb + p.kchunk);
  const bf16 zero = __float2bfloat16(0.0f);
  float acc[2][4][4];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.0f;
  for (int k0 = kb; k0 < ke; k0 += 32) {
    for (int e = tid; e < 64 * 32; e += 128) {
      const int r = e >> 5, cc = e & 31;
      const int gk = k0 + cc;
      const int gm = m0 + r, gn = n0 + r;
      As[r][cc] = (gm < p.M && gk < ke) ? p.A[(long long)gm * p.sam + (long long)gk * p.sak] : zero;
      Bs[r][cc] = (gn < p.N && gk < ke) ? p.B[(long long)gn * p.sbn + (long long)gk * p.sbk] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      uint32_t a[2][4], b[4][2];
      const int c = kk + t4 * 2;
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm * 32 + mt * 16 + g;
        a[mt][0] = *reinterpret_cast<const uint32_t*>(&As[r][c]);
        a[mt][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c]);
        a[mt][2] = *reinterpret_cast<const uint32_t*>(&As[r][c + 8]);
        a[mt][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][c + 8]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int nn = wn * 32 + nt * 8 + g;
        b[nt][0] = *reinterpret_cast<const uint32_t*>(&Bs[nn][c]);
        b[nt][1] = *reinterpret_cast<const uint32_t*>(&Bs[nn][c + 8]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt], b[nt]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int hf = 0; hf < 2; ++hf)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int m = m0 + wm * 32 + mt * 16 + g + hf * 8;
          const int n = n0 + wn * 32 + nt * 8 + t4 * 2 + j;
          if (m >= p.M || n >= p.N) continue;
          const float v = acc[mt][nt][hf * 2 + j];
          if (p.mode == 0) {
            p.C[(long long)blockIdx.z * p.zstride + (long long)m * p.ldc + n] = v;
          } else if (p.mode == 1) {
            const float z = v + p.bias[n];
            if (p.Zout) p.Zout[(long long)m * p.N + n] = z;
            p.Hout[(long long)m * p.N + n] = __float2bfloat16(gelu(z));
          } else {
            p.dZout[(long long)m * p.N + n] = __float2bfloat16(v * gelu_grad(p.Zin[(long long)m * p.N + n]));
          }
        }
}

// ---------------------------------------------------------------------------
// output head (128 -> 2), one warp per row. Training: loss, dZ2, per-warp partial
// gradients of W3/b3. Prediction: denormalised outputs.
// ---------------------------------------------------------------------------
struct HeadP {
  const bf16* H2;
  const float* Z2;
  const bf16* W3;   // [2][128] bf16
  const float* b3;  // [2]
  const float* Tb;  // standardised targets [rows][2] (training)
  int rows;
  float inv_B;
  bf16* dZ2;
  float* part;      // [warps][2*128 + 2 + 1]
  const float* norm_t;  // mu_t[2], sd_t[2] (prediction)
  float* ln_cost;
  float* ln_h0;
  float* cost;      // exp(ln_cost)
  double* h0;       // max(exp(ln_h0), 1e-14); NaN for a row flagged in out_of_range
  unsigned char* out_of_range;  // [rows] rows with a feature beyond the range (cleared here)
  int64_t out0;     // output row offset
};

__global__ void k_head(const HeadP p, int train) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  float w0[4], w1[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    w0[j] = __bfloat162float(p.W3[lane * 4 + j]);
    w1[j] = __bfloat162float(p.W3[kH + lane * 4 + j]);
  }
  float gW0[4] = {0, 0, 0, 0}, gW1[4] = {0, 0, 0, 0}, gb0 = 0, gb1 = 0, loss = 0;
  for (int r = gw; r < p.rows; r += nw) {
    float h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) h[j] = __bfloat162float(p.H2[(size_t)r * kH + lane * 4 + j]);
    float o0 = 0, o1 = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o0 += h[j] * w0[j];
      o1 += h[j] * w1[j];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      o0 += __shfl_xor_sync(0xffffffffu, o0, o);
      o1 += __shfl_xor_sync(0xffffffffu, o1, o);
    }
    o0 += p.b3[0];
    o1 += p.b3[1];
    if (train) {
      const float r0 = o0 - p.Tb[2 * r], r1 = o1 - p.Tb[2 * r + 1];
      loss += 0.5f * (r0 * r0 + r1 * r1) * p.inv_B;
      const float d0 = r0 * p.inv_B, d1 = r1 * p.inv_B;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float z = p.Z2[(size_t)r * kH + lane * 4 + j];
        p.dZ2[(size_t)r * kH + lane * 4 + j] = __float2bfloat16((d0 * w0[j] + d1 * w1[j]) * gelu_grad(z));
        gW0[j] += d0 * h[j];
        gW1[j] += d1 * h[j];
      }
      gb0 += d0;
      gb1 += d1;
    } else if (lane == 0) {
      const float l0 = o0 * p.norm_t[2] + p.norm_t[0];
      const float l1 = o1 * p.norm_t[3] + p.norm_t[1];
      const int64_t q = p.out0 + r;
      if (p.ln_cost) p.ln_cost[q] = l0;
      if (p.ln_h0) p.ln_h0[q] = l1;
      if (p.cost) p.cost[q] = expf(fminf(l0, 80.0f));
      bool far = false;
      if (p.out_of_range && p.out_of_range[r]) {
        far = true;
        p.out_of_range[r] = 0;
      }
      if (p.h0) p.h0[q] = far ? __longlong_as_double(0x7ff8000000000000LL) : fmax(exp((double)l1), 1e-14);
    }
  }
  if (train) {
    float* pp = p.part + (size_t)gw * (2 * kH + 3);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      pp[lane * 4 + j] = gW0[j];
      pp[kH + lane * 4 + j] = gW1[j];
    }
    if (lane == 0) {
      pp[2 * kH] = gb0;
      pp[2 * kH + 1] = gb1;
      pp[2 * kH + 2] = loss;
    }
  }
}

// out[j] = sum_s part[s * stride + j], j < len (fixed order)
__global__ void k_reduce(const float* part, int S, int stride, int len, float* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < len; j += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int i = 0; i < S; ++i) s += part[(size_t)i * stride + j];
    out[j] = s;
  }
}

// column sums of a [rows][128] bf16 matrix into part[chunk][128]
__global__ void k_colsum(const bf16* Z, int rows, int rows_per_block, float* part) {
  const int col = threadIdx.x;
  const int r0 = blockIdx.x * rows_per_block, r1 = min(rows, r0 + rows_per_block);
  float s = 0.0f;
  for (int r = r0; r < r1; ++r) s += __bfloat162float(Z[(size_t)r * kH + col]);
  part[(size_t)blockIdx.x * kH + col] = s;
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, bf16* wb, int64_t n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16(wi);
  }
}

__global__ void k_to_bf16(const float* w, bf16* wb, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16(w[i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// model object
// ---------------------------------------------------------------------------
struct chem_mlp_s {
  int K = 0, D = 0;
  int64_t nw = 0;  // weight+bias floats
  int64_t oW1 = 0, ob1 = 0, oW2 = 0, ob2 = 0, oW3 = 0, ob3 = 0;
  float* w = nullptr;  // FP32 master [nw]
  float* g = nullptr;  // gradient [nw]
  float* m = nullptr;
  float* v = nullptr;
  bf16* wb = nullptr;  // BF16 copy [nw]
  float* norm = nullptr;          // device: mu_x[D], sd_x[D], mu_t[2], sd_t[2]
  std::vector<float> norm_h;      // host copy
  int64_t adam_t = 0;
  // scratch
  int64_t cap = 0;
  bf16 *X = nullptr, *H1 = nullptr, *H2 = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  float *Z1 = nullptr, *Z2 = nullptr, *Tb = nullptr, *part = nullptr;
  int64_t part_cap = 0;
  unsigned char* out_of_range = nullptr;  // [kChunk] per-row range flags (kept zero between calls)
  std::string err;
};

static chem_status mlp_cuda(chem_mlp m, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CHEM_OK;
  if (m) m->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? CHEM_ERR_OOM : CHEM_ERR_CUDA;
}

#define MLP_TRY(m, call)                                    \
  do {                                                      \
    chem_status s_ = mlp_cuda((m), (call), #call);          \
    if (s_ != CHEM_OK) return s_;                           \
  } while (0)

static void mlp_free_scratch(chem_mlp m) {
  for (void* p : {(void*)m->X, (void*)m->H1, (void*)m->H2, (void*)m->dZ2, (void*)m->dZ1, (void*)m->Z1, (void*)m->Z2,
                  (void*)m->Tb})
    if (p) cudaFree(p);
  m->X = m->H1 = m->H2 = m->dZ2 = m->dZ1 = nullptr;
  m->Z1 = m->Z2 = m->Tb = nullptr;
  m->cap = 0;
}

static chem_status mlp_scratch(chem_mlp m, int64_t rows, bool train) {
  if (rows <= m->cap && (!train || m->Z1)) return CHEM_OK;
  cudaDeviceSynchronize();
  mlp_free_scratch(m);
  const int64_t r = std::max<int64_t>(rows, 1024);
  MLP_TRY(m, cudaMalloc(&m->X, r * m->D * sizeof(bf16)));
  MLP_TRY(m, cudaMalloc(&m->H1, r * kH * sizeof(bf16)));
  MLP_TRY(m, cudaMalloc(&m->H2, r * kH * sizeof(bf16)));
  if (train) {
    MLP_TRY(m, cudaMalloc(&m->dZ2, r * kH * sizeof(bf16)));
    MLP_TRY(m, cudaMalloc(&m->dZ1, r * kH * sizeof(bf16)));
    MLP_TRY(m, cudaMalloc(&m->Z1, r * kH * sizeof(float)));
    MLP_TRY(m, cudaMalloc(&m->Z2, r * kH * sizeof(float)));
    MLP_TRY(m, cudaMalloc(&m->Tb, r * 2 * sizeof(float)));
  }
  m->cap = r;
  return CHEM_OK;
}

static chem_status mlp_part(chem_mlp m, int64_t floats) {
  if (floats <= m->part_cap) return CHEM_OK;
  cudaDeviceSynchronize();
  if (m->part) cudaFree(m->part);
  m->part = nullptr;
  MLP_TRY(m, cudaMalloc(&m->part, floats * sizeof(float)));
  m->part_cap = floats;
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_create(int32_t n_species, uint64_t seed, chem_mlp* out) {
  if (!out || n_species < 1 || n_species > 255) return CHEM_ERR_INVALID_ARG;
  *out = nullptr;
  chem_mlp m = new chem_mlp_s();
  m->K = n_species;
  m->D = n_species + 2;
  const int D = m->D;
  m->oW1 = 0;
  m->ob1 = m->oW1 + (int64_t)kH * D;
  m->oW2 = m->ob1 + kH;
  m->ob2 = m->oW2 + (int64_t)kH * kH;
  m->oW3 = m->ob2 + kH;
  m->ob3 = m->oW3 + 2 * kH;
  m->nw = m->ob3 + 2;
  std::vector<float> w(m->nw);
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  auto fill = [&](int64_t o, int64_t cnt, int fan) {
    for (int64_t i = 0; i < cnt; ++i) w[o + i] = (float)(U(rng) / std::sqrt((double)fan));
  };
  fill(m->oW1, (int64_t)kH * D, D);
  fill(m->ob1, kH, D);
  fill(m->oW2, (int64_t)kH * kH, kH);
  fill(m->ob2, kH, kH);
  fill(m->oW3, 2 * kH, kH);
  fill(m->ob3, 2, kH);
  m->norm_h.assign(2 * D + 4, 0.0f);
  for (int d = 0; d < D; ++d) m->norm_h[D + d] = 1.0f;
  m->norm_h[2 * D + 2] = m->norm_h[2 * D + 3] = 1.0f;
  cudaError_t e = cudaMalloc(&m->w, m->nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->g, m->nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->m, m->nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->v, m->nw * 4);
  if (e == cudaSuccess) e = cudaMalloc(&m->wb, m->nw * sizeof(bf16));
  if (e == cudaSuccess) e = cudaMalloc(&m->norm, m->norm_h.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(m->w, w.data(), m->nw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m, 0, m->nw * 4);
  if (e == cudaSuccess) e = cudaMemset(m->v, 0, m->nw * 4);
  if (e == cudaSuccess) e = cudaMemcpy(m->norm, m->norm_h.data(), m->norm_h.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_to_bf16<<<64, 256>>>(m->w, m->wb, m->nw);
    e = cudaDeviceSynchronize();
  }
  if (e != cudaSuccess) {
    chem_mlp_destroy(m);
    return e == cudaErrorMemoryAllocation ? CHEM_ERR_OOM : CHEM_ERR_CUDA;
  }
  *out = m;
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_destroy(chem_mlp m) {
  if (!m) return CHEM_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  mlp_free_scratch(m);
  for (void* p : {(void*)m->w, (void*)m->g, (void*)m->m, (void*)m->v, (void*)m->wb, (void*)m->norm, (void*)m->part,
                  (void*)m->out_of_range})
    if (p) cudaFree(p);
  delete m;
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_attach(chem_handle h, chem_mlp m) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (m && m->K != h->K) {
    h->err = "chem_mlp_attach: model and mechanism disagree on the number of species";
    return CHEM_ERR_INVALID_ARG;
  }
  h->mlp = m;
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_get_params(chem_mlp m, float* buf, int64_t* n_floats) {
  if (!m || !n_floats) return CHEM_ERR_INVALID_ARG;
  const int64_t nn = (int64_t)m->norm_h.size();
  *n_floats = nn + m->nw;
  if (!buf) return CHEM_OK;
  std::memcpy(buf, m->norm_h.data(), nn * 4);
  MLP_TRY(m, cudaMemcpy(buf + nn, m->w, m->nw * 4, cudaMemcpyDeviceToHost));
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_set_params(chem_mlp m, const float* buf, int64_t n_floats) {
  if (!m || !buf) return CHEM_ERR_INVALID_ARG;
  const int64_t nn = (int64_t)m->norm_h.size();
  if (n_floats != nn + m->nw) {
    m->err = "chem_mlp_set_params: wrong length";
    return CHEM_ERR_INVALID_ARG;
  }
  std::memcpy(m->norm_h.data(), buf, nn * 4);
  MLP_TRY(m, cudaMemcpy(m->norm, buf, nn * 4, cudaMemcpyHostToDevice));
  MLP_TRY(m, cudaMemcpy(m->w, buf + nn, m->nw * 4, cudaMemcpyHostToDevice));
  k_to_bf16<<<64, 256>>>(m->w, m->wb, m->nw);
  MLP_TRY(m, cudaDeviceSynchronize());
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------
// returns the number of K splits used
static int gemm(cudaStream_t st, const bf16* A, long long sam, long long sak, const bf16* B, long long sbn,
                 long long sbk, int M, int N, int K, int splits, int mode, float* C, long long ldc,
                 const float* bias, float* Zout, bf16* Hout, const float* Zin, bf16* dZout) {
  GemmP p;
  p.A = A;
  p.sam = sam;
  p.sak = sak;
  p.B = B;
  p.sbn = sbn;
  p.sbk = sbk;
  p.M = M;
  p.N = N;
  p.K = K;
  p.kchunk = ((K + splits - 1) / splits + 31) / 32 * 32;
  p.mode = mode;
  p.C = C;
  p.ldc = ldc;
  p.zstride = (long long)M * ldc;
  p.bias = bias;
  p.Zout = Zout;
  p.Hout = Hout;
  p.Zin = Zin;
  p.dZout = dZout;
  dim3 grid((M + 63) / 64, (N + 63) / 64, (K + p.kchunk - 1) / p.kchunk);
  k_gemm<<<grid, 128, 0, st>>>(p);
  return (int)grid.z;
}

// forward of `rows` standardised rows in m->X; training keeps Z1, Z2
static void forward(chem_mlp m, int rows, bool train, cudaStream_t st) {
  const int D = m->D;
  gemm(st, m->X, D, 1, m->wb + m->oW1, D, 1, rows, kH, D, 1, 1, nullptr, 0, m->w + m->ob1, train ? m->Z1 : nullptr,
       m->H1, nullptr, nullptr);
  gemm(st, m->H1, kH, 1, m->wb + m->oW2, kH, 1, rows, kH, kH, 1, 1, nullptr, 0, m->w + m->ob2,
       train ? m->Z2 : nullptr, m->H2, nullptr, nullptr);
}

static int head_warps(int rows) { return std::max(1, std::min(1024, (rows + 31) / 32)); }

// forward + backward of the batch in m->X / m->Tb; gradient into m->g; returns device loss in part tail
static chem_status fwd_bwd(chem_mlp m, int rows, cudaStream_t st, float* loss_dev) {
  const int D = m->D;
  forward(m, rows, true, st);
  const int hw = head_warps(rows);
  const int splits = std::max(1, std::min(64, rows / 256));
  const int colblocks = std::max(1, std::min(256, rows / 64));
  const int64_t need = std::max<int64_t>({(int64_t)hw * (2 * kH + 3), (int64_t)splits * kH * std::max(D, kH),
                                          (int64_t)colblocks * kH});
  chem_status s = mlp_part(m, need);
  if (s != CHEM_OK) return s;
  HeadP hp{};
  hp.H2 = m->H2;
  hp.Z2 = m->Z2;
  hp.W3 = m->wb + m->oW3;
  hp.b3 = m->w + m->ob3;
  hp.Tb = m->Tb;
  hp.rows = rows;
  hp.inv_B = 1.0f / (float)rows;
  hp.dZ2 = m->dZ2;
  hp.part = m->part;
  k_head<<<(hw * 32 + 255) / 256, 256, 0, st>>>(hp, 1);
  // W3, b3 gradient and the loss
  k_reduce<<<2, 128, 0, st>>>(m->part, hw, 2 * kH + 3, 2 * kH + 2, m->g + m->oW3);
  k_reduce<<<1, 32, 0, st>>>(m->part + 2 * kH + 2, hw, 2 * kH + 3, 1, loss_dev);
  // dW2 = dZ2^T H1 (split-K over the batch), db2 = column sums of dZ2
  const int S2 = gemm(st, m->dZ2, 1, kH, m->H1, 1, kH, kH, kH, rows, splits, 0, m->part, kH, nullptr, nullptr,
                      nullptr, nullptr, nullptr);
  k_reduce<<<64, 256, 0, st>>>(m->part, S2, kH * kH, kH * kH, m->g + m->oW2);
  const int rpb = (rows + colblocks - 1) / colblocks;
  k_colsum<<<colblocks, kH, 0, st>>>(m->dZ2, rows, rpb, m->part);
  k_reduce<<<1, kH, 0, st>>>(m->part, colblocks, kH, kH, m->g + m->ob2);
  // dZ1 = (dZ2 W2) * GELU'(Z1)
  gemm(st, m->dZ2, kH, 1, m->wb + m->oW2, 1, kH, rows, kH, kH, 1, 2, nullptr, 0, nullptr, nullptr, nullptr, m->Z1,
       m->dZ1);
  // dW1 = dZ1^T X, db1 = column sums of dZ1
  const int S1 = gemm(st, m->dZ1, 1, kH, m->X, 1, D, kH, D, rows, splits, 0, m->part, D, nullptr, nullptr, nullptr,
                      nullptr, nullptr);
  k_reduce<<<64, 256, 0, st>>>(m->part, S1, kH * D, kH * D, m->g + m->oW1);
  k_colsum<<<colblocks, kH, 0, st>>>(m->dZ1, rows, rpb, m->part);
  k_reduce<<<1, kH, 0, st>>>(m->part, colblocks, kH, kH, m->g + m->ob1);
  return mlp_cuda(m, cudaGetLastError(), "mlp backward");
}

// Adam's bias corrections 1 - beta^t for the FP32 betas the kernel uses, evaluated in
// double and rounded once (1 - beta2^t in float loses ~1e-5 relative for small t).
static void adam_corrections(float b1, float b2, int64_t t, float* c1, float* c2) {
  *c1 = (float)(1.0 - std::pow((double)b1, (double)t));
  *c2 = (float)(1.0 - std::pow((double)b2, (double)t));
}

static chem_status set_normalisation(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                                     const int32_t* sub, const double* hf, cudaStream_t st) {
  const int D = m->D;
  double* sums = nullptr;
  MLP_TRY(m, cudaMalloc(&sums, (2 * D + 4) * sizeof(double)));
  cudaMemsetAsync(sums, 0, (2 * D + 4) * sizeof(double), st);
  const int grid = (int)std::min<int64_t>(n, 512);
  k_feature_stats<<<grid, 128, 2 * D * sizeof(double), st>>>(T, p, Y, m->K, n, sums);
  k_target_stats<<<(int)std::min<int64_t>((n + 255) / 256, 512), 256, 0, st>>>(sub, hf, n, sums + 2 * D);
  std::vector<double> h(2 * D + 4);
  cudaError_t e = cudaMemcpyAsync(h.data(), sums, h.size() * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sums);
  MLP_TRY(m, e);
  for (int d = 0; d < D; ++d) {
    const double mu = h[d] / n;
    const double var = std::max(h[D + d] / n - mu * mu, 0.0);
    m->norm_h[d] = (float)mu;
    m->norm_h[D + d] = (float)std::max(std::sqrt(var), 1e-3);
  }
  for (int t = 0; t < 2; ++t) {
    const double mu = h[2 * D + 2 * t] / n;
    const double var = std::max(h[2 * D + 2 * t + 1] / n - mu * mu, 0.0);
    m->norm_h[2 * D + t] = (float)mu;
    m->norm_h[2 * D + 2 + t] = (float)std::max(std::sqrt(var), 1e-3);
  }
  MLP_TRY(m, cudaMemcpyAsync(m->norm, m->norm_h.data(), m->norm_h.size() * 4, cudaMemcpyHostToDevice, st));
  MLP_TRY(m, cudaStreamSynchronize(st));
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_train(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                                      const int32_t* substeps, const double* h_first, int32_t epochs,
                                      int32_t batch, double lr, uint64_t seed, float* loss_host, void* stream) {
  if (!m || n < 1 || !T || !p || !Y || !substeps || !h_first || epochs < 0 || batch < 32 || !(lr > 0.0))
    return CHEM_ERR_INVALID_ARG;
  if (n > 2147483647LL) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int D = m->D;
  chem_status s = set_normalisation(m, n, T, p, Y, substeps, h_first, st);
  if (s != CHEM_OK) return s;
  // standardised features and targets of all samples
  bf16* Xall = nullptr;
  float* Tall = nullptr;
  int* perm_d = nullptr;
  float* loss_d = nullptr;
  MLP_TRY(m, cudaMalloc(&Xall, (size_t)n * D * sizeof(bf16)));
  MLP_TRY(m, cudaMalloc(&Tall, (size_t)n * 2 * sizeof(float)));
  MLP_TRY(m, cudaMalloc(&perm_d, (size_t)n * sizeof(int)));
  const int B = (int)std::min<int64_t>(batch, n);
  const int nb = (int)((n + B - 1) / B);
  MLP_TRY(m, cudaMalloc(&loss_d, (size_t)nb * sizeof(float)));
  const int gridE = (int)std::min<int64_t>(((int64_t)n * D + 255) / 256, 4096);
  k_features<<<gridE, 256, 0, st>>>(T, p, Y, m->K, 0, n, m->norm, Xall);
  k_targets<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(substeps, h_first, n, m->norm + 2 * D,
                                                                            Tall);
  s = mlp_scratch(m, B, true);
  if (s != CHEM_OK) return s;
  std::vector<int> perm(n);
  std::mt19937_64 rng(seed);
  std::vector<float> batch_losses(nb);
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
    std::shuffle(perm.begin(), perm.end(), rng);
    MLP_TRY(m, cudaMemcpyAsync(perm_d, perm.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    for (int bi = 0; bi < nb; ++bi) {
      const int64_t b0 = (int64_t)bi * B;
      const int rows = (int)std::min<int64_t>(B, n - b0);
      k_gather<<<256, 256, 0, st>>>(Xall, Tall, perm_d, b0, rows, D, m->X, m->Tb);
      s = fwd_bwd(m, rows, st, loss_d + bi);
      if (s != CHEM_OK) return s;
      ++m->adam_t;
      float c1, c2;
      adam_corrections(b1, b2, m->adam_t, &c1, &c2);
      k_adam<<<64, 256, 0, st>>>(m->w, m->g, m->m, m->v, m->wb, m->nw, (float)lr, b1, b2, eps, c1, c2);
    }
    // the host permutation buffer is reused next epoch: wait, and collect the batch losses
    MLP_TRY(m, cudaMemcpyAsync(batch_losses.data(), loss_d, nb * sizeof(float), cudaMemcpyDeviceToHost, st));
    MLP_TRY(m, cudaStreamSynchronize(st));
    if (loss_host) {
      double acc = 0.0;
      for (int bi = 0; bi < nb; ++bi) acc += batch_losses[bi];
      loss_host[ep] = (float)(acc / nb);
    }
  }
  MLP_TRY(m, cudaStreamSynchronize(st));
  cudaFree(Xall);
  cudaFree(Tall);
  cudaFree(perm_d);
  cudaFree(loss_d);
  return mlp_cuda(m, cudaGetLastError(), "chem_mlp_train");
}

extern "C" chem_status chem_mlp_gradient(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                                         const int32_t* substeps, const double* h_first, float* loss_host,
                                         float* grad_host, void* stream) {
  if (!m || n < 1 || n > 1 << 20 || !T || !p || !Y || !substeps || !h_first) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int D = m->D;
  chem_status s = mlp_scratch(m, n, true);
  if (s != CHEM_OK) return s;
  const int gridE = (int)std::min<int64_t>(((int64_t)n * D + 255) / 256, 4096);
  k_features<<<gridE, 256, 0, st>>>(T, p, Y, m->K, 0, n, m->norm, m->X);
  k_targets<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(substeps, h_first, n, m->norm + 2 * D,
                                                                            m->Tb);
  float* loss_d = nullptr;
  MLP_TRY(m, cudaMalloc(&loss_d, sizeof(float)));
  s = fwd_bwd(m, (int)n, st, loss_d);
  if (s != CHEM_OK) return s;
  float l = 0.0f;
  MLP_TRY(m, cudaMemcpyAsync(&l, loss_d, 4, cudaMemcpyDeviceToHost, st));
  if (grad_host) MLP_TRY(m, cudaMemcpyAsync(grad_host, m->g, m->nw * 4, cudaMemcpyDeviceToHost, st));
  MLP_TRY(m, cudaStreamSynchronize(st));
  cudaFree(loss_d);
  if (loss_host) *loss_host = l;
  return CHEM_OK;
}

extern "C" chem_status chem_mlp_apply_gradient(chem_mlp m, const float* grad_host, double lr, void* stream) {
  if (!m || !grad_host || !(lr > 0.0) || !std::isfinite(lr)) return CHEM_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  MLP_TRY(m, cudaMemcpyAsync(m->g, grad_host, m->nw * 4, cudaMemcpyHostToDevice, st));
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  ++m->adam_t;
  float c1, c2;
  adam_corrections(b1, b2, m->adam_t, &c1, &c2);
  k_adam<<<64, 256, 0, st>>>(m->w, m->g, m->m, m->v, m->wb, m->nw, (float)lr, b1, b2, eps, c1, c2);
  MLP_TRY(m, cudaGetLastError());
  MLP_TRY(m, cudaStreamSynchronize(st));
  return CHEM_OK;
}

// zmax > 0: cells with a standardised feature beyond +-zmax training standard
// deviations get a NaN initial step (the integrator then takes its heuristic).
static chem_status predict_into(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y, float* ln_cost,
                                float* ln_h0, float* cost, double* h0, cudaStream_t st, float zmax = 0.0f) {
  const int D = m->D;
  chem_status s = mlp_scratch(m, std::min<int64_t>(n, kChunk), false);
  if (s != CHEM_OK) return s;
  if (zmax > 0.0f && h0 && !m->out_of_range) {
    MLP_TRY(m, cudaMalloc(&m->out_of_range, kChunk));
    MLP_TRY(m, cudaMemsetAsync(m->out_of_range, 0, kChunk, st));
  }
  if (!h0) zmax = 0.0f;
  for (int64_t r0 = 0; r0 < n; r0 += kChunk) {
    const int rows = (int)std::min<int64_t>(kChunk, n - r0);
    const int gridE = (int)std::min<int64_t>(((int64_t)rows * D + 255) / 256, 4096);
    k_features<<<gridE, 256, 0, st>>>(T, p, Y, m->K, r0, rows, m->norm, m->X, zmax, m->out_of_range);
    forward(m, rows, false, st);
    HeadP hp{};
    hp.H2 = m->H2;
    hp.W3 = m->wb + m->oW3;
    hp.b3 = m->w + m->ob3;
    hp.rows = rows;
    hp.norm_t = m->norm + 2 * D;
    hp.ln_cost = ln_cost;
    hp.ln_h0 = ln_h0;
    hp.cost = cost;
    hp.h0 = h0;
    hp.out_of_range = zmax > 0.0f ? m->out_of_range : nullptr;
    hp.out0 = r0;
    const int hw = head_warps(rows);
    k_head<<<(hw * 32 + 255) / 256, 256, 0, st>>>(hp, 0);
  }
  return mlp_cuda(m, cudaGetLastError(), "chem_mlp_predict");
}

extern "C" chem_status chem_mlp_predict(chem_mlp m, int64_t n, const double* T, const double* p, const double* Y,
                                        float* ln_cost, float* ln_h0, void* stream) {
  if (!m || n < 0 || (n > 0 && (!T || !p || !Y))) return CHEM_ERR_INVALID_ARG;
  if (n == 0) return CHEM_OK;
  return predict_into(m, n, T, p, Y, ln_cost, ln_h0, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

// Scheduler hook: predicted cost (float, substeps) and initial step (double) per cell.
chem_status chem_internal_mlp_predict(chem_handle h, const double* T, const double* p, const double* Y, int64_t n,
                                      cudaStream_t st, const float** cost, const double** h0) {
  float* c = nullptr;
  double* hh = nullptr;
  chem_status s = chem_internal_learned_buffers(h, n, &c, &hh, nullptr);
  if (s != CHEM_OK) return s;
  s = predict_into(h->mlp, n, T, p, Y, nullptr, nullptr, c, h0 ? hh : nullptr, st,
                   (float)h->h0_range);
  if (s != CHEM_OK) {
    h->err = h->mlp->err;
    return s;
  }
  *cost = c;
  if (h0) *h0 = hh;
  return CHEM_OK;
}

void chem_internal_release_learned(chem_handle h) { h->mlp = nullptr; }
