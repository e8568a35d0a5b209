// Reference mapping by Bilger's mixture fraction, DLBFoam's zonal mapping (paper,
// Methodology, "DLBFoam: Dynamic load balancing"): a cell whose mixture fraction Z
// lies in a zone is not integrated but takes its solution from a reference cell of
// the same zone. Readings taken here:
//   - zone: |Z - Z_center| <= Z_tol; the reference is the zone cell with the lowest
//     index, and it is integrated like any other cell;
//   - a zone cell other than the reference is mapped when |T - T_ref| <= T_tol
//     (T at the start of the step); the other zone cells are integrated;
//   - a mapped cell receives the reference's change of state over the step,
//     T += T_ref(dt) - T_ref(0) and Y_k += Y_ref,k(dt) - Y_ref,k(0): the reference's
//     reaction rates applied to the cell, which keeps the cell's own element content
//     (and so its Z and sum of Y) when the reference conserves its elements.
//
// Bilger's coupling function beta = 2 Z_C/W_C + Z_H/(2 W_H) - Z_O/W_O of the element
// mass fractions Z_e = sum_k a_ek W_e Y_k / W_k is linear in Y:
//   beta(Y) = sum_k b_k Y_k,   b_k = (2 a_Ck + a_Hk / 2 - a_Ok) / W_k,
// and Z = (beta - beta_ox) / (beta_fuel - beta_ox): 0 in the oxidiser stream, 1 in
// the fuel stream.
//
// Inside chem_integrate, on the caller's stream (nothing returns to the host):
//   k_rm_zone     one warp per cell: Z and the zone flag; the reference index by an
//                 unsigned atomicMin over zone cells (initialised to all ones)
//   k_rm_count    per 1024-item tile of the work order: the mapped flags, the
//                 number of integrated cells of the tile
//   k_rm_scan     one CTA: exclusive tile offsets, the number of mapped cells (the
//                 work queue's start), a copy of the reference's initial state
//   k_rm_scatter  stable partition of the work order, mapped cells first
//   (integration kernel: its queue starts past the mapped cells, which it never sees)
//   k_rm_apply    one warp per mapped cell: the reference's change and the cell's
//                 statistics (0 substeps, the reference's status and last step)

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "chem.h"
#include "chem_capi_internal.h"
#include "chem_internal.h"

using namespace chem;

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kTile = 1024;        // work items per partition tile
constexpr int kTileThreads = 256;  // four consecutive items a thread
constexpr int kZoneThreads = 256;  // eight cells a CTA in k_rm_zone / k_rm_apply

// Z of every cell; with `flag`, also the zone flag and the reference candidate.
__global__ void __launch_bounds__(kZoneThreads) k_rm_zone(int64_t n, int K, const double* __restrict__ Y,
                                                          const double* __restrict__ b, double beta_o,
                                                          double dbeta, double Zc, double Ztol,
                                                          double* __restrict__ Z, int32_t* __restrict__ flag,
                                                          unsigned* __restrict__ ref) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < n; c += nw) {
    const double* y = Y + c * K;
    double s = 0.0;
    for (int k = lane; k < K; k += 32) s = fma(b[k], y[k], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane == 0) {
      const double z = (s - beta_o) / dbeta;
      if (Z) Z[c] = z;
      if (flag) {
        const bool in = fabs(z - Zc) <= Ztol;  // false for a NaN Z
        flag[c] = in ? 1 : 0;
        if (in) atomicMin(ref, (unsigned)c);
      }
    }
  }
}

// Per tile of the work order: zone flag -> mapped flag, integrated cells counted.
__global__ void __launch_bounds__(kTileThreads) k_rm_count(int64_t n, const int* __restrict__ perm,
                                                           int32_t* __restrict__ flag,
                                                           const double* __restrict__ T,
                                                           const unsigned* __restrict__ ref, double Ttol,
                                                           int* __restrict__ tile_cnt) {
  __shared__ int s_cnt[kTileThreads / 32];
  const unsigned r = *ref;
  const bool has_ref = (int64_t)r < n;
  const double Tr = has_ref ? T[r] : 0.0;
  const int64_t t0 = (int64_t)blockIdx.x * kTile + 4 * threadIdx.x;
  int cnt = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t w = t0 + e;
    if (w < n) {
      const int64_t g = perm ? perm[w] : w;
      int m = flag[g];
      if (m) m = has_ref && g != (int64_t)r && fabs(T[g] - Tr) <= Ttol;
      flag[g] = m;  // each cell appears once in the work order
      cnt += !m;
    }
  }
  cnt = __reduce_add_sync(kFull, cnt);
  if ((threadIdx.x & 31) == 0) s_cnt[threadIdx.x >> 5] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int i = 0; i < kTileThreads / 32; ++i) s += s_cnt[i];
    tile_cnt[blockIdx.x] = s;
  }
}

// Inclusive scan over the 32 lanes of a warp.
__device__ int warp_scan(int x, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// One CTA of 1024 threads: tile counts -> exclusive offsets; queue start; reference state.
__global__ void __launch_bounds__(1024) k_rm_scan(int n_tiles, int64_t n, int K, int* __restrict__ tile_cnt,
                                                  int* __restrict__ queue, int* __restrict__ info,
                                                  const unsigned* __restrict__ ref,
                                                  const double* __restrict__ T, const double* __restrict__ Y,
                                                  double* __restrict__ ref0) {
  __shared__ int s_w[32];
  __shared__ int s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n_tiles; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < n_tiles ? tile_cnt[i] : 0;
    const int x = warp_scan(v, lane);
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) s_w[lane] = warp_scan(s_w[lane], lane);
    __syncthreads();
    const int excl = s_carry + (warp ? s_w[warp - 1] : 0) + x - v;
    if (i < n_tiles) tile_cnt[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = excl + v;
    __syncthreads();
  }
  const unsigned r = *ref;
  const bool has_ref = (int64_t)r < n;
  if (threadIdx.x == 0) {
    const int n_mapped = (int)(n - s_carry);
    *queue = n_mapped;  // the integration kernel's first work item
    info[0] = n_mapped;
    info[1] = has_ref ? (int)r : -1;
  }
  if (has_ref)
    for (int k = threadIdx.x; k <= K; k += 1024) ref0[k] = k == 0 ? T[r] : Y[(int64_t)r * K + k - 1];
}

// Stable partition of the work order: mapped cells to the front, integrated cells after.
__global__ void __launch_bounds__(kTileThreads) k_rm_scatter(int64_t n, const int* __restrict__ perm,
                                                             const int32_t* __restrict__ flag,
                                                             const int* __restrict__ tile_off,
                                                             const int* __restrict__ info, int* __restrict__ out) {
  __shared__ int s_w[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * kTile + 4 * threadIdx.x;
  int g[4];
  bool sol[4];
  int cnt = 0;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t w = t0 + e;
    g[e] = w < n ? (perm ? perm[w] : (int)w) : -1;
    sol[e] = w < n && !flag[g[e]];
    cnt += sol[e];
  }
  const int x = warp_scan(cnt, lane);
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) s_w[lane] = warp_scan(lane < kTileThreads / 32 ? s_w[lane] : 0, lane);
  __syncthreads();
  int64_t before = (int64_t)tile_off[blockIdx.x] + (warp ? s_w[warp - 1] : 0) + x - cnt;  // integrated before t0
  const int64_t n_mapped = info[0];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t w = t0 + e;
    if (w >= n) break;
    if (sol[e]) {
      out[n_mapped + before] = g[e];
      ++before;
    } else {
      out[w - before] = g[e];
    }
  }
}

// After the integration: mapped cells take the reference's change over the step.
__global__ void __launch_bounds__(kZoneThreads) k_rm_apply(int64_t n, int K, const int32_t* __restrict__ flag,
                                                           const int* __restrict__ info,
                                                           const double* __restrict__ ref0, double* T, double* Y,
                                                           CellStats st, float* __restrict__ cost) {
  const int r = info[1];
  if (r < 0 || info[0] == 0) return;
  const int rstat = st.status ? st.status[r] : (int)CHEM_CELL_OK;
  const bool ok = rstat == CHEM_CELL_OK;
  const double dT = T[r] - ref0[0];
  const double hl = st.h_last ? st.h_last[r] : 0.0;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = w0; c < n; c += nw) {
    if (!flag[c]) continue;
    if (ok) {
      for (int k = lane; k < K; k += 32) Y[c * K + k] += Y[(int64_t)r * K + k] - ref0[1 + k];
    }
    if (lane == 0) {
      if (ok) T[c] += dT;
      if (st.substeps) st.substeps[c] = 0;
      if (st.rejects) st.rejects[c] = 0;
      if (st.h_first) st.h_first[c] = 0.0;
      if (st.status) st.status[c] = rstat;
      if (st.h_last) st.h_last[c] = ok ? hl : 0.0;
      if (cost) cost[c] = 0.0f;
    }
  }
}

int grid_warps(chem_handle h, int64_t n) {
  const int64_t want = (n + kZoneThreads / 32 - 1) / (kZoneThreads / 32);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)h->num_sms * 16));
}

chem_status fail(chem_handle h, const char* what, cudaError_t e) {
  h->err = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  return e == cudaErrorMemoryAllocation ? CHEM_ERR_OOM : CHEM_ERR_CUDA;
}

void release_rm(chem_handle h, void*& p) {
  if (!p) return;
  auto it = std::find(h->allocations.begin(), h->allocations.end(), p);
  if (it != h->allocations.end()) h->allocations.erase(it);
  cudaFree(p);
  p = nullptr;
}

// Buffers for n cells: flags, partitioned order, tile counts.
chem_status ensure_buffers(chem_handle h, int64_t n) {
  chem_status s;
  if (!h->d_rm_misc) {
    // ref (unsigned) and info[2] in the first 16 bytes, then ref0[K+1] doubles
    if ((s = chem_internal_alloc(h, &h->d_rm_misc, 16 + (size_t)(h->K + 1) * sizeof(double))) != CHEM_OK)
      return s;
  }
  if (n <= h->rm_cap) return CHEM_OK;
  cudaDeviceSynchronize();
  release_rm(h, h->d_rm_flag);
  release_rm(h, h->d_rm_perm);
  release_rm(h, h->d_rm_tiles);
  h->rm_cap = 0;
  const int64_t cap = std::max<int64_t>(n, 1024);
  if ((s = chem_internal_alloc(h, &h->d_rm_flag, (size_t)cap * 4)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_rm_perm, (size_t)cap * 4)) != CHEM_OK) return s;
  if ((s = chem_internal_alloc(h, &h->d_rm_tiles, (size_t)((cap + kTile - 1) / kTile) * 4)) != CHEM_OK) return s;
  h->rm_cap = cap;
  return CHEM_OK;
}

}  // namespace

// Called by chem_internal_integrate after the work order is fixed and before the
// integration launch: classifies the cells, moves the mapped ones to the front of
// the work order and sets the queue's start past them.
chem_status chem_internal_refmap_prepare(chem_handle h, const chem_job& job, IntegrateArgs* a, cudaStream_t st) {
  const int64_t n = job.n_cells;
  chem_status s = ensure_buffers(h, n);
  if (s != CHEM_OK) return s;
  unsigned* ref = static_cast<unsigned*>(h->d_rm_misc);
  int* info = reinterpret_cast<int*>(static_cast<unsigned char*>(h->d_rm_misc) + 4);
  double* ref0 = reinterpret_cast<double*>(static_cast<unsigned char*>(h->d_rm_misc) + 16);
  int32_t* flag = static_cast<int32_t*>(h->d_rm_flag);
  int* out = static_cast<int*>(h->d_rm_perm);
  int* tiles = static_cast<int*>(h->d_rm_tiles);
  const int n_tiles = (int)((n + kTile - 1) / kTile);
  cudaError_t e = cudaMemsetAsync(ref, 0xff, sizeof(unsigned), st);
  if (e != cudaSuccess) return fail(h, "reference mapping", e);
  k_rm_zone<<<grid_warps(h, n), kZoneThreads, 0, st>>>(n, h->K, job.Y, h->d_rm_b, h->rm_beta_o, h->rm_dbeta,
                                                        h->rm_Zc, h->rm_Ztol, nullptr, flag, ref);
  k_rm_count<<<n_tiles, kTileThreads, 0, st>>>(n, a->perm, flag, job.T, ref, h->rm_Ttol, tiles);
  k_rm_scan<<<1, 1024, 0, st>>>(n_tiles, n, h->K, tiles, a->queue, info, ref, job.T, job.Y, ref0);
  k_rm_scatter<<<n_tiles, kTileThreads, 0, st>>>(n, a->perm, flag, tiles, info, out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(h, "reference mapping", e);
  a->perm = out;
  h->queue_preset = true;
  h->rm_last_n = n;
  return CHEM_OK;
}

// Called after the integration launch (same stream).
chem_status chem_internal_refmap_apply(chem_handle h, const chem_job& job, cudaStream_t st) {
  const int64_t n = job.n_cells;
  const int* info = reinterpret_cast<const int*>(static_cast<unsigned char*>(h->d_rm_misc) + 4);
  const double* ref0 = reinterpret_cast<const double*>(static_cast<unsigned char*>(h->d_rm_misc) + 16);
  CellStats cs{h->d_sub, h->d_rej, h->d_hfirst, h->d_status, h->d_hlast};
  k_rm_apply<<<grid_warps(h, n), kZoneThreads, 0, st>>>(n, h->K, static_cast<const int32_t*>(h->d_rm_flag), info,
                                                         ref0, job.T, job.Y, cs, h->d_cost);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHEM_OK : fail(h, "reference mapping", e);
}

extern "C" chem_status chem_set_reference_mapping(chem_handle h, int32_t elem_C, int32_t elem_H, int32_t elem_O,
                                                  const double* Y_fuel, const double* Y_ox, double Z_center,
                                                  double Z_tol, double T_tol) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  const int K = h->K, E = h->n_elem;
  auto bad = [&](const char* m) {
    h->err = std::string("chem_set_reference_mapping: ") + m;
    return CHEM_ERR_INVALID_ARG;
  };
  if (std::isnan(Z_tol)) return bad("Z_tol is NaN");
  if (Z_tol < 0.0) {  // mapping off; the stream definitions are kept
    h->refmap = false;
    return CHEM_OK;
  }
  if (!std::isfinite(Z_tol) || !std::isfinite(Z_center) || !std::isfinite(T_tol) || T_tol < 0.0)
    return bad("Z_center, Z_tol and T_tol must be finite, T_tol >= 0");
  if (!Y_fuel || !Y_ox) return bad("NULL stream composition");
  const int cols[3] = {elem_C, elem_H, elem_O};
  bool any = false;
  for (int c : cols) {
    if (c < -1 || c >= E) return bad("element column out of range");
    any = any || c >= 0;
  }
  if (!any) return bad("none of carbon, hydrogen, oxygen given");
  std::vector<double> b(K);
  const double w[3] = {2.0, 0.5, -1.0};  // Bilger's weights of C, H, O atoms per mole
  for (int k = 0; k < K; ++k) {
    double atoms = 0.0;
    for (int i = 0; i < 3; ++i)
      if (cols[i] >= 0) atoms += w[i] * h->elem_host[(size_t)k * E + cols[i]];
    b[k] = atoms / h->W_host[k];
  }
  double bf = 0.0, bo = 0.0;
  for (int k = 0; k < K; ++k) {
    if (!std::isfinite(Y_fuel[k]) || !std::isfinite(Y_ox[k])) return bad("non-finite stream composition");
    bf += b[k] * Y_fuel[k];
    bo += b[k] * Y_ox[k];
  }
  const double db = bf - bo;
  if (!(std::fabs(db) > 0.0) || !std::isfinite(db)) return bad("fuel and oxidiser streams have the same beta");
  if (!h->d_rm_b) {
    chem_status s = chem_internal_alloc(h, &h->d_rm_b, (size_t)K * sizeof(double));
    if (s != CHEM_OK) return s;
  }
  cudaError_t e = cudaMemcpy(h->d_rm_b, b.data(), (size_t)K * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(h, "chem_set_reference_mapping", e);
  h->rm_streams = true;
  h->refmap = true;
  h->rm_beta_o = bo;
  h->rm_dbeta = db;
  h->rm_Zc = Z_center;
  h->rm_Ztol = Z_tol;
  h->rm_Ttol = T_tol;
  h->rm_last_n = -1;
  return CHEM_OK;
}

extern "C" chem_status chem_eval_mixture_fraction(chem_handle h, int64_t n_cells, const double* Y, double* Z,
                                                  void* stream) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (n_cells < 0 || (n_cells > 0 && (!Y || !Z))) {
    h->err = "chem_eval_mixture_fraction: n_cells < 0 or NULL array";
    return CHEM_ERR_INVALID_ARG;
  }
  if (!h->rm_streams) {
    h->err = "chem_eval_mixture_fraction: no fuel/oxidiser streams (chem_set_reference_mapping)";
    return CHEM_ERR_INVALID_ARG;
  }
  if (n_cells == 0) return CHEM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_rm_zone<<<grid_warps(h, n_cells), kZoneThreads, 0, st>>>(n_cells, h->K, Y, h->d_rm_b, h->rm_beta_o,
                                                              h->rm_dbeta, 0.0, 0.0, Z, nullptr, nullptr);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHEM_OK : fail(h, "chem_eval_mixture_fraction", e);
}

extern "C" chem_status chem_get_reference_mapping(chem_handle h, void* stream, int32_t* mapped, int64_t* n_mapped,
                                                  int64_t* ref_cell) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (h->rm_last_n < 0) {
    h->err = "chem_get_reference_mapping: the last integration ran without reference mapping";
    return CHEM_ERR_INVALID_ARG;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int info[2] = {0, -1};
  cudaError_t e = cudaMemcpyAsync(info, static_cast<unsigned char*>(h->d_rm_misc) + 4, sizeof info,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && mapped && h->rm_last_n > 0)
    e = cudaMemcpyAsync(mapped, h->d_rm_flag, (size_t)h->rm_last_n * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(h, "chem_get_reference_mapping", e);
  if (n_mapped) *n_mapped = info[0];
  if (ref_cell) *ref_cell = info[1];
  return CHEM_OK;
}
