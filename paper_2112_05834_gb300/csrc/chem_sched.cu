// Scheduling around the integration kernel: cost ordering of the work queue
// (counting sort of cells by cost, heaviest first), CUDA-graph capture of the
// launch sequence, and the block-size autotuner.
//
// This replaces DLBFoam's MPI redistribution of cell problems (paper:
// Methodology, "DLBFoam: Dynamic load balancing"): instead of moving problems
// from busy to idle ranks, persistent CTAs pull cells from one device counter,
// and the queue starts with the most expensive tenth of the cells, heaviest
// first, so no expensive cell is left for the tail of the launch; the rest keep
// their index order (sorting them as well measured slower than leaving the
// bulk of the batch mixed).

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "chem.h"
#include "chem_capi_internal.h"
#include "chem_internal.h"
#include "chem_kernels.h"
#include "chem_mlp_internal.h"

using namespace chem;

namespace {

constexpr int kBuckets = 256;

// Bucket of a cost value: 32 buckets per factor of 2... mapped heaviest first.
__device__ __forceinline__ int cost_bucket(float c) {
  if (!(c > 0.0f)) c = 0.0f;
  float l = log2f(1.0f + c) * 16.0f;  // 16 buckets per octave
  int b = (int)l;
  b = b < 0 ? 0 : (b > kBuckets - 1 ? kBuckets - 1 : b);
  return kBuckets - 1 - b;  // descending cost
}

__global__ void k_hist(const float* cost, int64_t n, int* hist) {
  __shared__ int sh[kBuckets];
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&sh[cost_bucket(cost[i])], 1);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Heaviest share of the cells that is ordered by cost; the rest keeps index order.
constexpr float kHeavyShare = 0.1f;

__global__ void k_scan(int* hist, int64_t n) {
  // single block of kBuckets threads: exclusive prefix sum in place; hist[kBuckets]
  // receives the last bucket of the heavy share (its inclusive sum reaches the share)
  __shared__ int sh[kBuckets];
  const int t = threadIdx.x;
  sh[t] = hist[t];
  __syncthreads();
  for (int o = 1; o < kBuckets; o <<= 1) {
    int v = t >= o ? sh[t - o] : 0;
    __syncthreads();
    sh[t] += v;
    __syncthreads();
  }
  hist[t] = t == 0 ? 0 : sh[t - 1];
  const long long share = (long long)(kHeavyShare * (float)n) > 0 ? (long long)(kHeavyShare * (float)n) : 1;
  const bool reach = sh[t] >= share, before = t > 0 && sh[t - 1] >= share;
  if (reach && !before) hist[kBuckets] = t;
}

__global__ void k_scatter(const float* cost, int64_t n, int* offs, int* perm) {
  const int last = offs[kBuckets];  // buckets after it form one index-ordered group
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int b = cost_bucket(cost[i]);
    if (b > last) b = last + 1;
    const int pos = atomicAdd(&offs[b], 1);
    perm[pos] = (int)i;
  }
}

}  // namespace

// perm[0..n): the heaviest tenth of the cells by decreasing cost, then the others
// (order within a cost bucket and within the others set by the scatter's atomics).
chem_status chem_internal_cost_order(chem_handle h, const float* d_cost, int64_t n, cudaStream_t st,
                                     const int** perm_out) {
  if (n > h->order_cap) {
    cudaStreamSynchronize(st);
    if (h->d_order) {
      auto it = std::find(h->allocations.begin(), h->allocations.end(), h->d_order);
      if (it != h->allocations.end()) h->allocations.erase(it);
      cudaFree(h->d_order);
      h->d_order = nullptr;
    }
    chem_status s = chem_internal_alloc(h, &h->d_order, (size_t)n * 4 + (kBuckets + 1) * 4);
    if (s != CHEM_OK) return s;
    h->order_cap = n;
  }
  int* perm = static_cast<int*>(h->d_order);
  int* hist = perm + h->order_cap;
  cudaMemsetAsync(hist, 0, (kBuckets + 1) * 4, st);
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * (int64_t)h->num_sms);
  k_hist<<<grid, 256, 0, st>>>(d_cost, n, hist);
  k_scan<<<1, kBuckets, 0, st>>>(hist, n);
  k_scatter<<<grid, 256, 0, st>>>(d_cost, n, hist, perm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("cost order: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  *perm_out = perm;
  return CHEM_OK;
}

chem_status chem_internal_prepare_learned(chem_handle h, const chem_job* jobs, int32_t n_jobs, IntegrateArgs* a,
                                          cudaStream_t st) {
  if (h->order == 0 && h->h0mode != 1) return CHEM_OK;
  if (n_jobs != 1) {
    h->err = "order/h0 options apply to single-mechanism calls";
    return CHEM_ERR_INVALID_ARG;
  }
  const int64_t n = jobs[0].n_cells;
  const float* cost = nullptr;
  if (h->order == 1 || h->h0mode == 1) {
    if (!h->mlp) {
      h->err = "learned order/h0 requested but no trained model is attached (chem_mlp_attach)";
      return CHEM_ERR_INVALID_ARG;
    }
    chem_status s = chem_internal_mlp_predict(h, jobs[0].T, jobs[0].p, jobs[0].Y, n, st, &cost,
                                              h->h0mode == 1 ? &a->jobs[0].h0 : nullptr);
    if (s != CHEM_OK) return s;
    a->use_h0 = h->h0mode == 1;
  }
  if (h->order == 2) {
    if (!h->cost_valid || h->cost_n != n) {
      // no previous cost of this size yet: index order this time
      cost = nullptr;
    } else {
      // snapshot: the kernel overwrites d_cost while running
      cost = h->d_cost;
    }
  }
  if (h->order != 0 && cost) {
    const int* perm = nullptr;
    float* snap = nullptr;
    if (h->order == 2) {
      // copy the previous cost aside, the running kernel writes the new one
      chem_status s = chem_internal_learned_buffers(h, n, nullptr, nullptr, &snap);
      if (s != CHEM_OK) return s;
      cudaMemcpyAsync(snap, cost, n * 4, cudaMemcpyDeviceToDevice, st);
      cost = snap;
    }
    chem_status s = chem_internal_cost_order(h, cost, n, st, &perm);
    if (s != CHEM_OK) return s;
    a->perm = perm;
  }
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// CUDA graph of the launch sequence (queue reset + integration kernel)
// ---------------------------------------------------------------------------
chem_status chem_internal_graph_launch(chem_handle h, const IntegrateArgs& a, int block, int grid,
                                       cudaStream_t st) {
  std::vector<unsigned char> key(sizeof(IntegrateArgs) + 4 * sizeof(int));
  std::memcpy(key.data(), &a, sizeof(IntegrateArgs));
  int extra[4] = {block, grid, h->precision, h->queue_preset ? 1 : 0};
  std::memcpy(key.data() + sizeof(IntegrateArgs), extra, sizeof extra);
  if (!h->gexec || key != h->gkey) {
    if (h->gexec) {
      cudaGraphExecDestroy(h->gexec);
      h->gexec = nullptr;
    }
    if (!h->cap_stream) {
      cudaError_t e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
      if (e != cudaSuccess) {
        h->err = std::string("graph stream: ") + cudaGetErrorString(e);
        return CHEM_ERR_CUDA;
      }
    }
    int occ = 0;
    occupancy_integrate(block, h->precision, a.smem_K, a.smem_I, &occ, a.m0_scratch != nullptr);  // sets kernel attributes
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess && a.sched == SCHED_QUEUE && !h->queue_preset)
      e = cudaMemsetAsync(a.queue, 0, sizeof(int), h->cap_stream);
    if (e == cudaSuccess) e = launch_integrate(a, block, h->precision, grid, h->cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(h->cap_stream, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&h->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      h->err = std::string("graph capture: ") + cudaGetErrorString(e);
      return CHEM_ERR_CUDA;
    }
    h->gkey = key;
  }
  cudaError_t e = cudaGraphLaunch(h->gexec, st);
  if (e != cudaSuccess) {
    h->err = std::string("graph launch: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time the block sizes on a sample of the call's cells (copies, the
// caller's arrays are not touched) and keep the fastest. Results are cached in
// the handle and, when the environment variable CHEM_AUTOTUNE_CACHE names a
// file, in that file (one "key block" pair per line).
// ---------------------------------------------------------------------------
static long long tune_key(const chem_handle h, const IntegrateArgs& a) {
  long long n_bucket = (long long)std::log2((double)std::max<int64_t>(a.n_total, 1));
  return ((long long)a.smem_K << 40) ^ ((long long)a.smem_I << 24) ^ ((long long)h->precision << 20) ^
         ((long long)a.sched << 16) ^ n_bucket;
}

static bool cache_lookup(long long key, int* block, int* ctas, int* m0g) {
  const char* path = std::getenv("CHEM_AUTOTUNE_CACHE");
  if (!path) return false;
  std::ifstream f(path);
  long long k;
  int b, c, g;
  while (f >> k >> b >> c >> g)
    if (k == key && (b == 64 || b == 128 || b == 256) && c >= 0 && g >= -1 && g <= 1) {
      *block = b;
      *ctas = c;
      *m0g = g;
      return true;
    }
  return false;
}

static void cache_store(long long key, int block, int ctas, int m0g) {
  const char* path = std::getenv("CHEM_AUTOTUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << " " << block << " " << ctas << " " << m0g << "\n";
}

// Candidates: CTA size (2, 4 or 8 warps on one cell) x matrix layout of the mixed form
// (assembled matrix in shared memory, or in a per-CTA global slot, which leaves room
// for more CTAs) x resident CTAs per SM on persistent grids (as many as fit, or one
// fewer: fewer CTAs compete for the SM's FP64 pipe and issue slots). Each is timed on a
// sample of the call's cells (copies; the caller's arrays are not touched), one warm-up
// and one timed launch, and the fastest is kept: *block, *ctas (0 = as many as fit) and
// *m0g (-1 unless the layout was a choice).
chem_status chem_internal_autotune(chem_handle h, const IntegrateArgs& a, cudaStream_t st, int* block, int* ctas,
                                   int* m0g) {
  const long long key = tune_key(h, a);
  if (h->autotuned_key == key) {
    *block = h->autotuned_block;
    *ctas = h->autotuned_ctas;
    *m0g = h->autotuned_m0g;
    return CHEM_OK;
  }
  int cb = 0, cc = 0, cg = -1;
  if (cache_lookup(key, &cb, &cc, &cg)) {
    h->autotuned_key = key;
    h->autotuned_block = *block = cb;
    h->autotuned_ctas = *ctas = cc;
    h->autotuned_m0g = *m0g = cg;
    return CHEM_OK;
  }
  if (a.n_jobs != 1 || a.perm) return CHEM_OK;  // tune single-job, index-ordered calls only (keep *block)
  const Job& J = a.jobs[0];
  const int64_t S = std::min<int64_t>(J.n_cells, 4 * 1024);
  const int K = J.m.K;
  const bool persistent = a.sched != SCHED_PLAIN;
  const bool layouts = persistent && h->precision == PREC_MIXED;
  // candidates and the largest grid any of them needs (for the matrix slots)
  struct Cand { int b, g, c; };
  std::vector<Cand> cands;
  int64_t max_grid = 1;
  for (int b : {64, 128, 256})
    for (int g = 0; g <= (layouts ? 1 : 0); ++g) {
      int occ = 0;
      if (occupancy_integrate(b, h->precision, a.smem_K, a.smem_I, &occ, g == 1) != cudaSuccess) {
        cudaGetLastError();
        continue;
      }
      if (occ < 1) continue;
      for (int c = occ; c >= (persistent ? std::max(1, occ - 1) : occ); --c) {
        cands.push_back({b, g, c});
        max_grid = std::max<int64_t>(max_grid, std::min<int64_t>(S, (int64_t)c * h->num_sms));
      }
    }
  if (cands.empty()) return CHEM_OK;
  const int64_t stride = (int64_t)(a.smem_K + 1) * ((a.smem_K + 1) | 1);
  const size_t sample_doubles = (size_t)S * (K + 2) * 2;
  const size_t slot_doubles = layouts ? (size_t)max_grid * stride : 0;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (sample_doubles + slot_doubles) * sizeof(double));
  if (e != cudaSuccess) {
    h->err = std::string("autotune: ") + cudaGetErrorString(e);
    return CHEM_ERR_OOM;
  }
  double *T0 = buf, *p0 = buf + S, *Y0 = buf + 2 * S;
  double* work = buf + (size_t)S * (K + 2);
  double* slots = buf + sample_doubles;
  cudaMemcpyAsync(T0, J.T, S * 8, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(p0, J.p, S * 8, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(Y0, J.Y, (size_t)S * K * 8, cudaMemcpyDeviceToDevice, st);
  cudaEvent_t ev0, ev1;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  float best = 1e30f;
  Cand best_c{*block, -1, 0};
  for (const Cand& cd : cands) {
    IntegrateArgs t = a;
    t.n_total = S;
    t.jobs[0].n_cells = S;
    t.jobs[0].T = work;
    t.jobs[0].p = work + S;
    t.jobs[0].Y = work + 2 * S;
    t.jobs[0].cost_out = nullptr;
    t.jobs[0].st.h_last = nullptr;  // keep the carried-over steps of the real call intact
    t.jobs[0].h0 = nullptr;
    t.m0_scratch = cd.g == 1 ? slots : nullptr;
    t.m0_stride = cd.g == 1 ? stride : 0;
    const int grid = persistent ? (int)std::min<int64_t>(S, (int64_t)cd.c * h->num_sms) : (int)S;
    float ms_total = 0.0f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaMemcpyAsync(work, T0, (size_t)S * (K + 2) * 8, cudaMemcpyDeviceToDevice, st);
      if (t.sched == SCHED_QUEUE) cudaMemsetAsync(t.queue, 0, sizeof(int), st);
      cudaEventRecord(ev0, st);
      launch_integrate(t, cd.b, h->precision, grid, st);
      cudaEventRecord(ev1, st);
      cudaEventSynchronize(ev1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev0, ev1);
      if (rep == 1) ms_total = ms;  // first run warms up
    }
    if (ms_total < best) {
      best = ms_total;
      best_c = cd;
    }
  }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  cudaStreamSynchronize(st);
  cudaFree(buf);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    h->err = std::string("autotune: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  const int tuned_m0g = layouts ? best_c.g : -1;
  const int tuned_ctas = persistent ? best_c.c : 0;
  h->autotuned_key = key;
  h->autotuned_block = best_c.b;
  h->autotuned_ctas = tuned_ctas;
  h->autotuned_m0g = tuned_m0g;
  cache_store(key, best_c.b, tuned_ctas, tuned_m0g);
  *block = best_c.b;
  *ctas = tuned_ctas;
  *m0g = tuned_m0g;
  return CHEM_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

chem_status chem_internal_learned_buffers(chem_handle h, int64_t n, float** cost, double** h0, float** snap) {
  if (n > h->h0_cap) {
    cudaDeviceSynchronize();
    if (h->d_h0) {
      auto it = std::find(h->allocations.begin(), h->allocations.end(), h->d_h0);
      if (it != h->allocations.end()) h->allocations.erase(it);
      cudaFree(h->d_h0);
      h->d_h0 = nullptr;
    }
    const size_t bytes = align256((size_t)n * 4) * 2 + align256((size_t)n * 8);
    chem_status s = chem_internal_alloc(h, &h->d_h0, bytes);
    if (s != CHEM_OK) return s;
    h->h0_cap = n;
  }
  unsigned char* b = static_cast<unsigned char*>(h->d_h0);
  const size_t c4 = align256((size_t)h->h0_cap * 4), c8 = align256((size_t)h->h0_cap * 8);
  if (cost) *cost = reinterpret_cast<float*>(b);
  if (h0) *h0 = reinterpret_cast<double*>(b + c4);
  if (snap) *snap = reinterpret_cast<float*>(b + c4 + c8);
  return CHEM_OK;
}
