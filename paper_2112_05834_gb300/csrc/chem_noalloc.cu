// chem_integrate_noalloc: the integration entry point for callers that cannot
// allocate device memory.
//
// chem_integrate grows handle-owned buffers on demand (per-cell statistics, the
// work-queue counter, learned-order scratch), which may call cudaMalloc and
// cudaFree. Some callers cannot allow that: applications whose device memory is
// fixed up front by their own pool or budget (a CFD code that reserves the GPU's
// memory for its fields and solvers at start-up, where a late cudaMalloc fails
// or evicts its pool), and callers inside a time-step loop that cannot accept
// the device-wide synchronisation a cudaMalloc/cudaFree may imply while other
// streams are busy.
//
// This variant keeps the scratch of the integration kernel (the work-queue
// counter and the per-cell statistics it writes) in one file-scope device array
// of fixed size instead. Every GPU that loads the library holds that array until
// the process exits. It calls no allocating routine.

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "chem.h"
#include "chem_capi_internal.h"
#include "chem_internal.h"
#include "chem_kernels.h"

#define CHEM_STR2(x) #x
#define CHEM_STR(x) CHEM_STR2(x)

namespace {

// Largest batch this entry point accepts.
constexpr int64_t kMaxCells = CHEM_NOALLOC_MAX_CELLS;
// Layout: [0, 256) queue counter; then substeps, rejects, status (int32 each) and
// h_first (double) per cell, each region 256-byte aligned.
constexpr size_t kCounterBytes = 256;
constexpr size_t kI32Bytes = ((size_t)kMaxCells * 4 + 255) / 256 * 256;
constexpr size_t kF64Bytes = (size_t)kMaxCells * 8;
constexpr size_t kScratchBytes = kCounterBytes + 3 * kI32Bytes + kF64Bytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once per
// device, with that device current). The host-side symbol itself is only a
// stand-in and must never be handed to a kernel.
chem_status scratch_address(chem_handle h, unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    h->err = "chem_integrate_noalloc: no usable current device";
    return CHEM_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      h->err = std::string("chem_integrate_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return CHEM_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return CHEM_OK;
}

}  // namespace

extern "C" chem_status chem_integrate_noalloc(chem_handle h, int64_t n_cells, double* T, const double* p,
                                              double* Y, double dt, double rtol, double atol, void* stream) {
  if (!h) return CHEM_ERR_INVALID_ARG;
  if (n_cells < 0 || (n_cells > 0 && (!T || !p || !Y)) || chem_internal_bad_tol(dt, rtol, atol)) {
    h->err = "chem_integrate_noalloc: invalid argument (n_cells < 0, NULL array, or dt/rtol/atol out of range)";
    return CHEM_ERR_INVALID_ARG;
  }
  if (n_cells > kMaxCells) {
    h->err = "chem_integrate_noalloc: n_cells exceeds the fixed scratch capacity of "
             CHEM_STR(CHEM_NOALLOC_MAX_CELLS) " cells; split the batch or use chem_integrate";
    return CHEM_ERR_INVALID_ARG;
  }
  if (h->refmap) {
    h->err = "chem_integrate_noalloc: reference mapping needs handle-owned buffers; use chem_integrate";
    return CHEM_ERR_INVALID_ARG;
  }
  // from here on the handle's statistics queries read this call's cells from the
  // fixed array; the last-call cost order and carried-over steps of the handle's
  // own buffers no longer describe the cells it was last given
  h->noalloc_n = n_cells;
  h->cost_valid = false;
  h->hlast_valid = false;
  if (n_cells == 0) return CHEM_OK;
  unsigned char* base = nullptr;
  chem_status s = scratch_address(h, &base);
  if (s != CHEM_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  chem::IntegrateArgs a;
  std::memset(&a, 0, sizeof a);
  chem::Job& J = a.jobs[0];
  J.m = h->dm;
  J.n_cells = n_cells;
  J.offset = 0;
  J.T = T;
  J.p = p;
  J.Y = Y;
  J.st.substeps = reinterpret_cast<int32_t*>(base + kCounterBytes);
  J.st.rejects = reinterpret_cast<int32_t*>(base + kCounterBytes + kI32Bytes);
  J.st.status = reinterpret_cast<int32_t*>(base + kCounterBytes + 2 * kI32Bytes);
  J.st.h_first = reinterpret_cast<double*>(base + kCounterBytes + 3 * kI32Bytes);
  J.cost_out = nullptr;
  J.h0 = nullptr;
  a.n_jobs = 1;
  a.n_total = n_cells;
  a.perm = nullptr;  // index order: the learned order needs handle-owned buffers
  a.queue = reinterpret_cast<int*>(base);
  a.dt = dt;
  a.rtol = rtol;
  a.atol = atol;
  a.max_steps = h->max_steps;
  a.sched = h->scheduler;
  a.ir_sweeps = h->ir_sweeps;
  a.jac_fd = h->jac_fd;
  a.no_pivot = h->pivoting ? 0 : 1;
  a.use_h0 = 0;
  a.tab = chem::method_tableau(h->method);
  a.smem_K = h->K;
  a.smem_I = h->I > 0 ? h->I : 1;
  const int block = h->block ? h->block : chem_internal_pick_block(h, a.smem_K, a.smem_I);
  int grid;
  if (a.sched == chem::SCHED_PLAIN) {
    grid = (int)n_cells;
  } else {
    int occ = 0;
    cudaError_t e = chem::occupancy_integrate(block, h->precision, a.smem_K, a.smem_I, &occ);
    if (e != cudaSuccess || occ < 1) {
      h->err = "chem_integrate_noalloc: kernel does not fit on an SM";
      return CHEM_ERR_CUDA;
    }
    if (h->ctas_per_sm > 0 && h->ctas_per_sm < occ) occ = h->ctas_per_sm;
    grid = (int)((int64_t)occ * h->num_sms < n_cells ? (int64_t)occ * h->num_sms : n_cells);
  }
  // the queue counter must start at zero; the statistics are overwritten per cell
  cudaError_t e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
  if (e == cudaSuccess) e = chem::launch_integrate(a, block, h->precision, grid, st);
  if (e != cudaSuccess) {
    h->err = std::string("chem_integrate_noalloc: ") + cudaGetErrorString(e);
    return CHEM_ERR_CUDA;
  }
  return CHEM_OK;
}

chem_status chem_internal_noalloc_stats(chem_handle h, int64_t n, chem_stats_view* v) {
  if (n == 0) {
    *v = chem_stats_view{0, nullptr, nullptr, nullptr, nullptr};
    return CHEM_OK;
  }
  unsigned char* base = nullptr;
  chem_status s = scratch_address(h, &base);
  if (s != CHEM_OK) return s;
  v->n = n;
  v->substeps = reinterpret_cast<const int32_t*>(base + kCounterBytes);
  v->rejects = reinterpret_cast<const int32_t*>(base + kCounterBytes + kI32Bytes);
  v->status = reinterpret_cast<const int32_t*>(base + kCounterBytes + 2 * kI32Bytes);
  v->h_first = reinterpret_cast<const double*>(base + kCounterBytes + 3 * kI32Bytes);
  return CHEM_OK;
}
