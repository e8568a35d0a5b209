// Handle definition and internal hooks shared by the host translation units.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "chem.h"
#include "chem_internal.h"

struct chem_mlp_s;

struct chem_handle_s {
  int device = 0;
  int num_sms = 1;
  int K = 0;
  int I = 0;       // reactions as stored on the device (kind groups padded to 32)
  int I_user = 0;  // reactions of the caller's mechanism
  chem::DevMech dm{};
  void* d_tables = nullptr;
  std::vector<int> rxn_order;       // sorted reaction position -> caller's reaction index
  std::vector<void*> allocations;   // every other device allocation of the handle
  // options
  int precision = chem::PREC_FP64;
  int ir_sweeps = 1;
  int scheduler = chem::SCHED_QUEUE;
  int order = 0;
  int h0mode = 0;
  int max_steps = 100000;
  int block = 0;  // 0: chosen per call by chem_internal_pick_block
  int last_block = 0;  // threads per CTA of the last integration launch (option "last_block", read-only)
  int ctas_per_sm = 0;
  int graph = 0;
  int autotune = 0;
  int profile = 0;
  unsigned long long* d_phase = nullptr;  // [8] per-phase cycle counters (option "profile")
  double* d_m0 = nullptr;                 // per-CTA slots of the mixed form's assembled matrix
  size_t m0_cap = 0;                      // bytes
  int time_kernel = 0;                    // option "time_kernel": events around the integration launch
  int jac_fd = 0;                         // option "jacobian": 1 = forward differences (FP64 form)
  int pivoting = 1;                       // option "pivoting": 0 = no row interchanges (FP64 form)
  int job_launch = 0;                     // option "job_launch": 1 = one launch per job, concurrent streams
  int method = 0;                         // option "method": 0 = RODAS4, 1 = ROS34PW2 (W-method)
  int h0_guard = 1;                       // option "h0_guard": envelope check of supplied initial steps
  int h0_range = 10;                      // option "h0_range": learned h0 only within +-h0_range sd (0: off)
  cudaStream_t side = nullptr;            // the handle's stream for concurrent jobs
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t kev0 = nullptr, kev1 = nullptr;
  bool kev_recorded = false;
  // per-cell statistics of the last call
  int64_t stats_cap = 0;
  int64_t last_n = 0;
  int64_t noalloc_n = -1;  // cells of the last call when it was chem_integrate_noalloc, else -1
  int32_t* d_sub = nullptr;
  int32_t* d_rej = nullptr;
  int32_t* d_status = nullptr;
  double* d_hfirst = nullptr;
  double* d_hlast = nullptr;  // controller's proposal after each cell's last step (option h0 = 2)
  bool hlast_valid = false;
  int64_t hlast_n = 0;
  float* d_cost = nullptr;  // substeps of the last call, for cost ordering
  bool cost_valid = false;
  int64_t cost_n = 0;
  void* d_queue = nullptr;
  // staging buffers of chem_integrate_host
  void* d_stage = nullptr;
  int64_t stage_cap = 0;
  // learned scheduling / initial step
  chem_mlp_s* mlp = nullptr;        // model attached with chem_mlp_attach (not owned)
  void* d_order = nullptr;          // permutation + sort scratch
  int64_t order_cap = 0;
  void* d_h0 = nullptr;             // predicted initial steps
  int64_t h0_cap = 0;
  // CUDA graph cache
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned char> gkey;
  // reference mapping by mixture fraction (chem_set_reference_mapping)
  std::vector<int> elem_host;     // [K][n_elem] atom counts kept from chem_create
  std::vector<double> W_host;     // [K] molar masses
  int n_elem = 0;
  bool rm_streams = false;        // fuel / oxidiser streams defined
  bool refmap = false;            // mapping on
  double rm_beta_o = 0.0, rm_dbeta = 1.0;  // beta of the oxidiser; beta_fuel - beta_ox
  double rm_Zc = 0.0, rm_Ztol = -1.0, rm_Ttol = 0.0;
  double* d_rm_b = nullptr;       // [K] Bilger coefficients b_k
  void* d_rm_misc = nullptr;      // reference index, info[2] (mapped count, reference), ref0[K+1]
  void* d_rm_flag = nullptr;      // [cap] int32: zone flags, then mapped flags
  void* d_rm_perm = nullptr;      // [cap] int32: partitioned work order
  void* d_rm_tiles = nullptr;     // [cap / 1024] tile counts / offsets
  int64_t rm_cap = 0;
  int64_t rm_last_n = -1;         // cells of the last mapped call (-1: last call unmapped)
  bool queue_preset = false;      // the next launch keeps the queue's start (set by the mapping)
  // autotuner cache: key -> (block, resident CTAs per SM, matrix layout)
  long long autotuned_key = -1;
  int autotuned_block = 128;
  int autotuned_ctas = 0;   // 0: as many as fit
  int autotuned_m0g = -1;   // mixed form's assembled matrix: 0 shared memory, 1 global slot, -1 automatic
  std::string err;
};

// dt, rtol, atol outside the accepted range (dt > 0, rtol > 0, atol >= 0, all finite)
inline bool chem_internal_bad_tol(double dt, double rtol, double atol) {
  return !(dt > 0.0) || !std::isfinite(dt) || !(rtol > 0.0) || !std::isfinite(rtol) || !(atol >= 0.0) ||
         !std::isfinite(atol);
}

// Device arrays holding the per-cell statistics of a handle's last call: its own
// buffers, or the allocation-free entry point's fixed array after a call of that
// entry point (the array's current contents: the last such call on the device).
struct chem_stats_view {
  int64_t n;
  const int32_t *substeps, *rejects, *status;
  const double* h_first;
};
chem_status chem_internal_stats_view(chem_handle h, chem_stats_view* v);
chem_status chem_internal_noalloc_stats(chem_handle h, int64_t n, chem_stats_view* v);

chem_status chem_internal_alloc(chem_handle h, void* pp, size_t bytes);
chem_status chem_internal_integrate(const chem_job* jobs, int32_t n_jobs, double dt, double rtol, double atol,
                                    cudaStream_t st);
chem_status chem_internal_launch(chem_handle h, const chem::IntegrateArgs& a, int block, int grid,
                                 cudaStream_t st);
int chem_internal_pick_block(chem_handle h, int K, int I, bool allow_m0_global = false);
chem_status chem_internal_graph_launch(chem_handle h, const chem::IntegrateArgs& a, int block, int grid,
                                       cudaStream_t st);
chem_status chem_internal_autotune(chem_handle h, const chem::IntegrateArgs& a, cudaStream_t st, int* block,
                                   int* ctas, int* m0g);
chem_status chem_internal_prepare_learned(chem_handle h, const chem_job* jobs, int32_t n_jobs,
                                          chem::IntegrateArgs* a, cudaStream_t st);
void chem_internal_release_learned(chem_handle h);
chem_status chem_internal_refmap_prepare(chem_handle h, const chem_job& job, chem::IntegrateArgs* a,
                                         cudaStream_t st);
chem_status chem_internal_refmap_apply(chem_handle h, const chem_job& job, cudaStream_t st);
