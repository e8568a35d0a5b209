// Internal structures shared by the host C-ABI and the device kernels.
#pragma once

#include <vector_types.h>

#include <cstdint>

namespace chem {

struct ff2;

constexpr int kMaxJobs = 8;
constexpr double kRc = 8.31446261815324e7;  // erg / (mol K)
constexpr double kP0 = 1.01325e6;           // dyn / cm^2, standard state (1 atm)
constexpr double kTmin = 200.0, kTmax = 6000.0;
// Largest |G/RT| of a species for which the reverse-rate ratio is formed as a product
// of per-species factors exp(+-G/RT): four factors then stay within e^+-600.
constexpr double kBigGRT = 150.0;

// FP64: everything in FP64.
// MIXED: Jacobian assembled in float-float arithmetic (about 48 bits, FP32 pipe; kept
//        for the refinement residual), FP32 Gauss-Jordan inverse and solves, every
//        solve refined with residuals computed as compensated FP32 dot products.
// FP32ASM: Jacobian assembled in FP32 as well; refinement residual against the
//        FP32-assembled matrix (kept for comparison: it perturbs the method).
enum Precision { PREC_FP64 = 0, PREC_MIXED = 1, PREC_FP32ASM = 2 };
enum Sched { SCHED_PLAIN = 0, SCHED_STATIC = 1, SCHED_QUEUE = 2 };

// Rosenbrock methods of the stepper: RODAS4 (order 4, exact Jacobian) or the
// ROS34PW2 W-method (order 3 for any approximation of the Jacobian).
enum Method { METHOD_RODAS4 = 0, METHOD_ROS34PW2 = 1 };

// A method in the transformed form of the device stepper, u_i = sum_j gamma_ij k_j:
//   (I/(h gamma) - W) u_i = f(y0 + sum_{j<i} a_ij u_j) + sum_{j<i} (c_ij / h) u_j,
//   y1 = y0 + sum m_i u_i, error estimate y1 - yhat = sum e_i u_i.
struct MethodTab {
  int s;       // stages (<= 6)
  int q;       // embedded order + 1: step-size factor err^(-1/q) and starting-step exponent 1/q
  int e_last;  // 1: the error estimate is the last stage's u (e = unit vector)
  double gamma;
  double a[6][6], c[6][6], m[6], e[6];
};

// Reaction kinds after the host sorts reactions by kind (warp-uniform branches).
enum RxnKind { RK_ELEM = 0, RK_TB = 1, RK_LIND = 2, RK_TROE = 3 };

// Device-resident struct-of-arrays tables of one mechanism. Reactions are stored
// sorted by kind; species keep the caller's order.
struct DevMech {
  int K, I;     // I counts null padding reactions (slot 0 = -1): kind groups fill 32-reaction chunks
  int n_chunks;            // I / 32
  // Chunks dealt to the warps of a CTA of 64, 128 or 256 threads (table v = 0, 1, 2):
  // [NW + 1] offsets, then the chunk indices of warp 0, warp 1, ... (NW = 2 << v).
  const int* chunk_sched[3];
  int n_tb;   // reactions with a third-body concentration (kinds 1..3)
  int n_fo;   // falloff reactions (kinds 2, 3)
  int i_tb0;  // first reaction of kind >= 1 (sorted order)
  int i_fo0;  // first reaction of kind >= 2
  int i_troe0;  // first reaction of kind 3
  double T_bigG;  // below this T some species may have |G/RT| > kBigGRT (0: never in [kTmin, kTmax])
  const double* W;      // [K]
  const double* invW;   // [K]
  const struct ff2* invW_ff;  // [K] as float-float pairs (hi, lo)
  const double* nasa;   // [K][36]: for range r (0 below T_mid, 1 above) at 17 r:
                        //   cp/R coefficients a1..a5, H/RT coefficients a1, a2/2, a3/3,
                        //   a4/4, a5/5, a6, S/R coefficients a1, a2, a3/2, a4/3, a5/4, a7;
                        //   [34] = T_mid
  const double* arr;    // [I][4]: ln A, b, Ea_R, dnu
  const int4* slots;    // [I]: reactant slot 0/1, product slot 0/1 species (-1 empty);
                        //      a coefficient of 2 appears as two equal slots
  const int* rev;       // [I] bit 0: reversible; bits 1-2: dnu + 1 (dnu = -1, 0, 1)
  const double* fo;     // [n_fo][8]: ln(A0/A), b0 - b, Ea0_R - Ea_R, alpha, 1/T***, 1/T*, T**, 0
  const double* eff;    // [n_tb][K] (row r belongs to reaction i_tb0 + r)
  const struct ff2* eff_ff;  // the same efficiencies as float-float pairs (hi, lo)
  const double* effT;        // [K][n_tb]: the efficiencies species-major
  const struct ff2* effT_ff;  // the same as float-float pairs
  const int* sp_ptr;    // [K+1] species -> (reaction, nu) CSR
  const int2* sp_ent;
  const double* sp_nu;  // the same nu as doubles
  // Mass-action Jacobian terms A_kj = sum nu_ki dq_i/dC_j, one sum per (row k,
  // column j) pair, dealt to the threads of a CTA of 64, 128 or 256 threads
  // (table v = 0, 1, 2) so that each thread has about as many terms as any other.
  // Entry (r, t) of table v, at r * (64 << v) + t, is thread t's r-th term:
  // x = index 4 i + slot into the per-reaction dq/dC data (-1: padding), y = the
  // matrix offset the finished sum goes to (-1: the pair continues).
  const int2* js_ent[3];
  const double* js_nu[3];  // nu_ki W_k of the term
  const struct ff2* js_nu_ff[3];  // the same as float-float pairs
  int js_rounds[3];
  const unsigned* jmask;   // [K][ceil(K/32)]: bit l of word (k, u) set if pair (k, l + 32 u) exists
  const double* tr_nu;  // nu_ki W_k of the tr_ent entries
  const struct ff2* tr_nu_ff;  // the same as float-float pairs
  const int* tr_ptr;    // [K+1] row k -> (reaction i with [M], nu_ki)
  const int2* tr_ent;
};

struct CellStats {
  int32_t* substeps;
  int32_t* rejects;
  double* h_first;
  int32_t* status;
  double* h_last;  // optional: step size the controller proposes after the cell's last step
};

struct Job {
  DevMech m;
  int64_t n_cells;
  int64_t offset;  // first global work index of this job
  double* T;
  const double* p;
  double* Y;
  CellStats st;
  const double* h0;   // optional per-cell initial step (learned), may be null
  float* cost_out;    // optional per-cell cost (substeps) for the next call's ordering
};

struct IntegrateArgs {
  Job jobs[kMaxJobs];
  int n_jobs;
  int64_t n_total;
  const int* perm;     // optional order of global work indices (queue/plain)
  int* queue;          // device counter (queue scheduler)
  double dt, rtol, atol;
  int max_steps;
  int sched;
  int ir_sweeps;
  int use_h0;          // 1: take jobs[j].h0 when finite and positive
  int h0_guard;        // 1: keep a supplied initial step inside the starting-step envelope
  int jac_fd;          // FP64 form only: 1 = forward-difference Jacobian (n extra RHS evaluations)
  int no_pivot;        // FP64 form only: 1 = Gaussian elimination without row interchanges
  int smem_K, smem_I;  // sizes the shared-memory carve-up was computed for
  unsigned long long* phase;  // optional [8] per-phase cycle counters (diagnostic)
  double* m0_scratch;  // mixed form, persistent grids: per-CTA slots for the assembled matrix
  int64_t m0_stride;   //   (8-byte entries; null: it stays in shared memory); entries per slot
  MethodTab tab;       // the Rosenbrock method
};

// The transformed tableau of a method (host; chem_capi.cu).
MethodTab method_tableau(int method);

}  // namespace chem
