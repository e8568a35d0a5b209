/*
 * chem.h - C ABI of the GB300 batched stiff-chemistry integrator.
 *
 * The library advances, for every cell of a batch, the constant-pressure
 * adiabatic finite-rate kinetics ODE  f = d(phi)/dt  (paper: Introduction,
 * composition vector phi and f = d phi / dt) over one CFD time step dt. Each
 * cell is integrated by an adaptive Rosenbrock method (RODAS4) whose iteration
 * matrix (I/(h gamma) - J) uses the fully analytical Jacobian
 * J_ij = d f_i / d phi_j (paper: Methodology, "Analytical Jacobian and improved
 * ODE solution") and is handled by dense LU decomposition with partial
 * pivoting and forward/back substitution (same section: LU decomposition and
 * back substitution). The uneven per-cell cost that the paper balances across
 * MPI ranks (Methodology, "DLBFoam: Dynamic load balancing") is balanced inside
 * one GPU by a device work queue, optionally ordered by a learned cost model.
 *
 * State vector per cell: y = [T, Y_1 .. Y_K] (K+1 unknowns); p is constant
 * over the step. Units: cgs-molar (mol, cm^3, s, K, erg, dyn/cm^2).
 *
 * Conventions for every entry point:
 *   - Return value: chem_status. CHEM_OK on success; argument errors are
 *     detected before any GPU work and return CHEM_ERR_INVALID_ARG; the message
 *     is available from chem_last_error(handle).
 *   - "device" pointers are CUDA device (or managed) memory of the current
 *     device; "host" pointers are CPU memory (pinned memory makes copies
 *     asynchronous). The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream. Integration calls are stream-ordered and return after enqueueing
 *     unless stated otherwise.
 *   - No entry point aborts the process or traps on the GPU. Per-cell failures
 *     are recorded as per-cell status codes (see chem_cell_status).
 *   - A handle may be used from one host thread / one stream at a time.
 */
#ifndef CHEM_H_
#define CHEM_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chem_handle_s* chem_handle;

typedef enum {
  CHEM_OK = 0,
  CHEM_ERR_INVALID_ARG = 1,
  CHEM_ERR_BAD_MECHANISM = 2,
  CHEM_ERR_CUDA = 3,
  CHEM_ERR_CELLS_FAILED = 4,
  CHEM_ERR_OOM = 5
} chem_status;

/* Per-cell outcome of an integration (chem_get_stats, cell_status array). */
typedef enum {
  CHEM_CELL_OK = 0,          /* reached dt; T recovered from the conserved enthalpy */
  CHEM_CELL_MAX_STEPS = 1,   /* step budget (option "max_steps") exhausted */
  CHEM_CELL_H_UNDERFLOW = 2, /* step size fell below 1e-20 s */
  CHEM_CELL_NONFINITE = 3,   /* non-finite input state */
  CHEM_CELL_T_RANGE = 4      /* final T outside [200, 6000] K */
} chem_cell_status;

/*
 * Reaction mechanism tables (host pointers, copied at chem_create; the caller
 * keeps ownership). K species, I reactions, E elements.
 *   W[K]                 molecular weights, g/mol (must equal sum of atomic masses
 *                        in the caller's convention; checked for positivity)
 *   elem[K][E]           atom counts (int32), used to check that every reaction
 *                        balances every element
 *   nasa_lo/hi[K][7]     NASA-7 coefficients a1..a7 below / above T_mid
 *   T_lo/T_mid/T_hi[K]   validity range and switch temperature, K
 *   rxn_type[I]          0 elementary, 1 third-body (+M), 2 Lindemann, 3 Troe falloff
 *   reac_idx/reac_nu[I][2], prod_idx/prod_nu[I][2]
 *                        up to two distinct species per side with coefficient 1 or
 *                        2 (index -1 = empty slot); total order per side <= 2
 *   reversible[I]        nonzero: reverse rate from the equilibrium constant
 *   A, b, Ea_R [I]       k = A T^b exp(-Ea_R/T) (high-pressure limit for falloff)
 *   A0, b0, Ea0_R [I]    low-pressure limit (falloff only)
 *   troe[I][4]           alpha, T***, T*, T** (T** <= 0: that term absent)
 *   eff[I][K]            third-body efficiencies (read for types 1..3)
 */
typedef struct {
  int32_t n_species, n_reactions, n_elements;
  const double* W;
  const int32_t* elem;
  const double *nasa_lo, *nasa_hi;
  const double *T_lo, *T_mid, *T_hi;
  const int32_t* rxn_type;
  const int32_t *reac_idx, *reac_nu, *prod_idx, *prod_nu;
  const int32_t* reversible;
  const double *A, *b, *Ea_R;
  const double *A0, *b0, *Ea0_R;
  const double* troe;
  const double* eff;
} chem_mechanism_desc;

/*
 * Validates the mechanism (index ranges, coefficients, element balance of every
 * reaction, positive W and Arrhenius prefactors, H/RT and S/R continuity at T_mid
 * within 1e-6), builds the device tables on the current device and returns a
 * handle in *out. Errors: CHEM_ERR_INVALID_ARG (NULL pointers),
 * CHEM_ERR_BAD_MECHANISM (validation; message via chem_last_error(NULL)),
 * CHEM_ERR_CUDA / CHEM_ERR_OOM.
 */
chem_status chem_create(const chem_mechanism_desc* desc, chem_handle* out);

/* Frees the handle and its device memory (synchronises the device first). */
chem_status chem_destroy(chem_handle h);

/*
 * Integrates n_cells cells over [0, dt] at relative/absolute tolerances
 * rtol/atol (weighted RMS norm of the embedded error, scale atol + rtol*|y|).
 *   T[n_cells]          device, in/out: temperature, K
 *   p[n_cells]          device, in: pressure, dyn/cm^2
 *   Y[n_cells][K]       device, in/out: mass fractions, cell-major contiguous
 * A failed cell keeps its last accepted state and records its status; query
 * with chem_get_stats. n_cells == 0 is a no-op. Errors: CHEM_ERR_INVALID_ARG
 * (n_cells < 0, NULL pointers with n_cells > 0, dt <= 0, rtol <= 0, atol < 0,
 * non-finite arguments), CHEM_ERR_CUDA.
 */
chem_status chem_integrate(chem_handle h, int64_t n_cells, double* T, const double* p, double* Y,
                           double dt, double rtol, double atol, void* stream);

/*
 * As chem_integrate, but T, p, Y are HOST arrays: the call copies them to
 * handle-owned device buffers, integrates, copies T and Y back and synchronises
 * `stream` before returning.
 */
chem_status chem_integrate_host(chem_handle h, int64_t n_cells, double* T, const double* p,
                                double* Y, double dt, double rtol, double atol, void* stream);

/*
 * Integration for callers that cannot allocate device memory. The paper has no
 * counterpart: this exists for users of this library, not for the method.
 *
 * chem_integrate may grow handle-owned device buffers with cudaMalloc/cudaFree.
 * Callers that cannot allow that -- applications whose device memory is fixed up
 * front by their own pool or budget (a CFD code that reserves the GPU's memory
 * for its fields and solvers at start-up, where a late cudaMalloc fails or
 * evicts its pool), and callers inside a time-step loop that cannot accept the
 * device synchronisation an allocation or free may imply while other streams are
 * busy -- use this entry point instead. It allocates nothing: the integration
 * kernel's scratch (work-queue counter and per-cell statistics) lives in one
 * fixed-size device array inside the library, sized for CHEM_NOALLOC_MAX_CELLS
 * cells (about 1.3 MB), which every GPU that loads the library holds until the
 * process exits.
 *
 * Arguments, layout and results are those of chem_integrate (device pointers,
 * in-place T and Y, stream-ordered), and for the same handle options and block
 * size the results are bitwise those of chem_integrate. The handle's precision,
 * scheduler, block, ir_sweeps, max_steps and ctas_per_sm options apply; cells
 * are taken in index order with the starting-step heuristic (the learned order
 * and initial step, the autotuner and CUDA-graph replay need handle-owned
 * buffers and are not used).
 *
 * After this call, chem_get_stats and chem_get_totals on the handle report this
 * call's cells (substeps, rejections, first step, status -- a failed cell keeps
 * its last accepted state, as in chem_integrate) by reading the fixed array: read
 * them before another call of this entry point on the same device overwrites it.
 *
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture. All calls share the one array and it keeps the last call's contents:
 * the call clears what must start at zero (the queue counter) on `stream`, and
 * calls that overlap on the GPU (concurrent streams or handles) race on it.
 * Errors: CHEM_ERR_INVALID_ARG as for chem_integrate, for
 * n_cells > CHEM_NOALLOC_MAX_CELLS (split the batch) and for a handle with
 * reference mapping on; CHEM_ERR_CUDA.
 */
#define CHEM_NOALLOC_MAX_CELLS 65536
chem_status chem_integrate_noalloc(chem_handle h, int64_t n_cells, double* T, const double* p, double* Y,
                                   double dt, double rtol, double atol, void* stream);

/* One batch of cells of one mechanism; pointers as in chem_integrate. */
typedef struct {
  chem_handle h;
  int64_t n_cells;
  double* T;
  const double* p;
  double* Y;
} chem_job;

/*
 * Integrates up to 8 jobs (each with its own mechanism handle) in ONE kernel
 * launch sharing one work queue. Options (precision, scheduler, block size)
 * are taken from jobs[0].h; per-cell statistics go to each job's handle. The
 * launch's CTA size and shared memory are those of the largest mechanism.
 * With option "job_launch" = 1 on jobs[0].h, each job is instead integrated by
 * its own launch with its own handle's options, on a stream the handle owns,
 * forked from `stream` and joined back into it by events (the launches may run
 * concurrently; `stream` orders after all of them). Errors: CHEM_ERR_INVALID_ARG
 * (n_jobs outside 1..8, NULL or invalid jobs, a handle used twice, reference
 * mapping on any handle in one-launch mode), as for chem_integrate otherwise.
 */
chem_status chem_integrate_jobs(const chem_job* jobs, int32_t n_jobs, double dt, double rtol,
                                double atol, void* stream);

/*
 * Handle options (numeric values):
 *   "precision"   0 = FP64 throughout;
 *                 1 = mixed: the iteration matrix assembled in float-float
 *                 arithmetic (about 48 significant bits, on the FP32 pipe),
 *                 factorised (Gauss-Jordan inverse) in FP32, every solve refined
 *                 with residuals against the assembled matrix computed as
 *                 compensated FP32 dot products (state, rates, exp/log, error
 *                 control in FP64); matrix entries below 2^-126 in magnitude
 *                 lose precision and entries of 2^128 or more overflow (FP32's
 *                 exponent range: a cell whose iteration matrix overflows fails
 *                 its steps and ends with a failure status; precision 0 has the
 *                 FP64 range);
 *                 2 = as 1 but with the Jacobian assembled in FP32 and the
 *                 refinement residual taken against that FP32 matrix
 *   "ir_sweeps"   0..3 refinement sweeps per solve in precision 1 and 2 (default 1)
 *   "scheduler"   0 = plain (one CTA per cell, hardware block order),
 *                 1 = static (persistent CTAs, fixed round-robin cells),
 *                 2 = queue (persistent CTAs pulling cells from a device counter)
 *   "order"       0 = cell index order; 1 = learned cost order (needs a trained
 *                 model, see chem_mlp_*); 2 = last-call cost order
 *   "h0"          0 = starting-step heuristic; 1 = learned initial step;
 *                 2 = carried over: each cell starts from the step size the
 *                 controller proposed after its last step in the handle's
 *                 previous call of the same size (the heuristic otherwise)
 *   "h0_guard"    1 (default) = a supplied initial step (learned or carried over)
 *                 is kept, at the cell's first step, inside the starting-step
 *                 heuristic's envelope [h_a, 100 h_a], h_a = 0.01 |y0| / |f(y0)| in
 *                 the WRMS norm (no extra RHS evaluation); 0 = taken as supplied
 *   "h0_range"    with h0 = 1: z > 0 = a cell whose standardised model input has a
 *                 feature beyond +-z standard deviations of the training data
 *                 starts from the heuristic instead of the prediction (the model is
 *                 not trusted outside the states it was trained on; default 10);
 *                 0 = off
 *   "max_steps"   step budget per cell (default 100000)
 *   "block"       threads per cell: 64, 128 or 256; 0 (default) = the size with
 *                 the most resident warps per SM for the mechanism and precision
 *   "ctas_per_sm" resident CTAs per SM for persistent schedulers (0 = maximum)
 *   "graph"       1 = capture the launch sequence in a CUDA graph and replay it
 *                 while arguments repeat
 *   "autotune"    1 = time block sizes on a sample at the first call for a
 *                 new size and keep the fastest
 *   "profile"     1 = accumulate per-phase cycle counters (chem_get_phase_cycles)
 *   "jacobian"    FP64 form (precision 0) only: 0 = analytical (default);
 *                 1 = forward differences, column j from f(y + d_j e_j) with
 *                 d_j = sqrt(eps) max(|y_j|, 1 K for T or 1e-6), n extra RHS
 *                 evaluations per Jacobian (the classical alternative the paper's
 *                 analytical Jacobian replaces); also used by chem_eval_jacobian
 *   "pivoting"    FP64 form only: 1 = partial pivoting (default); 0 = Gaussian
 *                 elimination without row interchanges (a zero pivot rejects the step)
 *   "job_launch"  chem_integrate_jobs only (read from jobs[0].h): 0 = one kernel
 *                 launch for all jobs (default); 1 = one launch per job on
 *                 concurrent streams, each with its own handle's options
 *   "method"      0 = RODAS4 (default; order 4, embedded order 3, for the exact
 *                 Jacobian); 1 = ROS34PW2 (Rang & Angermann 2005: a W-method, order
 *                 3 for ANY approximation W of the Jacobian, embedded order 2). The
 *                 W-method is the consistent partner of precision 2: the FP32-
 *                 assembled matrix is a W, and the order survives its rounding,
 *                 where RODAS4 loses order (Methodology, "Analytical Jacobian and
 *                 improved ODE solution", leaves the ODE scheme open)
 *   "time_kernel" 1 = record CUDA events on the stream around each integration
 *                 kernel launch (chem_get_kernel_ms); chem_integrate_noalloc
 *                 does not record them
 * Errors: CHEM_ERR_INVALID_ARG for an unknown key or out-of-range value.
 * chem_get_option also reads "last_block" (read-only): the threads per CTA of
 * the handle's last integration launch, as chosen by "block", the automatic
 * choice or the autotuner (0 before the first launch).
 */
chem_status chem_set_option(chem_handle h, const char* key, double value);
chem_status chem_get_option(chem_handle h, const char* key, double* value);

/*
 * Copies per-cell statistics of the handle's last integration into the given
 * DEVICE arrays (each may be NULL; length >= that call's n_cells), synchronises
 * `stream`, and returns CHEM_ERR_CELLS_FAILED if any cell's status is not
 * CHEM_CELL_OK. substeps counts accepted and rejected steps; h_first is the
 * first accepted step size (s).
 */
chem_status chem_get_stats(chem_handle h, void* stream, int32_t* substeps, int32_t* rejects,
                           double* h_first, int32_t* cell_status);

/* Totals of the last integration (host outputs, any may be NULL); synchronises. */
chem_status chem_get_totals(chem_handle h, void* stream, int64_t* n_cells, int64_t* substeps,
                            int64_t* rejects, int64_t* failed);

/*
 * Per-phase SM cycles accumulated by integrations run with option "profile" = 1
 * (host output cycles[8], summed over cells; thread 0 of each CTA reads the clock
 * at the barriers that close each phase): 0 load + starting step, 1 RHS and
 * Jacobian data at the step point, 2 iteration-matrix assembly, 3 factorisation,
 * 4 stage RHS evaluations, 5 stage linear solves, 6 stage combination + error
 * norm + control, 7 temperature recovery + store. reset != 0 zeroes the counters.
 * Synchronises `stream`.
 */
chem_status chem_get_phase_cycles(chem_handle h, void* stream, uint64_t* cycles, int32_t reset);

/*
 * Device time (ms) of the handle's last integration kernel launch, between CUDA
 * events recorded on the launching stream just before and after it (with option
 * "graph", around the graph launch). Waits for that launch to finish. Returns
 * CHEM_ERR_INVALID_ARG when option "time_kernel" was off for every launch so far.
 */
chem_status chem_get_kernel_ms(chem_handle h, float* ms);

/* ------------------------------------------------------------------------
 * Reference mapping by mixture fraction (paper: Methodology, "DLBFoam: Dynamic
 * load balancing": cells are either integrated or mapped from a reference
 * solution with a similar Bilger mixture fraction Z).
 *
 * Bilger's coupling function beta = 2 Z_C/W_C + Z_H/(2 W_H) - Z_O/W_O of the
 * element mass fractions is, per cell, beta = sum_k b_k Y_k with
 * b_k = (2 a_Ck + a_Hk/2 - a_Ok) / W_k (a_ek: the mechanism's atom counts), and
 * Z = (beta - beta_ox) / (beta_fuel - beta_ox).
 *
 * With mapping on, each chem_integrate call (one job, scheduler 2):
 *   - zone: cells with |Z - Z_center| <= Z_tol (Z of the initial state);
 *   - reference: the zone cell with the lowest index; it is integrated;
 *   - mapped: every other zone cell with |T - T_ref| <= T_tol (initial T); it
 *     is not integrated but receives the reference's change over the step,
 *     T += T_ref(dt) - T_ref(0), Y_k += Y_ref,k(dt) - Y_ref,k(0). Its statistics
 *     read 0 substeps, 0 rejections, h_first 0 and the reference's status; if the
 *     reference failed, the mapped cells keep their initial state;
 *   - every other cell is integrated as without mapping.
 * Everything runs on the device on the call's stream (a few small kernels
 * before and one after the integration kernel); the mapped cells are moved to
 * the front of the work order and the work queue starts past them.
 * ------------------------------------------------------------------------ */

/*
 * Defines the fuel and oxidiser streams and switches mapping on.
 *   elem_C, elem_H, elem_O  columns of the mechanism's element table (desc.elem)
 *                           holding carbon, hydrogen and oxygen atoms; -1 for an
 *                           element the mechanism lacks (at least one >= 0)
 *   Y_fuel[K], Y_ox[K]      host: mass fractions of the two streams (copied)
 *   Z_center, Z_tol, T_tol  the zone and the temperature tolerance (K)
 * Z_tol < 0 switches mapping off (the streams stay defined for
 * chem_eval_mixture_fraction). Synchronous (uploads K coefficients). Errors:
 * CHEM_ERR_INVALID_ARG for a column out of range, NULL or non-finite streams,
 * equal beta of the two streams, NaN Z_tol, non-finite Z_center / T_tol or
 * T_tol < 0. chem_integrate returns CHEM_ERR_INVALID_ARG while mapping is on
 * for several jobs or a scheduler other than 2; chem_integrate_noalloc refuses
 * a handle with mapping on.
 */
chem_status chem_set_reference_mapping(chem_handle h, int32_t elem_C, int32_t elem_H, int32_t elem_O,
                                       const double* Y_fuel, const double* Y_ox, double Z_center,
                                       double Z_tol, double T_tol);

/*
 * Z[n_cells] (device) = Bilger mixture fraction of the cells Y[n_cells][K]
 * (device) for the streams of chem_set_reference_mapping. Stream-ordered.
 * Errors: CHEM_ERR_INVALID_ARG (no streams defined, n_cells < 0, NULL arrays).
 */
chem_status chem_eval_mixture_fraction(chem_handle h, int64_t n_cells, const double* Y, double* Z,
                                       void* stream);

/*
 * Outcome of the handle's last integration with mapping on: mapped[n] (DEVICE,
 * may be NULL; 1 = mapped) and, on the host, the number of mapped cells and the
 * reference cell's index (-1: empty zone). Synchronises `stream`. Returns
 * CHEM_ERR_INVALID_ARG when the last integration ran without mapping.
 */
chem_status chem_get_reference_mapping(chem_handle h, void* stream, int32_t* mapped, int64_t* n_mapped,
                                       int64_t* ref_cell);

/* Last error message of the handle (or of the last chem_create when h is NULL). */
const char* chem_last_error(chem_handle h);

/* Number of species / reactions of a handle. */
int32_t chem_n_species(chem_handle h);
int32_t chem_n_reactions(chem_handle h);

/* ------------------------------------------------------------------------
 * Diagnostic entry points: the same device code the integrator runs, exposed
 * for parity testing against an independent CPU implementation.
 * ------------------------------------------------------------------------ */

/* f[n_cells][K+1] = RHS at the given states (device pointers). */
chem_status chem_eval_rhs(chem_handle h, int64_t n_cells, const double* T, const double* p,
                          const double* Y, double* f, void* stream);

/*
 * J[n_cells][K+1][K+1] (row-major) = analytical Jacobian at the given states.
 * With option precision = 2 the Jacobian is assembled in FP32 and returned
 * widened to double.
 */
chem_status chem_eval_jacobian(chem_handle h, int64_t n_cells, const double* T, const double* p,
                               const double* Y, double* J, void* stream);

/* h0[n_cells] = starting step of the heuristic used by chem_integrate. */
chem_status chem_eval_h0(chem_handle h, int64_t n_cells, const double* T, const double* p,
                         const double* Y, double dt, double rtol, double atol, double* h0,
                         void* stream);

/*
 * Batched dense solve with the integrator's LU and triangular-solve code:
 * for each of n_mat systems, A[dim][dim] x = b (device, row-major, A unchanged).
 * precision 0: FP64 LU; 1: FP32 Gauss-Jordan inverse of A with `ir_sweeps`
 * refinement sweeps against A held as float-float pairs (residuals as compensated
 * FP32 dot products, about 48 bits); 2: as 1 against A rounded to FP32.
 * info[n_mat] (device, may be NULL): 0, or 1+k for a zero pivot at column k.
 * dim <= 128.
 */
chem_status chem_lu_solve_batched(int64_t n_mat, int32_t dim, const double* A, const double* b,
                                  double* x, int32_t* info, int32_t precision, int32_t ir_sweeps,
                                  void* stream);

/*
 * y[i] = f(x[i]) for n elements of device arrays x, y (n >= 0) by the elementary
 * functions the rate kernels use: op 0 exp (Tang's table-driven method), op 1 ln
 * (table-driven, Tang's manner), op 2 1/x (Newton's iteration on the hardware's
 * approximate reciprocal); arguments outside their reduced ranges (see the kernel
 * source) follow the CUDA library routine or the IEEE division. Ops 3 and 4 return
 * the hi and lo parts (widened to double) of the split of x into a float-float pair
 * that the mixed form's Jacobian assembly and refinement use: hi = x truncated to 24
 * significant bits, lo = x - hi rounded to FP32; |x| < 2^-126 gives (0, 0), |x| >=
 * 2^128 gives (+-inf, 0). Returns CHEM_ERR_INVALID_ARG for an unknown op, n < 0 or
 * NULL arrays with n > 0.
 */
chem_status chem_eval_math(int32_t op, int64_t n, const double* x, double* y, void* stream);

/*
 * The Rosenbrock coefficients the device code uses, in the transformed form
 * (Hairer & Wanner II, Sec. IV.7): gamma, a[6][6], c[6][6] (row-major,
 * strictly lower), m[6] (solution weights), e[6] (error weights). Host only;
 * needs no GPU.
 */
void chem_rosenbrock_tableau(double* gamma, double* a, double* c, double* m, double* e);

/*
 * As chem_rosenbrock_tableau for option "method" = `method` (0 RODAS4,
 * 1 ROS34PW2); entries beyond the method's stage count are zero. Returns the
 * number of stages, or -1 for an unknown method. Host only; needs no GPU.
 */
int32_t chem_method_tableau(int32_t method, double* gamma, double* a, double* c, double* m, double* e);

#ifdef __cplusplus
}
#endif

#endif /* CHEM_H_ */
