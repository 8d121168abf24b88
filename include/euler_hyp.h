/*
 * euler_hyp.h -- C ABI of the GB300 (sm_103a) hyperbolic Euler solver.
 *
 * The library advances the compressible Euler equations (the hyperbolic
 * operator S_H of Guermond, Kronbichler, Maier, Popov & Tomas,
 * arXiv:2106.02159) on continuous P1/Q1 finite elements: one forward-Euler
 * step is Algorithm 1 of the paper's Appendix B (graph viscosity, low-order
 * update, local bounds, high-order fluxes, convex limiting with two
 * symmetrised passes), followed by the boundary post-processing of Sec. 4,
 * inside the SSPRK(3,3) time loop of Sec. 4.1 (eq. SPPRK33).
 *
 * Conventions shared by every entry point:
 *  - Every function returns an eh_status and never aborts the process. On
 *    failure eh_last_error() describes the cause.
 *  - State vectors are component-major: U[s * n + i], s = 0 density,
 *    1..dim momentum, dim+1 total energy (S = dim + 2 components).
 *  - Host arrays passed to eh_upload_mesh are copied; the caller keeps
 *    ownership. Device pointers (is_device_ptr = 1) are only read or written
 *    during the call, on the context's stream.
 *  - All device memory is owned by the context and freed by eh_destroy.
 *  - Work is queued on the context's stream; eh_step/eh_run do not
 *    synchronise unless a host result is requested.
 */
#ifndef EULER_HYP_H
#define EULER_HYP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eh_ctx eh_ctx;

typedef enum {
  EH_OK = 0,
  EH_ERR_INVALID_ARG = 1,     /* a NULL pointer, a size or a parameter out of range */
  EH_ERR_OOM = 2,             /* device memory allocation failed */
  EH_ERR_BAD_MESH = 3,        /* CSR not sorted / no diagonal / pattern not symmetric / bad boundary list */
  EH_ERR_NOT_ADMISSIBLE = 4,  /* a state with rho <= 0 or internal energy <= 0 (Sec. 2.1, set A) */
  EH_ERR_CFL = 5,             /* a prescribed dt above the invariant-domain limit (Sec. 3.1, c_cfl <= 1) */
  EH_ERR_CUDA = 6,            /* a CUDA runtime error */
  EH_ERR_STATE = 7            /* called out of order (e.g. eh_step before a mesh and a state) */
} eh_status;

/* Boundary kinds (Sec. 4): slip (eq. slip_bc), Dirichlet / supersonic inflow
 * (eq. Supersonic_inflow), do nothing (supersonic outflow, eq.
 * Supersonic_outflow), and the two non-reflecting post-processings of
 * Sec. 4.2 with the node's outward normal and its Dirichlet (far-field)
 * state: by characteristic variables (eqs. Supersonic_inflow, Subsonic_inflow,
 * Subsonic_outflow, Supersonic_outflow, chosen by the node's normal velocity
 * and sound speed) and by the exact Riemann value at the boundary (eq.
 * Godunov_bc). */
enum { EH_BC_SLIP = 1, EH_BC_DIRICHLET = 2, EH_BC_DO_NOTHING = 3, EH_BC_CHARACTERISTIC = 4, EH_BC_GODUNOV = 5 };

/* Arithmetic of the step. FP64: everything in IEEE double. MIXED: c_ij,
 * lambda_max, d_ij and the high-order fluxes in FP32; state, bounds, limiter
 * and dt in FP64. */
enum { EH_PRECISION_FP64 = 0, EH_PRECISION_MIXED = 1 };

typedef struct {
  int dim;              /* 2 or 3 */
  double gamma;         /* ratio of specific heats, 1 < gamma <= 5/3 (lambda_max is a bound there) */
  double cfl;           /* c_cfl of eq. dtCfl, 0 < cfl <= 1 */
  int limiter_passes;   /* limiting passes of Sec. 3.3, >= 1 (the paper uses 2) */
  int bound_relaxation; /* 0: strict local bounds (the paper's text); 1: bounds scaled by
                           (1 -/+ r_i), r_i = (m_i / sum_j m_j)^(1.5/dim) */
  int precision;        /* EH_PRECISION_* */
  int device;           /* CUDA device ordinal */
  void *stream;         /* cudaStream_t to run on, or NULL for a stream owned by the context */
} eh_config;

typedef struct {
  double t;                   /* simulated time advanced by eh_step/eh_run (instance 0) */
  int64_t steps;              /* SSPRK(3,3) steps taken */
  double last_dt;             /* dt of the last step */
  double last_stage_bound[3]; /* c_cfl min_i m_i / (2 |d_ii|) of the last step's three stages */
  int64_t cfl_violations;     /* stages 2-3 whose dt exceeded min_i m_i/(2|d_ii|) (c_cfl = 1) */
  int64_t not_admissible;     /* non-admissible nodes found after a step (0 unless an error) */
  int64_t line_searches_deferred; /* limiter line searches (Sec. 3.3) not settled by the check at
                                     l = 1 and run in a separate pass, summed over all steps */
  int64_t line_searches_iterated; /* of those, searches that ran the bracketing iteration */
  int64_t low_order_not_admissible; /* rows whose low-order update U^L left the admissible set
                                       (always 0 with c_cfl <= 1; see eh_step_adaptive) */
  /* of the current state (all instances together; 0 before eh_set_state): */
  double rho_min;             /* min_i rho_i */
  double e_min;               /* min_i of the specific internal energy E/rho - |m|^2/(2 rho^2) */
  double total[5];            /* sum_i m_i U_i with the lumped masses: mass, momentum, total energy
                                 (S = dim + 2 values, the rest 0); constant up to the boundary
                                 fluxes (Lemma 3.1; exactly so, to roundoff, on periodic or closed
                                 slip domains, Lemma 4.5) */
} eh_diagnostics;

/* Fills *cfg with the defaults: dim 2, gamma 1.4, cfl 0.5, 2 limiter passes,
 * strict bounds, FP64, device 0, own stream. */
void eh_config_default(eh_config *cfg);

/* Creates a context on cfg->device. Returns EH_ERR_INVALID_ARG for an
 * out-of-range parameter. *out receives the context (NULL on error). */
eh_status eh_create(const eh_config *cfg, eh_ctx **out);

/* Uploads a mesh (Sec. 2.2). Host pointers, copied.
 *   n, nnz        : nodes and CSR entries (diagonal included), nnz < 2^31
 *   row_ptr[n+1]  : int64 CSR offsets; col[nnz] int32 columns, sorted and
 *                   unique within a row, diagonal present, pattern symmetric
 *   cij[dim][nnz] : c_ij = int phi_i grad phi_j (component-major)
 *   mij[nnz]      : consistent mass m_ij, symmetric (m_ij = m_ji to 1e-12
 *                   relative, else EH_ERR_BAD_MESH); mi[n]: lumped mass m_i > 0
 *   n_bnd, bnd_node[n_bnd], bnd_kind[n_bnd] (EH_BC_*): every node on the
 *                   boundary, once (nodes not listed are interior)
 *   bnd_normal[dim][n_bnd] : unit normal of the node's kind: n^s_i of eq.
 *                            def_ns_nio for slip nodes, n^nr_i (the normalised
 *                            integral of phi_i n over the non-reflecting faces)
 *                            for non-reflecting nodes
 *   bnd_state[S][n_bnd]    : Dirichlet / far-field states (read for Dirichlet and
 *                            non-reflecting nodes; may be NULL if there are none)
 * The library builds the transpose index itself. Errors: EH_ERR_BAD_MESH for
 * an invalid pattern or boundary list, EH_ERR_OOM. A second call replaces the
 * mesh and invalidates the state. */
eh_status eh_upload_mesh(eh_ctx *ctx, int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                         const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                         const double *bnd_state);

/* Sets the state U[S][n] (host or device pointer). Returns
 * EH_ERR_NOT_ADMISSIBLE (state left unset) if some node has rho <= 0 or
 * internal energy <= 0. Synchronises the stream. */
eh_status eh_set_state(eh_ctx *ctx, const double *U, int is_device_ptr);

/* Copies the state into U_out[S][n] (host or device pointer). Synchronises
 * and reports a pending device-side error (EH_ERR_CFL, EH_ERR_NOT_ADMISSIBLE). */
eh_status eh_get_state(eh_ctx *ctx, double *U_out, int is_device_ptr);

/* Applies the boundary post-processing of Sec. 4 to the current state (use
 * once on initial data that does not satisfy the boundary conditions). */
eh_status eh_apply_boundary_conditions(eh_ctx *ctx);

/* CFL time step tau = c_cfl min_i m_i / (2 |d_ii|) of the current state
 * (Sec. 3.1, eq. dtCfl). Synchronises. */
eh_status eh_cfl_dt(eh_ctx *ctx, double *dt);

/* One forward-Euler stage (Algorithm 1) plus boundary post-processing applied
 * to the current state: U <- BC(FE(U)). tau > 0: that step; tau <= 0: the
 * stage's CFL step. tau_used may be NULL (then no synchronisation). */
eh_status eh_stage(eh_ctx *ctx, double tau, double *tau_used);

/* One SSPRK(3,3) step. dt > 0: that step (EH_ERR_CFL if it exceeds the
 * invariant-domain limit of the first stage; the state is then unchanged);
 * dt <= 0: the CFL step of the first stage, reused by stages 2 and 3.
 * dt_used may be NULL (then no synchronisation). The step is a replay of the
 * CUDA graph that eh_run caches (captured on first use) when dt <= 0 or dt is
 * the one the graph holds; another dt launches the kernels one by one. */
eh_status eh_step(eh_ctx *ctx, double dt, double *dt_used);

/* nsteps SSPRK(3,3) steps with the same dt rule as eh_step, replayed from a
 * CUDA graph, without synchronising. */
eh_status eh_run(eh_ctx *ctx, int32_t nsteps, double dt);

/* One SSPRK(3,3) step with a CFL number above 1 (Sec. 3.1, remark on high
 * aspect-ratio meshes): the step is tried with c_cfl = cfl_max (0 < cfl_max
 * <= 64) in place of the context's CFL number; while the low-order update U^L
 * of a stage, or the result, leaves the admissible set, the state and time
 * are put back and the step restarts with c_cfl halved (c_cfl <= 1 always
 * passes). Synchronises after every attempt. Outputs (may be NULL): the
 * accepted dt, its CFL number and the number of restarts. One instance only
 * (EH_ERR_STATE after eh_set_instances with more than one). */
eh_status eh_step_adaptive(eh_ctx *ctx, double cfl_max, double *dt_used, double *cfl_used, int32_t *restarts);

/* ---- the parabolic sub-step and the Navier-Stokes step (Sec. 5, 2D only) ----
 * eh_set_viscosity: the shear and bulk viscosities mu, lambda >= 0 and
 * kappa / c_v >= 0 (sigma(v) = 2 mu eps(v) + (lambda - 2 mu/3) div v I, heat
 * flux -kappa/c_v grad e), the finite-element data of the mesh (host arrays,
 * copied): L[nnz] = int grad phi_i . grad phi_j, G[2][2][nnz] = int d_k phi_i
 * d_m phi_j, and the cells with their quadrature (n_cells cells of nv = 3 or 4
 * nodes, nq points: cells[n_cells][nv], qw[n_cells][nq] weights x |det J|,
 * qphi[n_cells][nq][nv], qgrad[n_cells][nq][2][nv]); the no-slip nodes
 * wall[n_wall] (velocity 0; homogeneous Neumann elsewhere and for e); the
 * relative residual cg_tol and the iteration limit of the CG solves.
 * EH_ERR_INVALID_ARG / EH_ERR_BAD_MESH on bad input, EH_ERR_STATE without a
 * mesh. */
eh_status eh_set_viscosity(eh_ctx *ctx, double mu, double lambda, double kappa_cv, const double *L, const double *G,
                           int32_t n_cells, int32_t nv, int32_t nq, const int32_t *cells, const double *qw,
                           const double *qphi, const double *qgrad, int32_t n_wall, const int32_t *wall, double cg_tol,
                           int32_t cg_max_iter);

typedef struct {
  int32_t cg_iter_velocity, cg_iter_energy, cg_iter_low; /* CG iterations (low: 0 unless limited) */
  int32_t limited;  /* 1 if Crank-Nicolson gave a non-positive internal energy and FCT was applied */
  double min_e;     /* min_i e_i^{n+1} */
} eh_parabolic_info;

/* One parabolic sub-step S_P over dt on the current state (synchronises):
 * rho unchanged; velocity by Crank-Nicolson (eqs. mt_parabolic_discrete,
 * vel_parabolic_discrete); internal energy by Crank-Nicolson with the viscous
 * source (eqs. def_Ki_nplusone, high_int_energy_CN) and, if that gives a
 * non-positive value, the low-order update and FCT limiting (eqs.
 * low_order_update_internal_energy, Aij_for_internal_energy); total energy by
 * eq. energy_parabolic_discrete. info may be NULL. */
eh_status eh_parabolic_step(eh_ctx *ctx, double dt, eh_parabolic_info *info);

/* One Strang-split Navier-Stokes step (eq. continuous_Strang): H(tau) P(2 tau)
 * H(tau) with tau the CFL step of the first hyperbolic step (dt <= 0) or dt;
 * the second hyperbolic step is held to the invariant-domain limit like a
 * prescribed dt (EH_ERR_CFL). Synchronises. tau_used and info may be NULL. */
eh_status eh_step_ns(eh_ctx *ctx, double dt, double *tau_used, eh_parabolic_info *info);

/* Waits for queued work and reports a pending device-side error. */
eh_status eh_synchronize(eh_ctx *ctx);

/* Diagnostics of the last steps and of the current state (synchronises; the
 * state statistics are two reductions on the device, in a fixed order, so the
 * same state gives the same bits). */
eh_status eh_get_diagnostics(eh_ctx *ctx, eh_diagnostics *out);

/* Intermediate arrays of the last forward-Euler stage, for checking against
 * a reference (synchronises). 'what' selects one of EH_TRACE_*; host_out must
 * hold 'count' doubles, which must equal the array's size:
 *   D_IJ [nnz] graph viscosity d^L_ij (diagonal included; Sec. 3.1)
 *   ALPHA [n] indicator alpha_i (Sec. 3.2)
 *   U_LOW [S][n] low-order update U^L (eq. loworder_bis)
 *   F_HIGH [S][n] high-order fluxes F^H_i (Algorithm 1, step 3)
 *   BOUNDS [3][n] rho_min, rho_max, Phi_min (Sec. 3.3)
 *   L_PASS1 [nnz] symmetrised limiter l_ij = min(l_j^i, l_i^j) of the first
 *     pass (1 on the diagonal; Sec. 3.3)
 *   U_PASS1 [S][n] state after the first limiting pass
 *   TAU [1] the stage's tau; TAU_BOUND [1] its own CFL bound
 *   P_PASS1 [S][nnz] limiter directions P_ij of the first pass (eq.
 *     LambdaArrangement; 0 on the diagonal)
 *   L_LAST [nnz] symmetrised limiter of the last pass (1 on the diagonal)
 * The trace buffers are allocated by the first eh_stage call of a mesh. */
enum {
  EH_TRACE_D_IJ = 0, EH_TRACE_ALPHA = 1, EH_TRACE_U_LOW = 2, EH_TRACE_F_HIGH = 3, EH_TRACE_BOUNDS = 4,
  EH_TRACE_L_PASS1 = 5, EH_TRACE_U_PASS1 = 6, EH_TRACE_TAU = 7, EH_TRACE_TAU_BOUND = 8, EH_TRACE_P_PASS1 = 9,
  EH_TRACE_L_LAST = 10
};
eh_status eh_trace(eh_ctx *ctx, int what, double *host_out, int64_t count);

/* The integer mesh data as the device holds it (synchronises; host arrays,
 * any may be NULL): row_ptr[n+1] and col[nnz] as uploaded, and transpose[nnz],
 * the position of entry (j, i) for every entry (i, j), built by
 * eh_upload_mesh -- the index through which the symmetric edge quantities
 * (d_ij, Sec. 3.1; l_ij, Sec. 3.3) are written once and mirrored.
 * EH_ERR_STATE without a mesh. */
eh_status eh_get_mesh_index(eh_ctx *ctx, int64_t *row_ptr, int32_t *col, int32_t *transpose);

/* Per-kernel timing with CUDA events on the context's stream, for profiling.
 * While enabled, eh_step/eh_stage/eh_run launch eagerly (no graph) and record
 * an event pair around every kernel. eh_profile_read returns, for one kernel
 * kind (EH_KERNEL_*), the summed duration in milliseconds and the number of
 * launches since profiling was enabled (synchronises). EH_KERNEL_VISC covers
 * the viscosity and indicator kernels; EH_KERNEL_LSEARCH the line searches that
 * the limiter passes left to a separate kernel (Sec. 3.3). */
enum {
  EH_KERNEL_PREP = 0, EH_KERNEL_VISC = 1, EH_KERNEL_LOW = 2, EH_KERNEL_TAU = 3, EH_KERNEL_LIM1 = 4,
  EH_KERNEL_PASS = 5, EH_KERNEL_FINAL = 6, EH_KERNEL_LSEARCH = 7, EH_KERNEL_COUNT = 8
};
eh_status eh_profile_enable(eh_ctx *ctx, int enable);
eh_status eh_profile_read(eh_ctx *ctx, int kernel, double *total_ms, int64_t *launches);

/* Allocation-free CFL time step. (The paper has no counterpart: this is a
 * service of the library, not a step of the method.)
 *
 * For callers that cannot allocate device memory when they need a time step --
 * a host framework that owns all device memory through its own pool and does
 * not let plug-in libraries call cudaMalloc, or a real-time loop where an
 * allocation (which can synchronise the device) is not allowed. It needs no
 * eh_ctx. It computes tau = cfl * min_i m_i / (2 sum_{j != i} d_ij) with d_ij
 * the graph viscosity of the state (the same quantity as eh_cfl_dt) from the
 * caller's own device arrays:
 *   row_ptr[n+1] (int64), col[nnz] (int32): CSR as for eh_upload_mesh (sorted,
 *     diagonal present, symmetric pattern -- not checked here);
 *   cij[dim][nnz], mi[n]; is_boundary[n] (1 for boundary nodes) or NULL when
 *     no node lies on the boundary; U[dim+2][n] an admissible state;
 *   dt_out: device pointer to one double, written by the last kernel. It
 *     receives NaN when a row's state is not admissible (rho <= 0 or
 *     internal energy <= 0 give an undefined wave speed): the reduction keeps
 *     NaN rather than dropping the row, so check the value for NaN.
 * Work is queued on 'stream' (a cudaStream_t, NULL for the default stream) of
 * the current device; the call does not synchronise. Returns EH_ERR_CUDA,
 * without launching, if a CUDA error from earlier work is pending (it is left
 * in place for the caller to read), and EH_ERR_CUDA if a launch fails.
 * Scratch: a file-scope device array of EH_CFL_NOALLOC_MAX_ROWS / 128 doubles
 * (512 KiB) that every GPU loading the library keeps until the process ends;
 * n above EH_CFL_NOALLOC_MAX_ROWS returns EH_ERR_INVALID_ARG before any work.
 * The first call in each CUDA context of a device looks the array's device
 * address up (cudaGetSymbolAddress, which allocates nothing) and caches it
 * under the context's id, so a device reset or a new context is handled; make
 * that first call before any stream capture.
 * Every call overwrites the entries it reads, so nothing needs clearing, but
 * all calls share the array: two calls whose kernels overlap on the GPU (on
 * different streams without ordering) race and give wrong results.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define EH_CFL_NOALLOC_MAX_ROWS (1 << 23)
eh_status eh_cfl_dt_noalloc(int32_t dim, double gamma, double cfl, int32_t n, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col, const double *cij, const double *mi,
                            const unsigned char *is_boundary, const double *U, double *dt_out, void *stream);

/* Independent instances in one context (batched solves). After
 * eh_upload_mesh of a block-diagonal mesh -- instance k owns the rows
 * [row_offset[k], row_offset[k+1]) and no CSR entry couples two instances --
 * this declares the split. Every step then advances all instances in the same
 * kernel launches, each with its own CFL step (eq. dtCfl per instance), its
 * own simulated time and, if t_final (host, ninst values, or NULL) is given, a
 * last step shortened to land on t_final[k]; finished instances stay frozen
 * (tau = 0). Resets the instance times. Errors: EH_ERR_INVALID_ARG for bad
 * offsets, EH_ERR_BAD_MESH if an entry couples two instances. */
eh_status eh_set_instances(eh_ctx *ctx, int32_t ninst, const int64_t *row_offset, const double *t_final);

/* Per-instance simulated time t[ninst], last tau[ninst] and CFL bounds of the
 * last step's three stages stage_bound[3][ninst] (host arrays; any may be
 * NULL). Synchronises. */
eh_status eh_get_instances(eh_ctx *ctx, double *t, double *last_dt, double *stage_bound);

/* Per-instance number of SSPRK(3,3) steps taken with tau > 0 since
 * eh_set_instances (a finished instance stops counting), steps[ninst] (host).
 * Synchronises. */
eh_status eh_get_instance_steps(eh_ctx *ctx, int64_t *steps);

/* Launch-shape autotuner: runs 'steps_per_candidate' SSPRK(3,3) steps for
 * every candidate -- 64, 128 and 256 rows per block, and for the grid-stride
 * kernels (EH_KERNEL_LIM1, _PASS, _FINAL) one thread per row or at most 256,
 * 512 or 768 rows in flight per SM -- times every kernel with CUDA events and
 * keeps the fastest shape per kernel kind. The state and the instance times
 * are restored afterwards. chosen (may be NULL) receives EH_KERNEL_COUNT
 * block sizes. */
eh_status eh_autotune(eh_ctx *ctx, int32_t steps_per_candidate, int32_t *chosen);

/* Current block size of every kernel kind (EH_KERNEL_COUNT values). */
eh_status eh_get_block_sizes(const eh_ctx *ctx, int32_t *tpb);

/* Rows in flight per SM of every kernel kind (EH_KERNEL_COUNT values; 0 = one
 * thread per row, the grid covering all rows at once). */
eh_status eh_get_rows_per_sm(const eh_ctx *ctx, int32_t *rows);

/* Sets one kernel kind's launch shape by hand: threads_per_block 64, 128 or
 * 256; rows_per_sm 0 (one thread per row) or, for EH_KERNEL_LIM1, _PASS and
 * _FINAL only, a cap of 1..2048 rows in flight per SM (the kernel then loops
 * over rows with a grid stride). EH_ERR_INVALID_ARG otherwise. Results do not
 * depend on the shape. */
eh_status eh_set_launch_shape(eh_ctx *ctx, int32_t kernel, int32_t threads_per_block, int32_t rows_per_sm);

/* Number of kernel launches one eh_step issues (for accounting). */
int32_t eh_launches_per_step(const eh_ctx *ctx);

/* ------------------------------------------------------------------------
 * Served stream of independent solves (continuous batching, one device; the
 * paper has no counterpart -- it serves the method's many-solve use).
 * A batch admits requests first come, first served while their device memory
 * fits a budget next to the requests already running and the device's free
 * memory; each admitted request keeps its mesh and state resident on the
 * device. Two modes (eh_batch_set_mode):
 *  - EH_BATCH_MERGED (default): the running requests are the instances of ONE
 *    batched context (as eh_set_instances on their block-diagonal union), so
 *    a step of the batch is a single set of kernel launches -- one CUDA-graph
 *    replay -- covering all of them, each with its own CFL step and final
 *    time. Requests join and leave between eh_batch_advance calls: the union
 *    is rebuilt on the device ("repacked") from the requests' resident data and
 *    current states; a request that reached its final time inside an advance
 *    stays frozen (tau = 0) until the next repack. Each request's result is the
 *    same, bit for bit, as solving it alone (per-row arithmetic, per-instance
 *    tau). One context steps every member: a device-side failure (e.g. a
 *    non-admissible state) stops every request in the batch at that advance.
 *  - EH_BATCH_PER_REQUEST_STREAMS: every request has a context of its own on
 *    its own stream, and an advance launches one step of each request in turn
 *    (their launches overlap on the device); a request's failure stops only it.
 * The caller owns the batch and frees it with eh_batch_destroy; the batch owns
 * the requests' device data. Not thread-safe: one host thread per batch.
 * ------------------------------------------------------------------------ */
typedef struct eh_batch eh_batch;
enum { EH_BATCH_MERGED = 0, EH_BATCH_PER_REQUEST_STREAMS = 1 };

/* Device bytes a context needs for a mesh of n nodes and nnz CSR entries in
 * dimension dim and precision EH_PRECISION_* (the estimate admission uses:
 * the arrays eh_upload_mesh allocates, plus 10% and 1 MiB). Host only.
 * EH_ERR_INVALID_ARG for dim not 2 or 3, an unknown precision, n < 1 or
 * nnz < n. */
eh_status eh_estimate_device_bytes(int32_t dim, int32_t precision, int32_t n, int64_t nnz, uint64_t *bytes);

/* Device bytes the admission of a batch in 'mode' (EH_BATCH_*) counts for a
 * request of n nodes, nnz CSR entries and n_bnd boundary nodes: the
 * eh_estimate_device_bytes estimate, plus in merged mode the request's own
 * resident copy of its mesh data and state. Host only. EH_ERR_INVALID_ARG for
 * bad sizes, dimension, precision or mode. */
eh_status eh_estimate_request_bytes(int32_t dim, int32_t precision, int32_t mode, int32_t n, int64_t nnz,
                                    int32_t n_bnd, uint64_t *bytes);

/* Creates an empty batch in merged mode. cfg as for eh_create, with
 * cfg->stream NULL (the batch's context, and in per-request mode every
 * request, runs on a stream of its own); hbm_budget_bytes > 0 is the device
 * memory the running requests may hold together. EH_ERR_INVALID_ARG
 * otherwise; *out is NULL on error. */
eh_status eh_batch_create(const eh_config *cfg, uint64_t hbm_budget_bytes, eh_batch **out);

/* Selects EH_BATCH_MERGED or EH_BATCH_PER_REQUEST_STREAMS; only while the
 * batch holds no request (EH_ERR_STATE otherwise, EH_ERR_INVALID_ARG for an
 * unknown mode). */
eh_status eh_batch_set_mode(eh_batch *b, int32_t mode);

/* Number of times a merged batch rebuilt its context so far. */
eh_status eh_batch_repacks(const eh_batch *b, int64_t *repacks);

/* Admits one request: a mesh (arguments as eh_upload_mesh, host pointers,
 * copied), its initial state U0[S][n] (host, copied; the boundary
 * post-processing of Sec. 4 is applied to it) and its end time t_final > 0
 * (the last step is shortened to land on it, as eh_set_instances). *ticket
 * receives the request's identifier. The request's device bytes (the
 * admission estimate; in merged mode also the request's own copy of its mesh)
 * must fit next to the running requests in the budget and in the device's
 * free memory: EH_ERR_OOM means "not now" (nothing changed; admit it after a
 * poll has freed memory); a request larger than the whole budget is refused
 * with EH_ERR_INVALID_ARG. Errors of eh_upload_mesh / eh_set_state otherwise
 * (nothing kept). */
eh_status eh_batch_admit(eh_batch *b, int32_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                         const double *cij, const double *mij, const double *mi, int32_t n_bnd,
                         const int32_t *bnd_node, const int32_t *bnd_kind, const double *bnd_normal,
                         const double *bnd_state, const double *U0, double t_final, int64_t *ticket);

/* Advances every running request by 'steps' >= 1 SSPRK(3,3) steps. Merged
 * mode: first rebuilds the batch's context if requests joined or finished
 * since the last advance, then replays its CUDA graph 'steps' times (one set
 * of launches per step for all requests). Per-request mode: one step of each
 * request in turn, on its own stream. Then synchronises and marks the
 * requests that reached t_final, or failed, as finished. *n_finished (may be
 * NULL) receives the number of finished requests not yet polled. */
eh_status eh_batch_advance(eh_batch *b, int32_t steps, int32_t *n_finished);

/* *done = 0 while the request runs. Once it has finished: *done = 1, U_out
 * (host, [S][n], or NULL) receives its state, t (may be NULL) its simulated
 * time, steps (may be NULL) the steps it took (tau > 0); its device data is
 * freed and its ticket retired. Returns the status that stopped the request
 * (EH_OK when it reached t_final); EH_ERR_INVALID_ARG for an unknown ticket. */
eh_status eh_batch_poll(eh_batch *b, int64_t ticket, int32_t *done, double *U_out, double *t, int64_t *steps);

/* Requests admitted and not yet polled, and the device bytes they hold by the
 * admission estimate (either pointer may be NULL). */
eh_status eh_batch_active(const eh_batch *b, int32_t *n_requests, uint64_t *bytes_in_use);

/* Text of the batch's last error (never NULL). */
const char *eh_batch_last_error(const eh_batch *b);

/* Frees the batch and every request still in it; NULL is a no-op. */
void eh_batch_destroy(eh_batch *b);

/* Text of the last error of this context (never NULL). */
const char *eh_last_error(const eh_ctx *ctx);

/* Name of a status code (never NULL). */
const char *eh_status_string(eh_status st);

/* Frees every resource of the context; NULL is a no-op. */
void eh_destroy(eh_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* EULER_HYP_H */
