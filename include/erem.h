/*
 * erem.h - C ABI of the GB300 (sm_103a) library for the Exponential
 * Rosenbrock-Euler method (EREM) with real Leja interpolation of phi_1,
 * applied to heat transport by Darcy flow in heterogeneous porous media
 * (Tambue, Berre, Nordbotten, arXiv 1209.5553).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Grid.  A uniform Cartesian grid of nx x ny (x nz) cells on
 *   [0,lx] x [0,ly] (x [0,lz]) (paper §3.1, structured mesh).  Cell-centred
 *   arrays have N = nx*ny*nz FP64 entries, contiguous, x fastest:
 *   i = ix + nx*(iy + ny*iz).  In 2D set dim = 2 and nz = 1 (unit thickness).
 * Boundary set-up.  x = 0: Dirichlet pressure head_left and Dirichlet
 *   temperature T_inflow (conduction through the half cell, inflow value for
 *   upwinding).  x = 1: Dirichlet pressure head_right; the face carries the
 *   boundary cell's temperature outwards and no conduction.  All other faces
 *   are closed (no flow, no heat flux).
 * Pointers.  Every array argument may be a device pointer (cudaMalloc, torch
 *   CUDA tensor) or a host pointer (pageable or pinned).  Host arrays are
 *   staged through buffers owned by the context; copies are enqueued on the
 *   given stream and the call returns after they complete.  The caller owns
 *   all arrays; the library never keeps a caller pointer after a call.
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = legacy
 *   default stream).  Every call enqueues its work on that stream and
 *   returns once its result is determined (the Leja stopping test and the
 *   linear solvers read small control blocks back to the host): stats and
 *   host output arrays are complete on return; device output arrays are
 *   complete in stream order (the call's last kernel may still be running,
 *   so synchronise the stream or put dependent work on it).
 * Errors.  Every entry point returns an erem_status; nothing is thrown
 *   across the ABI.  erem_last_error() gives a message for the last failure
 *   of a context.  Arguments are checked on the host (sizes, dt > 0,
 *   tolerances > 0, NULL pointers); non-finite input values, negative
 *   conductivities and porosities outside [0,1] are detected by the set-up
 *   kernels and reported as EREM_ENONFINITE / EREM_EINVAL.  A failing call
 *   leaves its in/out arrays unchanged.
 * Threads.  A context may be used by one host thread at a time; separate
 *   contexts are independent.
 */
#ifndef EREM_H
#define EREM_H

#if defined(__GNUC__)
#define EREM_API __attribute__((visibility("default")))
#else
#define EREM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EREM_OK = 0,
  EREM_EINVAL = 1,     /* bad argument, or physically invalid input field    */
  EREM_ENOMEM = 2,     /* device or pinned host allocation failed            */
  EREM_ENOTCONV = 3,   /* Leja interpolation or linear solver did not converge */
  EREM_ETIMEOUT = 4,   /* a pass bound ran out (a batched ensemble member)    */
  EREM_ENONFINITE = 5, /* NaN or Inf in an input or an intermediate result   */
  EREM_ECUDA = 6       /* CUDA runtime error (message in erem_last_error)    */
} erem_status;

/* Arithmetic of the Leja vectors and stencil sweeps.  EREM_FP64: everything
 * in FP64.  EREM_FP32_BULK: the Jacobian coefficients and the Newton vectors
 * q_m are FP32; divided differences, the spectral interval, the running sum
 * P_m, the error estimate and all linear-solver arithmetic stay FP64. */
typedef enum { EREM_FP64 = 0, EREM_FP32_BULK = 1 } erem_precision;

/* Rosenbrock-type schemes of §3.2: ROSM(1) and ROSM(1/2) (eq. ROS with
 * gamma = 1 and 1/2), the two-stage ROS2(1) (eq. ROSMh, Table ros2) and
 * the three-stage ROS3p (Table ros3). */
typedef enum { EREM_ROSM1 = 0, EREM_ROSM_HALF = 1, EREM_ROS2 = 2, EREM_ROS3P = 3 } erem_rosm_scheme;

typedef struct {
  int dim;          /* 2 or 3                                  */
  int nx, ny, nz;   /* cells per direction (nz = 1 in 2D)      */
  double lx, ly, lz; /* domain lengths (lz ignored in 2D)      */
} erem_grid;

/* Constants of the local-equilibrium heat model (§2 with he -> infinity):
 * volumetric capacity C = phi*rhoc_f + (1-phi)*rhoc_s, advective face flux
 * rhoc_f * v_sigma * X(T).  fluid_model = 0: X = T and constant fluid
 * properties.  fluid_model = 1: rho(T)/rho_0 = 1 - 3e-4 (T - 20) and
 * mu(T)/mu_0 = exp(-0.02 (T - 20)); the pressure equation uses the mass
 * mobility K rho/mu, the Darcy flux K/mu, and X = (rho/rho_0) T. */
typedef struct {
  double rhoc_f, rhoc_s;
  double head_left, head_right; /* Dirichlet pressure at x = 0 and x = 1 */
  double T_inflow;              /* Dirichlet temperature at x = 0        */
  int fluid_model;
} erem_physics;

/* Options of the real Leja phi_1 evaluation (§4.2).  Start from
 * erem_default_leja_opts(); a zero tol_a, tol_r, p_order, m_max or avg_window
 * takes its default, max_doublings is used as given (0 = never split). */
typedef struct {
  double tol_a, tol_r;  /* scal = tol_a + tol_r * ||T^n||_inf  (default 1e-6) */
  int p_order;          /* stop when 10^p * mean(e) < 1 (default 2)           */
  int m_max;            /* largest degree before the step is split (150)      */
  int max_doublings;    /* substep doublings before EREM_ENOTCONV (0..6)      */
  int avg_window;       /* number of estimates averaged (5)                   */
  const int* replay;    /* host array [s, m_1..m_s] forcing the substep count
                           and the degrees, or NULL for the stopping rule     */
  int n_replay;         /* entries in replay (1 + s)                          */
  int time_terms;       /* nonzero: time the Leja launches with CUDA events,
                           one pair around each chunk of launches            */
} erem_leja_opts;

typedef struct {
  int substeps;         /* s: substeps of the last phi_1 evaluation           */
  int degree_total;     /* sum of the degrees over the substeps               */
  int degrees[64];      /* degree m_k of substep k                            */
  double alpha, beta;   /* Gershgorin interval of dt*J                        */
  double err_est;       /* mean error estimate at the last stop              */
  int lin_iters;        /* linear-solver iterations (pressure / stages)       */
  double lin_resid;     /* final relative residual of the linear solver      */
  double flux_in;       /* pressure_solve: net Darcy inflow through x = 0     */
  double vmax;          /* pressure_solve: largest |face flux| / face area    */
  double t_ms;          /* wall time of the call, milliseconds                */
  double t_terms_ms;    /* time_terms: summed device time of the chunks of
                           Leja launches (gaps between launches and launches
                           that returned at once after the stop included)    */
  int n_terms_timed;    /* time_terms: Leja terms those chunks computed       */
  int launches;         /* CUDA kernels this call launched                    */
  int n_launches_timed; /* time_terms: Leja kernel launches in t_terms_ms
                           (those after the stop included)                   */
  int degree_phi2;      /* erem_step_forced: degree of the phi_2 interpolation */
  int terms_lagged;     /* 1: the Leja terms of this call took each stopping
                           test in the next launch (small grids, untaped):
                           the running sum was updated at every term         */
} erem_stats;

typedef struct erem_ctx erem_ctx;

/* Fill *opts with the defaults: tol 1e-6 (§5), p = 2 (§4.2: the order of
 * EREM), m_max = 150, 6 doublings, average of 5 estimates (§4.2). */
EREM_API void erem_default_leja_opts(erem_leja_opts* opts);

/* Create a context for one grid: validates the grid, allocates every device
 * buffer the other calls need (no allocation happens per step; staging
 * buffers for host pointers and linear-solver vectors are allocated on their
 * first use) and builds the Leja point table.  The current CUDA device at
 * this call is the context's device.  *out receives the context, or NULL on
 * failure.  Errors: EINVAL (bad grid or physics), ENOMEM, ECUDA. */
EREM_API erem_status erem_create(const erem_grid* grid, const erem_physics* phys,
                        erem_precision prec, erem_ctx** out);

/* Free every resource of the context (NULL is ignored). */
EREM_API erem_status erem_destroy(erem_ctx* ctx);

/* Replace the physics constants (used after a pressure solve has given the
 * velocity scale of a workload).  Takes effect at the next erem_set_state /
 * erem_step / rosm_step. */
EREM_API erem_status erem_set_physics(erem_ctx* ctx, const erem_physics* phys);

/* Steady pressure (§2, eq. masscon4 without storage terms; the paper's
 * initial state is the steady pressure, §5), discretized with the TPFA
 * harmonic transmissibilities of §3.1 and solved by conjugate gradients in
 * FP64, preconditioned by the context's choice (erem_set_pressure_precond:
 * an FP32 multigrid V-cycle by default, a Chebyshev polynomial, or Jacobi).
 *   lnk  [N]  ln K per cell
 *   T    [N]  temperature for the fluid laws (may be NULL: T = 20)
 *   p    [N]  in: initial guess; out: solution
 *   tol       stop when ||b - A p||_2 <= tol ||b||_2 (recursive residual)
 *   maxit     iteration limit; EREM_ENOTCONV (p holds the last iterate)
 * stats (may be NULL): lin_iters, lin_resid, flux_in, vmax, t_ms. */
EREM_API erem_status pressure_solve(erem_ctx* ctx, const double* lnk, const double* T,
                           double* p, double tol, int maxit, erem_stats* stats,
                           void* stream);

/* Set the state that phi1_apply uses: stores copies of the fields,
 * assembles the Darcy face fluxes from p (eq. darcy with TPFA), the
 * Jacobian J = D_T G(T, p) of the heat right-hand side (eq. linear; the
 * finite-volume fluxes of §3.1 with upwind advection) and the Gershgorin
 * interval [alpha, beta] of dt*J (§4.2).
 *   T, p, lnk, phi, lambda [N]; dt > 0.
 * Errors: EINVAL, ENONFINITE, ECUDA. */
EREM_API erem_status erem_set_state(erem_ctx* ctx, const double* T, const double* p,
                           const double* lnk, const double* phi,
                           const double* lambda, double dt, void* stream);

/* out = dt * phi_1(dt * J) v for the J and dt of the last erem_set_state
 * (or erem_step), by real Leja interpolation in Newton form (§4.2, eqs.
 * lejaa, div, newt) with the weighted error estimate and the stopping test
 * 10^p mean(||e||) < 1 of §4.2; when m_max terms do not meet the test the
 * step is split into s = 2, 4, ... substeps (§4.2).
 *   v [N] input vector, out [N] result (may alias v).
 * opts may be NULL (defaults).  stats (may be NULL): substeps, degrees,
 * alpha, beta, err_est, t_ms, t_terms_ms.
 * Errors: EINVAL (no state yet), ENOTCONV (out unchanged), ENONFINITE. */
EREM_API erem_status phi1_apply(erem_ctx* ctx, const double* v, double* out,
                       const erem_leja_opts* opts, erem_stats* stats,
                       void* stream);

/* One EREM step (eq. EERM):
 *   T <- T + dt * phi_1(dt * J_n) G(T, p),   J_n = D_T G(T, p).
 * p, lnk, phi, lambda: the fields of this step, or all NULL to keep the
 * fields of the previous call (with fluid_model = 0 and an unchanged dt the
 * Jacobian and the divided differences are then reused).  With
 * fluid_model = 1, J_n and the Darcy fluxes are re-evaluated at T every step.
 *   T [N] in/out.  Errors as phi1_apply; on error T is unchanged. */
EREM_API erem_status erem_step(erem_ctx* ctx, double* T, const double* p,
                      const double* lnk, const double* phi,
                      const double* lambda, double dt,
                      const erem_leja_opts* opts, erem_stats* stats,
                      void* stream);

/* One step of the non-autonomous EREM scheme (eq. nEERMg, §3.2) for the
 * heat problem whose inflow temperature depends on time:
 *   T <- T + dt phi_1(dt J) G(T, t_n) + dt^2 phi_2(dt J) D_t G(T, t_n),
 * G(T, t_n) with the inflow temperature T_in = T_in(t_n) (instead of the
 * physics' T_inflow) and D_t G = T_in_rate dG/dT_in, non-zero on the x = 0
 * cells only (their Dirichlet conduction and inflowing advection, §3.1).
 * phi_2(z) = (e^z - 1 - z)/z^2.  Both products are Leja interpolations on
 * the interval of dt J (§4.2; the phi_2 divided differences by the same
 * matrix-function route); the phi_2 interpolation is stopped by the same
 * test on its increments dt^2 d_m q_m.  When m_max terms do not suffice the
 * step is split into s pieces of length delta = dt / s: piece k adds
 * delta phi_1(delta J)(J y_k + G + k delta D_t G) + delta^2 phi_2(delta J) D_t G,
 * the exact flow of the linearised equation y' = J y + G + t D_t G.
 * opts->replay, if given, is [s, m_1..m_s, m_phi2] (n_replay = s + 2).
 * stats: as erem_step plus degree_phi2; degree_total counts both parts.
 * Needs fluid_model = 0 (G affine in T and T_in).  Other arguments and
 * errors as erem_step. */
EREM_API erem_status erem_step_forced(erem_ctx* ctx, double* T, double dt, double T_in,
                                      double T_in_rate, const double* p, const double* lnk,
                                      const double* phi, const double* lambda,
                                      const erem_leja_opts* opts, erem_stats* stats,
                                      void* stream);

/* One Rosenbrock-type step (§3.2): ROSM(gamma) (eq. ROS)
 *   T <- T + dt (I - dt gamma J_n)^{-1} G(T)
 * or the s-stage form of eq. ROSMh (autonomous: the gamma_i D_t f terms
 * vanish; the printed diagonal c_ii do not enter the sums over j < i) with
 * Table ros2 (ROS2(1), two stages) or Table ros3 (ROS3p, three stages):
 *   (I/(dt gamma) - J_n) k_i = G(T + sum_{j<i} a_ij k_j) - sum_{j<i} c_ij/dt k_j,
 *   T <- T + sum_i b_i k_i.
 * Every stage system is solved by BiCGSTAB in FP64 (preconditioner:
 * erem_set_stage_precond, a multigrid V-cycle by default) to
 * ||r - A k||_2 <= lin_tol ||r||_2 (maxit iterations).  For ROS2(1) and
 * ROS3p, stats->err_est = RMS over the cells of y - y_hat, the difference to
 * the embedded solution (weights b_hat of the tables: orders 1 and 2).
 * Fields as erem_step.
 * Errors: EINVAL, ENOTCONV, ENONFINITE, ECUDA. */
EREM_API erem_status rosm_step(erem_ctx* ctx, double* T, const double* p,
                      const double* lnk, const double* phi,
                      const double* lambda, double dt,
                      erem_rosm_scheme scheme, double lin_tol, int maxit,
                      erem_stats* stats, void* stream);

/* One step of the coupled pressure/temperature problem by operator
 * splitting (§3.2), with the steady pressure of this library:
 *   EREM_SPLIT_TROTTER (the paper's "sequential approach"): p <- steady
 *     pressure at T^n (CG from the guess in p), then one EREM heat step of
 *     dt with the Darcy fluxes of p (erem_step with the fields);
 *   EREM_SPLIT_STRANG: an EREM heat step of dt/2 with the Darcy fluxes of
 *     the last pressure solve (p, the pressure the previous step ended with,
 *     with the viscosity at T_p, the temperature it was solved at; for the
 *     first step the steady pressure at T^0 and T_p = T^0), p <- steady
 *     pressure at the new T, a second heat step of dt/2 with its fluxes.
 *     With an instantly relaxed pressure the symmetric splitting is first
 *     order like the sequential one (the coupling lags by half a step in
 *     each half).
 *   T [N], p [N] in/out; lnk, phi, lambda [N].  T_p [N] in/out, may be NULL:
 *     in, the temperature p was solved at (NULL: T, right for a first step
 *     and for a pressure solved at T^n; Strang only); out, the temperature the
 *     step's pressure was solved at (T^n for Trotter, the half-step
 *     temperature for Strang), to be passed to the next step; an array of
 *     its own (EINVAL if it is T or p).
 *   pressure_tol, pressure_maxit as pressure_solve.  opts: NULL or an array
 *   of one (Trotter) or two (Strang, one per half step) Leja option structs;
 *   stats: NULL or an array of as many erem_stats for the heat steps; pstats
 *   (may be NULL): the pressure solve.  Errors as pressure_solve and erem_step; on an error of
 *   the second half T holds the state after the first. */
typedef enum { EREM_SPLIT_TROTTER = 0, EREM_SPLIT_STRANG = 1 } erem_splitting;
EREM_API erem_status coupled_step(erem_ctx* ctx, double* T, double* p, double* T_p,
                                  const double* lnk, const double* phi, const double* lambda,
                                  double dt, erem_splitting splitting, double pressure_tol,
                                  int pressure_maxit, const erem_leja_opts* opts,
                                  erem_stats* stats, erem_stats* pstats, void* stream);

/* Adaptive Rosenbrock integration of the stored state (erem_set_state or the
 * last step's fields) over [0, t_end] with ROS2(1) or ROS3p and the error
 * control the paper points to (§3.2.3: Hairer-Wanner): each attempt of
 * length h is one rosm_step; err = RMS(y - y_hat) / (tol_a + tol_r
 * ||T^n||_inf); the attempt is accepted when err <= 1, else T is restored;
 * the next length is h min(facmax, max(0.2, 0.9 err^(-1/p))) with p the
 * scheme's order (2 or 3) and facmax = 5, or 1 right after a rejection; the
 * last step ends at t_end.
 *   T [N] in/out; dt0 > 0 the first length; max_attempts bounds accepted +
 *   rejected attempts (ENOTCONV when t_end is not reached, T then holds the
 *   state at the last accepted time, stats->t_reached).
 *   dts (may be NULL) receives the accepted lengths (capacity max_attempts).
 * Errors: EINVAL (scheme not ROS2/ROS3P, bad tolerances or lengths),
 * ENOTCONV, and those of rosm_step. */
typedef struct {
  int accepted, rejected;
  int lin_iters;        /* BiCGSTAB iterations over all attempts */
  int launches;
  double t_reached;     /* t_end unless max_attempts ran out     */
  double dt_min, dt_max;
  double t_ms;
} erem_adapt_stats;
EREM_API erem_status rosm_integrate(erem_ctx* ctx, double* T, double t_end, double dt0,
                                    erem_rosm_scheme scheme, double tol_a, double tol_r,
                                    double lin_tol, int maxit, int max_attempts, double* dts,
                                    erem_adapt_stats* stats, void* stream);

/* Steady pressure solve that allocates nothing (the paper has no
 * counterpart: this entry point exists for callers that cannot allocate).
 * Callers that run under a device-memory budget fixed at start-up, inside a
 * host callback, or under another runtime's allocator cannot call
 * cudaMalloc; erem_create does, so they could not reach pressure_solve.
 * This call needs no context: it runs the Jacobi-preconditioned CG of
 * pressure_solve (erem_set_pressure_precond degree 1), with its work vectors, reduction partials and control
 * block in one static device array compiled into the library (about 5.8 MB).
 * The runtime loads the library's device code lazily: the first call on a
 * device loads it there, which places the array in that device's memory, so
 * a caller under a fixed budget sees those 5.8 MB taken by its first call
 * (make it at start-up); the array then stays until the process exits, and
 * later calls take no device memory.
 *   grid, phys  as for erem_create (only the heads and fluid_model are used)
 *   lnk [N], T [N] (may be NULL: T = 20), p [N] in: guess, out: solution;
 *   all three must be device memory of the current device, or managed
 *   memory (host arrays, pinned or not, are refused: staging would allocate).
 *   tol, maxit as for pressure_solve; stats as for pressure_solve, with t_ms
 *   the host wall time of the call (it waits for its kernels).
 * Limit: round_up(nx, 4) * ny * nz <= 65536 cells, else EREM_EINVAL.
 * Every call looks up the array's device address with the current device
 * (after a device reset the module, and the array, are loaded anew); make
 * the first call on a device before any stream capture.  Every
 * call shares the array and finds there what the last call left; the call
 * clears what must start at zero, but calls that overlap on the GPU (from
 * other streams or threads) race on it.  The call calls no cudaMalloc or
 * cudaFree.  Errors: EINVAL, ENONFINITE, ENOTCONV, ECUDA (no message string:
 * there is no context to hold one). */
EREM_API erem_status erem_pressure_solve_static(const erem_grid* grid,
                                                const erem_physics* phys,
                                                const double* lnk, const double* T,
                                                double* p, double tol, int maxit,
                                                erem_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Krylov (Arnoldi) phi_1, the alternative of §4.1: phi_1(tau J) v is
 * approximated on a Krylov subspace of dimension m built by Arnoldi's
 * algorithm with modified Gram-Schmidt (Algorithm alg:al2) as
 * ||v|| V_{m+1} phi_1(tau Hbar_{m+1}) e_1 (eq. approphi).  The step is split
 * into substeps of y' = J y + v (each with its own basis from J y + v) whose
 * lengths follow a local error estimate from the first term of the expansion
 * that eq. approphi drops; a substep is accepted when that estimate is at
 * most 1.2 tol delta / tau, tol = (tol_a + tol_r ||T^n||_inf) sqrt(N), and
 * the next length is 0.9 delta (tol delta / (tau err))^(1/m).  Everything
 * runs in FP64 (the cell-form Jacobian), whatever the context's precision.
 * ------------------------------------------------------------------------ */
typedef struct {
  double tol_a, tol_r;  /* default 1e-6 each                                 */
  int m;                /* Krylov dimension, 1..32 (default 10, §5)          */
  int max_substeps;     /* substeps before EREM_ENOTCONV (default 1000)      */
  const double* replay; /* host array: substep lengths to take instead of the
                           error control, or NULL                            */
  int n_replay;         /* entries in replay                                 */
} erem_krylov_opts;

typedef struct {
  int substeps;         /* accepted substeps                                 */
  int rejections;       /* rejected substep lengths                          */
  int dims[64];         /* Krylov dimension of the first 64 substeps (m, or
                           less after a breakdown: an invariant subspace)    */
  double deltas[64];    /* their lengths                                     */
  double err[64];       /* their local error estimates                       */
  double t_ms;          /* wall time of the call                             */
  int launches;         /* CUDA kernels the call launched                    */
  int pad;
} erem_krylov_stats;

/* Defaults: tol 1e-6, m = 10, 1000 substeps, no replay. */
EREM_API void erem_default_krylov_opts(erem_krylov_opts* opts);

/* out = dt phi_1(dt J) v by Krylov substeps, for the J and dt of the last
 * erem_set_state (as phi1_apply).  opts and stats may be NULL.
 * Errors: EINVAL (no state, m outside 1..32), ENOTCONV (substep or rejection
 * limit; out unchanged), ENONFINITE, ECUDA. */
EREM_API erem_status phi1_apply_krylov(erem_ctx* ctx, const double* v, double* out,
                                       const erem_krylov_opts* opts, erem_krylov_stats* stats,
                                       void* stream);

/* One EREM step (eq. EERM) with phi_1 by Krylov substeps; arguments and
 * field handling as erem_step. */
EREM_API erem_status erem_step_krylov(erem_ctx* ctx, double* T, const double* p,
                                      const double* lnk, const double* phi,
                                      const double* lambda, double dt,
                                      const erem_krylov_opts* opts, erem_krylov_stats* stats,
                                      void* stream);

/* ------------------------------------------------------------------------
 * Adjoint of EREM steps: gradients of a function L of the temperatures with
 * respect to T^0 and to ln K, for the linear fluid model (fixed Darcy field
 * from one steady pressure solve).  The paper has no adjoint; each step is
 * differentiated as the map it computes with its Leja schedule and spectral
 * interval frozen: the Newton polynomial of §4.2 in J, whose transpose is
 * the same polynomial in J^T (evaluated backwards by Horner's rule).  The
 * derivative with respect to ln K runs through the upwind face fluxes and the
 * steady pressure (one adjoint pressure solve, Jacobi CG in FP64).
 *
 * Use, after a forward run of erem_step on this context:
 *   erem_adjoint_begin(ctx);
 *   lam = dL/dT^N;  for n = N-1 .. 0: erem_adjoint_step(ctx, T^n, lam, sched_n)
 *   (lam becomes dL/dT^n; T^n is recomputed by the caller from checkpoints,
 *   e.g. by erem_step with the schedules replayed);
 *   erem_adjoint_lnk(ctx, lnk, glnk, ...)  -> dL/dlnK.
 * ------------------------------------------------------------------------ */

/* Adjoint tape.  record = 1: reserve a device arena of at least `bytes`
 * (kept across calls, freed with the context), clear it, and from now on let
 * every erem_step (fluid_model 0) record what erem_adjoint_step would
 * otherwise recompute for that step: the start of every substep after the
 * first (FP64 [N] each) and the Newton vectors q_0..q_m of every substep (in
 * the Leja precision).  A step that does not fit is not recorded.
 * erem_adjoint_step uses the last record when its schedule is the step's and
 * then releases it (last in, first out), so replaying a checkpoint segment
 * forward with the tape on and then stepping back through it computes every
 * Newton vector once per segment instead of twice; the gradient is bitwise
 * the same.  record = 0: stop recording and drop the records (the arena is
 * kept).  Bytes per step: (s - 1) 8 N' + sum_k (m_k + 1) q N' with N' the
 * padded cell count (round_up(nx, 4) ny nz) and q = 4 (FP32-bulk) or 8.
 * Errors: EINVAL, ENOMEM. */
EREM_API erem_status erem_adjoint_tape(erem_ctx* ctx, size_t bytes, int record);

/* Clear the accumulated derivative with respect to the face fluxes.
 * Errors: EINVAL (no state, fluid_model != 0), ENOMEM, ECUDA. */
EREM_API erem_status erem_adjoint_begin(erem_ctx* ctx, void* stream);

/* One step backwards: lam [N] holds dL/dT^{n+1} on entry and dL/dT^n on
 * return, for the step the context took from T [N] = T^n with the schedule
 * [s, m_1..m_s] (erem_stats.substeps and .degrees of that step); the step's
 * contribution to dL/dF is added to the accumulator.  The J, dt and interval
 * are the context's current ones (those of the forward run).
 * Errors: EINVAL (bad schedule, no state, fluid_model != 0), ENOMEM, ECUDA. */
EREM_API erem_status erem_adjoint_step(erem_ctx* ctx, const double* T, double* lam,
                                       const int* schedule, int n_schedule, void* stream);

/* glnk [N] = dL/dlnK from the accumulated dL/dF, for lnk [N] the field of
 * the forward run (its steady pressure must be the one given to
 * erem_set_state).  The adjoint pressure system is solved to
 * ||r|| <= tol ||b|| (maxit iterations); stats (may be NULL): lin_iters,
 * lin_resid.  Errors: EINVAL, ENOTCONV, ECUDA. */
EREM_API erem_status erem_adjoint_lnk(erem_ctx* ctx, const double* lnk, double* glnk, double tol,
                                      int maxit, erem_stats* stats, void* stream);

/* Point set of the Leja interpolation (§4.2) for later calls on ctx.
 *   EREM_LEJA_EXACT (default): eq. lejaa, each point maximises
 *     prod_k |xi - xi_k| over the whole interval (ties to the smaller point).
 *   EREM_LEJA_FAST: the "fast" variant named in the title of §4.2 (the
 *     candidate rule of Baglama, Calvetti and Reichel): xi_0 = 2, xi_1 = -2,
 *     then the midpoint of a gap between consecutive chosen points with the
 *     largest product (ties to the smaller point); the points are dyadic.
 * The divided differences are recomputed for the new points; replayed
 * schedules keep their meaning (degrees per substep).  The batched ensemble
 * keeps the exact points.  Errors: EINVAL (ctx NULL, unknown kind). */
typedef enum { EREM_LEJA_EXACT = 0, EREM_LEJA_FAST = 1 } erem_leja_kind;
EREM_API erem_status erem_set_leja_points(erem_ctx* ctx, int kind);

/* Substep count the first attempt of a step takes (phi1_apply, erem_step,
 * the heat steps of coupled_step; not replayed steps).  §4.2 splits a step
 * whose interpolation needs more than m_max terms and fixes only that
 * doubling, not where it starts:
 *   EREM_SUBSTEPS_FROM_ONE (default): every step starts at one substep;
 *   EREM_SUBSTEPS_FROM_LAST: a step starts at the count the last step on
 *     ctx passed with (capped at 2^max_doublings) and doubles from there, so
 *     a run whose interval keeps needing s substeps does not repeat the
 *     failing attempts below s every step; it never goes back down.
 * erem_set_state restarts the count at one.  Errors: EINVAL (ctx NULL,
 * unknown mode). */
typedef enum { EREM_SUBSTEPS_FROM_ONE = 0, EREM_SUBSTEPS_FROM_LAST = 1 } erem_substep_start;
EREM_API erem_status erem_set_substep_start(erem_ctx* ctx, int mode);

/* Preconditioner of the pressure CG (pressure_solve, erem_adjoint_lnk) for
 * later calls on ctx.  degree 0: one multigrid V-cycle (aggregates of 2 x 2
 * (x 2) cells, Galerkin coarse operators, nu Chebyshev-Jacobi smoothing
 * steps on [1/4, 2] before and after, the coarse correction weighted by
 * omega, the coarsest level of <= 512 cells solved by its inverse, formed
 * once per solve; FP32;
 * parameters by erem_set_pressure_multigrid, default nu = 3, omega = 1.8).
 * degree 1: Jacobi (diagonal) preconditioning, plain CG
 * in FP64.  degree 2..64: z = p(D^-1 A) D^-1 r, `degree` steps of Chebyshev
 * iteration for A z = r on the interval [2/degree^2, 2] (D the diagonal of A,
 * the spectrum of D^-1 A lies in (0, 2]), applied in FP32; the outer CG stays
 * FP64 with the Polak-Ribiere beta (flexible CG), so the stopping rule and
 * accuracy of pressure_solve are unchanged and lin_iters counts outer
 * iterations.  Default 0 (multigrid).  Needs 8 FP32 vectors [N] (and the
 * coarse levels, about N/2 more in 2D) allocated on first use.
 * The paper's solver is BiCGSTAB with ILU(0) (§3.2.3, §5); both are
 * preconditioned Krylov methods for the same system.
 * Errors: EINVAL (ctx NULL, degree outside 0..64). */
EREM_API erem_status erem_set_pressure_precond(erem_ctx* ctx, int degree);

/* Host arrays for erem_step's T.  mode 1 (default): when T is page-locked
 * host memory mapped into the GPU's address space (cudaHostAlloc /
 * cudaMallocHost; reached over NVLink-C2C on Grace systems), the fused
 * linear-model path applies (fluid_model 0) and nx is a multiple of 4, a
 * streaming kernel reads T once into the context's copy of T^n and the
 * step's last kernel writes T^{n+1} directly: one pass each way, no staging
 * copies; the call returns after the write is complete.  mode 0, other host
 * memory and the other entry points: T is copied to a context buffer and
 * back.  Errors: EINVAL. */
EREM_API erem_status erem_set_host_access(erem_ctx* ctx, int mode);

/* Preconditioner of the Rosenbrock stage systems (sigma I - J) k = r for
 * later rosm_step / rosm_integrate calls: 0 = Jacobi BiCGSTAB; 1 (default)
 * = BiCGSTAB with one multigrid V-cycle as right preconditioner (aggregates
 * of 2 x 2 (x 2) cells, a Galerkin coarse operator with one coupling per
 * direction, two damped Jacobi sweeps (weight 0.8) before and after, 40 on
 * the coarsest level of <= 512 cells; FP32; a fixed linear map up to
 * rounding).  The stage tolerance and its meaning are unchanged.
 * Errors: EINVAL. */
EREM_API erem_status erem_set_stage_precond(erem_ctx* ctx, int kind);

/* Multigrid parameters (degree 0 above): nu in 1..16, omega in (0, 2).
 * Errors: EINVAL. */
EREM_API erem_status erem_set_pressure_multigrid(erem_ctx* ctx, int nu, double omega);

/* Hold the Gershgorin interval of J (§4.2, before the factor dt: the interval
 * of dt J becomes [dt lo, dt hi]) at [lo, hi] for every later step of ctx
 * instead of bounding it from the assembled J; hold = 0 releases it (lo, hi
 * ignored).  With the Leja schedules replayed this evaluates exactly the map
 * that erem_adjoint_step differentiates (interval and degrees frozen at the
 * forward run's), e.g. for finite-difference checks under perturbed fields.
 * lo and hi of a forward step are erem_stats.alpha / dt and .beta / dt.
 * Errors: EINVAL (ctx NULL; lo or hi not finite, or lo > hi). */
EREM_API erem_status erem_hold_interval(erem_ctx* ctx, int hold, double lo, double hi);

/* Coefficient arrays per cell in ctx's Leja copy of J (§4.2: the operator
 * every Leja term applies): 5 (2D) or 7 (3D) with the diagonal; 4 or 6 for
 * an FP32-bulk context whose assembled J has every row off the x = 0 inflow
 * plane summing to zero within 2^-28 of the row's couplings (a
 * divergence-free Darcy flux with the linear fluid model): the term then
 * forms sum_j J_ij (q_j - q_i) + r_i q_i with r_i kept for the x = 0 cells
 * only, one array fewer to stream (the environment variable
 * EREM_LEJA_DIAG=1, read at assembly, keeps the diagonal).  0 if ctx is
 * NULL or has no state yet. */
EREM_API int erem_leja_coefficients(const erem_ctx* ctx);

/* Message of the last failing call on ctx ("" if none; a static message if
 * ctx is NULL).  The pointer stays valid until the next call on ctx. */
EREM_API const char* erem_last_error(const erem_ctx* ctx);

/* Host-only helpers (no GPU needed) that expose the FP64 scalar side of the
 * Leja method; the device path uses the same routines.
 * erem_leja_points: xi_0..xi_M on [-2, 2] (eq. lejaa with xi_0 = 2, ties to
 *   the smaller point); returns 0, or -1 for M < 0 or M > 4096.
 * erem_phi1_divided_differences: d_j = phi_1[xi_0..xi_j] of
 *   xi -> phi_1(c + gamma xi), j = 0..M, the first column of
 *   phi_1(c I + gamma L_hat) (§4.2); returns 0, or -1 on bad arguments.
 * erem_phi2_divided_differences: the same for phi_2 (eq. nEERMg). */
EREM_API int erem_leja_points(int M, double* xi);
/* erem_fast_leja_points: the EREM_LEJA_FAST points xi_0..xi_M (see
 *   erem_set_leja_points); returns 0, or -1 for M < 0 or M > 4096. */
EREM_API int erem_fast_leja_points(int M, double* xi);
EREM_API int erem_phi2_divided_differences(int M, const double* xi, double c, double gamma,
                                           double* d);
EREM_API int erem_phi1_divided_differences(int M, const double* xi, double c,
                                  double gamma, double* d);

/* ------------------------------------------------------------------------
 * Batched ensembles.  The paper treats one realization at a time (§5); an
 * ensemble of independent 2D realizations of different sizes runs here as a
 * batch: every member takes exactly the EREM step of erem_step (fluid_model
 * 0: fixed Darcy fluxes, so J and the divided differences are set once per
 * member), and one run advances every member by the same number of steps.
 *
 * On the device every member is a small state machine (G(T^n) -> Leja terms
 * with the stopping test of §4.2 -> substep bookkeeping -> T^{n+1}) whose
 * phases are passes over the member's cells.  One launch runs the whole
 * run: a persistent grid of thread-block clusters takes members from a queue
 * (heaviest first) and each cluster runs its member through every step,
 * with the cluster barrier between passes and the pass's reduction shared
 * through distributed shared memory, so members proceed at their own Leja
 * degrees and substep counts and a member's Leja vectors and coefficients
 * stay in L2 while its cluster works on it.  Stopping, substep doubling and
 * the end of the run are decided on the device.  A member is bounded: it
 * stops after steps * (sum over substep levels of 2^l (m_max + 3) + 2) + 2
 * passes at most (EREM_ETIMEOUT).
 * ------------------------------------------------------------------------ */
typedef struct erem_ens erem_ens;

/* Where each step's substep count starts.  KEEP: at the count the member's
 * previous step passed with (the first step of a member starts at 1, or at
 * what erem_ensemble_autotune found).  RESTART: at 1 every step, doubling
 * on failure as erem_step does (the results then equal erem_step's). */
typedef enum { EREM_ENS_KEEP_SUBSTEPS = 0, EREM_ENS_RESTART_SUBSTEPS = 1 } erem_ens_policy;

typedef struct {
  int substep_policy;  /* erem_ens_policy (default KEEP)                    */
  int cluster_ctas;    /* CTAs of the cluster that runs one member: 2, 4, 8
                          or 16; 0 = 8, or the size erem_ensemble_autotune
                          chose                                             */
  int max_clusters;    /* 0: as many clusters as fit on the device at once */
  int reserved;        /* must be 0                                        */
} erem_ens_config;

typedef struct {
  int status;          /* EREM_OK, EREM_ENOTCONV, EREM_ENONFINITE or
                          EREM_ETIMEOUT                                     */
  int steps_done;      /* steps of the last run this member completed     */
  int substeps;        /* substeps of its last completed step              */
  int degree_total;    /* sum of that step's degrees                       */
  int degrees[64];     /* degree of each substep of that step              */
  int terms;           /* Leja terms evaluated in the last run (failed
                          attempts included)                               */
  int passes;          /* other passes over its cells in the last run      */
  int attempts;        /* failed attempts (substep doublings) in the run   */
  int leja_coefficients; /* arrays per cell of its Leja copy of J (as
                          erem_leja_coefficients: 5, or 4 without the
                          diagonal)                                          */
  double alpha, beta;  /* Gershgorin interval of dt*J                      */
} erem_ens_member_stats;

typedef struct {
  double t_ms;           /* device time of the last run (CUDA events)      */
  long long passes;      /* passes over member cells in the last run, summed
                            over members (Leja terms and the other passes) */
  long long cells;       /* sum of the members' cells                      */
  long long cell_terms;  /* sum over members of cells x Leja terms         */
  long long cell_passes; /* sum over members of cells x other passes       */
  int cluster_ctas;      /* CTAs per cluster of the last run                */
  int clusters;          /* clusters launched (resident at once)           */
  int cta_threads;       /* threads per CTA                                */
  int members_failed;
  int graph;             /* 1: the run was replayed from its captured CUDA
                            graph (uploads, the launch, the read-back);
                            0: launched directly (capture unavailable)     */
  int reserved;
} erem_ens_run_stats;

/* Create an ensemble of n_members 2D members (grids[e].dim must be 2),
 * each with its own grid and physics (fluid_model 0).  Allocates every
 * member's buffers (as erem_create does for each) and the batch tables.
 * Errors: EINVAL, ENOMEM, ECUDA. */
EREM_API erem_status erem_ensemble_create(int n_members, const erem_grid* grids,
                                          const erem_physics* phys, erem_precision prec,
                                          erem_ens** out);
EREM_API erem_status erem_ensemble_destroy(erem_ens* ens);

/* Member e's initial state and fields, as erem_set_state (T, p, lnk, phi,
 * lambda of that member's size; dt > 0).  The ensemble keeps T on the
 * device from here on.  Errors as erem_set_state. */
EREM_API erem_status erem_ensemble_set_member(erem_ens* ens, int e, const double* T,
                                              const double* p, const double* lnk,
                                              const double* phi, const double* lambda,
                                              double dt, void* stream);

/* Replace member e's temperature by T [N_e] (device or host), keeping its
 * fields, Jacobian and divided differences (a restart from a saved state).
 * Errors: EINVAL (no state yet, bad index), ECUDA. */
EREM_API erem_status erem_ensemble_set_temperature(erem_ens* ens, int e, const double* T,
                                                   void* stream);

/* Copy member e's current temperature into T [N_e] (device or host). */
EREM_API erem_status erem_ensemble_get_member(erem_ens* ens, int e, double* T, void* stream);

/* Leja options (as for erem_step; replay and time_terms are not accepted,
 * avg_window is at most 64) and batching configuration; either pointer may
 * be NULL (defaults). */
EREM_API erem_status erem_ensemble_configure(erem_ens* ens, const erem_leja_opts* opts,
                                             const erem_ens_config* cfg);

/* Cluster-size and substep autotuner: runs probe_steps steps of the whole
 * ensemble once to learn every member's substep level and work (the queue
 * order), then once for each cluster size that fits the device (2, 4, 8, 16
 * CTAs), keeps the fastest, and restores every member's temperature
 * afterwards.  The timing stands for runs of about probe_steps steps: a
 * short run ends with its heaviest member alone, which favours large
 * clusters, a long one is bound by throughput.  Under the KEEP policy each member then starts at the substep
 * count its first probe step passed with (the count erem_step would also
 * reach, by doubling).  Errors as erem_ensemble_run. */
EREM_API erem_status erem_ensemble_autotune(erem_ens* ens, int probe_steps, void* stream);

/* Advance every member by `steps` EREM steps (one kernel launch).  The run
 * (the member states and queue order uploaded from pinned host memory, the
 * persistent launch, the states read back) is captured once as a CUDA graph
 * per run configuration (the members' tables, the options, the cluster
 * shape) and replayed on `stream`; where capture is not available it is
 * launched directly (erem_ensemble_run_stats.graph tells which).  Returns
 * when the run is complete.  A member whose Leja interpolation fails (the
 * stopping test not met within m_max terms, or a non-finite estimate: the
 * Newton vectors left the range of the Leja precision) takes its step again
 * at twice the substeps, up to max_doublings times.  A member that fails
 * beyond that, or whose state is not finite, keeps the temperature of the
 * start of its failing step and stops; the call then returns the first
 * failing member's status (ENOTCONV, ENONFINITE or ETIMEOUT) and
 * erem_ensemble_member_stats tells which members failed.
 * Errors: EINVAL (a member without state), ENOTCONV, ENONFINITE, ETIMEOUT,
 * ECUDA. */
EREM_API erem_status erem_ensemble_run(erem_ens* ens, int steps, void* stream);

EREM_API erem_status erem_ensemble_member_stats(const erem_ens* ens, int e,
                                                erem_ens_member_stats* out);
EREM_API erem_status erem_ensemble_run_stats(const erem_ens* ens, erem_ens_run_stats* out);
EREM_API const char* erem_ensemble_last_error(const erem_ens* ens);

#ifdef __cplusplus
}
#endif

#endif /* EREM_H */
