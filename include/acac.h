/*
 * acac.h — C ABI of the GB300 (sm_103a) solver for one implicit time step of the
 * energy-stable discrete-variational-derivative (DVD) scheme for the coupled
 * Allen–Cahn / Cahn–Hilliard system of Huang, Yang & Wei, "Parallel energy-stable
 * solver for a coupled Allen–Cahn and Cahn–Hilliard system" (arXiv 2007.04560).
 *
 * The step solves F(X) = 0 of scheme (NSOA-1) (Sec. 2):
 *     (U^{n+1} - U^n) / dt = -A~ G~^S,    A~ = diag(-div c grad, c / rho),
 * with the Newton–Krylov–Schwarz method of Sec. 3.1 and the adaptive time step
 * of Sec. 3.2 (Eq. sencondt).
 *
 * Conventions shared by every entry point:
 *   - Grid: cell-centred, Nx x Ny (x Nz), spacing L/N per direction (Sec. 2).
 *     A field is a contiguous array of N = Nx*Ny(*Nz) values, x fastest.
 *   - A "state vector" is 2N contiguous values: the u field, then the v field.
 *     Residuals, Newton directions and Krylov vectors use the same layout.
 *   - Pointers named u, v, X, F, w, y, r, z, b, x, J are DEVICE pointers owned by
 *     the caller unless the name ends in _host.  Scalar outputs (double*, int*)
 *     are HOST pointers; NULL means "not wanted".
 *   - "Krylov precision": double when params.precision == ACAC_FP64, float when
 *     ACAC_MIXED.  Arguments typed void* below are in Krylov precision.
 *   - All device work is enqueued on the stream given to acac_create.  Calls that
 *     return host scalars or take decisions on device norms synchronise that
 *     stream; the others only enqueue.
 *   - Return value: ACAC_OK (0) or a negative ACAC_E_* code.  On error the
 *     caller's fields are left unchanged by acac_step / acac_step_host.
 *   - The handle owns all workspace (allocated in acac_create, freed in
 *     acac_destroy).  A handle is not thread-safe.
 */
#ifndef ACAC_H
#define ACAC_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define ACAC_OK               0
#define ACAC_E_ARG           -1   /* bad size, coefficient, partition or pointer     */
#define ACAC_E_CUDA          -2   /* a CUDA runtime call failed                      */
#define ACAC_E_DOMAIN        -3   /* input state outside the admissible set (Sec. 2:
                                     u+v and u-v in (0,1))                            */
#define ACAC_E_DIVERGED      -4   /* NKS failed (Newton maxit, line search, GMRES
                                     maxit, ILU pivot, non-finite norm)               */
#define ACAC_E_DT_UNDERFLOW  -5   /* adaptive retry pushed dt below dt_min (Sec. 3.2) */
#define ACAC_E_TIMEOUT       -6   /* a bounded device-side wait gave up              */
#define ACAC_E_NOMEM         -7   /* device or host allocation failed                */

/* ---- enumerations ---------------------------------------------------------- */
#define ACAC_BC_PERIODIC     0
#define ACAC_BC_NEUMANN      1    /* n.grad u = n.grad v = n.(c grad dE/du) = 0 (Sec. 1) */
#define ACAC_DT_FIXED        0
#define ACAC_DT_ADAPTIVE     1    /* Eq. sencondt with retry and eta doubling (Sec. 3.2)  */
#define ACAC_RAS_LEFT        0    /* sum_k R_k^0T inv(A_k) R_k^delta   (Sec. 3.1)        */
#define ACAC_RAS_AS          1    /* sum_k R_k^dT inv(A_k) R_k^delta   (Eq. invM)        */
#define ACAC_RAS_RIGHT       2    /* sum_k R_k^dT inv(A_k) R_k^0       (Sec. 3.1)        */
#define ACAC_FP64            0    /* every step of the solve in double                     */
#define ACAC_MIXED           1    /* Jacobian, Krylov vectors and ILU in float; residual,
                                     Newton update, energy, mass, dt estimator in double   */
#define ACAC_JAC_MATFREE     0    /* GMRES products by the analytic Jacobian action      */
#define ACAC_JAC_ASSEMBLED   1    /* GMRES products by the assembled stencil matrix      */
#define ACAC_MAX_BATCH       1024 /* largest ensemble (params.batch)                      */
#define ACAC_SUB_ILU0        0    /* subdomain solve by ILU(0), no fill (Sec. 3.1)        */
#define ACAC_SUB_ILU1        1    /* ILU with one level of fill (Sec. 4.2, Table 2)        */
#define ACAC_SUB_ILU2        2    /* ILU with two levels of fill (Sec. 4.2, Table 2)       */
#define ACAC_SUB_LU          3    /* exact LU of the subdomain matrix (Sec. 3.1, Table 2)  */

/* Problem and solver settings.  Defaults: acac_default_params(). */
typedef struct acac_params {
    int    dim;                 /* 2 or 3                                                */
    int    n[3];                /* Nx, Ny, Nz; each >= 4                                */
    double L[3];                /* domain lengths; dx = L[0]/n[0], ...                  */
    int    bc;                  /* ACAC_BC_*                                             */
    double alpha, beta, theta, gamma, rho;   /* > 0, Eq. 2 and Eq. 1                     */
    int    taylor_S;            /* series terms of Lemma 2.2, 1..30 (paper: 10)          */
    int    dt_mode;             /* ACAC_DT_*                                             */
    double dt0, dt_min, dt_max, eta0;        /* first step, bounds, eta of Eq. sencondt  */
    double newton_rtol, newton_atol;         /* eps_r, eps_a (Sec. 3.1)                  */
    int    newton_maxit;
    double gmres_rtol, gmres_atol;           /* xi_r, xi_a (Sec. 3.1)                    */
    int    gmres_restart;       /* 1..64                                                 */
    int    gmres_maxit;
    int    ras_parts[3];        /* subdomain boxes per direction                        */
    int    ras_overlap;         /* delta, mesh layers (Sec. 3.1)                        */
    int    ras_type;            /* ACAC_RAS_*                                            */
    int    ilu_reuse;           /* 1: factor at the first Newton iteration of each step
                                   and reuse within the step (Sec. 4.2)                  */
    int    precision;           /* ACAC_FP64 | ACAC_MIXED                                */
    int    jac_mode;            /* ACAC_JAC_*                                            */
    int    batch;               /* ensemble size B, 1..ACAC_MAX_BATCH: B independent
                                   problems of this size and these settings, each with
                                   its own coefficients (acac_set_coeffs), time step,
                                   eta and history                                       */
    int    cgs_refine;          /* 1: Gram–Schmidt applied twice (CGS2), 0: once         */
    int    graphs;              /* 1: replay each GMRES iteration from a captured CUDA
                                   graph (same kernels and results as 0: direct launches) */
    int    ras_window;          /* 2D Schwarz apply: 0 choose, 1 keep only the last wavefront
                                   levels in shared memory (forward result in global
                                   scratch), 2 keep the whole box vector (shared memory when
                                   it fits, else global); same results                    */
    int    subdomain_solver;    /* ACAC_SUB_*: how inv(A_k) is applied.  Levels of fill
                                   follow the usual definition: lev = 0 on the pattern of
                                   A_k, lev(i,j) = min(lev(i,j), lev(i,k) + lev(k,j) + 1)
                                   in natural order, entries of lev <= p kept.  ILU(1),
                                   ILU(2) and LU: FP64 and mixed; not with the adjoint;
                                   boxes of at most 62,500 cells (ACAC_E_ARG otherwise).   */
} acac_params;

/* Per-step report. */
typedef struct acac_step_info {
    double t;                   /* time after the step                                  */
    double dt;                  /* accepted dt                                          */
    double eta;                 /* eta after the step (doubled on every divergence)     */
    double energy;              /* discrete free energy E~ of the new state (Eq. freeenergy) */
    double mass;                /* sum u dx dy (dz) of the new state                    */
    double fnorm0, fnorm;       /* ||F(X_0)||, ||F(X_final)|| of the accepted solve      */
    int    newton_its;          /* Newton iterations, all attempts of this step         */
    int    gmres_its;           /* GMRES iterations, all attempts of this step          */
    int    divergences;         /* NKS divergences retried in this step                 */
    int    status;              /* ACAC_OK or the error returned                        */
    int    line_search_cuts;    /* halvings of lambda, all attempts                     */
    int    ilu_factorizations;  /* subdomain factorizations performed                   */
} acac_step_info;

typedef struct acac_handle acac_handle;

/* Fill *p with the paper's solver defaults: S = 10, Newton rtol 1e-8 / atol 1e-13,
 * GMRES rtol 1e-6 / atol 1e-14, restart 30, maxit 500, left-RAS, ILU(0) reuse,
 * FP64, matrix-free products, CGS2, unit domain, 64x64 periodic, alpha=3,
 * beta=1, theta=0.3, gamma=1e-3, rho=1, fixed dt 1e-3. */
void acac_default_params(acac_params *p);

/* Validate *p, allocate every workspace on the current CUDA device and build the
 * subdomain tables (Sec. 3.1: boxes of near-equal size extended by delta layers,
 * wrapped when periodic, clipped at Neumann walls).  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  *out receives the handle.
 * Errors: ACAC_E_ARG (sizes < 4, non-positive coefficient, periodic box that
 * would wrap onto itself, subdomain box under 4 or over 250 cells in some
 * direction, a 2D cell in more than four boxes (overlap not below the owned box
 * width), dim not 2 or 3, batch outside 1..ACAC_MAX_BATCH), ACAC_E_NOMEM,
 * ACAC_E_CUDA.
 * Ensembles (batch B > 1): the handle holds B independent problems of this grid and
 * box decomposition and solves them in lockstep: every kernel launch covers all
 * members, per-member masks on the device say which members take part, and every
 * per-member buffer is B copies at a fixed stride (device memory grows about B-fold).
 * The handle's work runs on a private stream ordered after cuda_stream at the start
 * of each call and before it at the end.  Every member starts with the coefficients
 * of *p. */
int acac_create(const acac_params *p, void *cuda_stream, acac_handle **out);

/* Coefficients alpha, beta, theta, gamma, rho (all > 0, Eq. 2 and Eq. 1) of ensemble
 * member `member` (0..batch-1; 0 for a batch-1 handle) from the next step on.  The
 * member's time-step history is kept.  ACAC_E_ARG on a bad member or value. */
int acac_set_coeffs(acac_handle *h, int member, double alpha, double beta, double theta,
                    double gamma, double rho);

/* One accepted time step, in place: u, v (device, N doubles each) hold U^n on
 * entry and U^{n+1} on return.  The handle keeps U^{n-1}, dt_{n-1}, eta and t for
 * the predictor of Eq. sencondt.  Synchronises the stream.  *info (host, may be
 * NULL) receives the report.  Errors: ACAC_E_DOMAIN, ACAC_E_DIVERGED (fixed dt),
 * ACAC_E_DT_UNDERFLOW (adaptive), ACAC_E_CUDA; fields unchanged on error.
 * Ensembles: u and v hold the B members' fields one after another (B*N doubles
 * each, member-major), info is an array of B reports (or NULL), and every member
 * takes one accepted step with its own dt.  Returns ACAC_OK when every member
 * succeeded, else the status of the first member that failed (each report carries
 * its member's status; a failed member's fields are unchanged). */
int acac_step(acac_handle *h, double *u, double *v, acac_step_info *info);

/* acac_step on HOST arrays: copies u_host, v_host to the device, steps, copies
 * the result back.  Host arrays may be pageable or pinned (B*N doubles each for an
 * ensemble). */
int acac_step_host(acac_handle *h, double *u_host, double *v_host, acac_step_info *info);

/* Discrete free energy E~ = <e~> (Eqs. relations, freeenergy, exact Phi with
 * 0 ln 0 = 0) and mass sum u dx dy of the state (u, v) (device).  Host outputs;
 * synchronises.  ACAC_E_DOMAIN if some u+v or u-v lies outside [0,1].
 * Ensembles: u, v member-major as in acac_step; energy and mass are arrays of B. */
int acac_energy(acac_handle *h, const double *u, const double *v, double *energy,
                double *mass);

/* Release every resource of h (NULL is ignored). */
void acac_destroy(acac_handle *h);

/* Static description of a status code. */
const char *acac_status_string(int status);

/* ---- component entry points (the pieces acac_step is made of) ---------------- */
/* These act on one problem: they return ACAC_E_ARG on an ensemble handle. */

/* F(X1) of scheme (NSOA-1) with X0 = U^n and time step dt (Sec. 2, Eqs. dvds-2,
 * D2-1, dvds-1, NSOA-1):  F_u = (u1-u0)/dt - [div c~ grad G_u],
 * F_v = (v1-v0)/dt + c G_v / rho, mobility at the midpoint state.  X1, X0, F:
 * device state vectors (double).  *fnorm (host, may be NULL) = ||F||_2, which
 * synchronises.  ACAC_E_DOMAIN if a midpoint leaves the admissible set. */
int acac_residual(acac_handle *h, const double *X1, const double *X0, double dt,
                  double *F, double *fnorm);

/* Assembled Jacobian dF/dX1 at (X1, X0, dt) in stencil-diagonal storage, Krylov
 * precision: J[(b*4 + e)*N + cell], e = 0:(u-row,u-col) 1:(u,v) 2:(v,u) 3:(v,v).
 * 2D, b = slot 0..12 in the order (dx,dy) = (0,0),(-1,0),(1,0),(0,-1),(0,1),(-2,0),
 * (2,0),(0,-2),(0,2),(-1,-1),(1,-1),(-1,1),(1,1): J holds 52*N values.
 * 3D, b = slot 0..24: centre; faces -x,+x,-y,+y,-z,+z; two steps -2x,+2x,-2y,+2y,-2z,+2z;
 * edge diagonals (dx,dy,dz) = (-1,-1,0),(1,-1,0),(-1,1,0),(1,1,0),(-1,0,-1),(1,0,-1),
 * (-1,0,1),(1,0,1),(0,-1,-1),(0,1,-1),(0,-1,1),(0,1,1): J holds 100*N values.
 * Couplings to cells outside a Neumann domain are stored as 0 (device). */
int acac_jacobian(acac_handle *h, const double *X1, const double *X0, double dt, void *J);

/* y = J w with J from acac_jacobian (Krylov precision, device). */
int acac_spmv(acac_handle *h, const void *J, const void *w, void *y);

/* y = J(X1) w by the analytic Jacobian action, without assembling J (Krylov
 * precision w, y; double X1, X0). */
int acac_jvp(acac_handle *h, const double *X1, const double *X0, double dt,
             const void *w, void *y);

/* Extract every subdomain matrix A_k = R_k J R_k^T (Eq. invM) from J (as stored by
 * acac_jacobian) and factor it by ILU(0) on the 2x2-block stencil pattern, in the
 * natural order of the box (x fastest, u before v).  ACAC_E_DIVERGED on a zero
 * pivot (synchronises). */
int acac_ras_factor(acac_handle *h, const void *J);

/* z = H^{-1} r with the Schwarz preconditioner of params.ras_type and the factors
 * of the last acac_ras_factor (Krylov precision, device).  Deterministic for every
 * ras_type: where boxes overlap (AS, right-RAS) their values are added per cell in a
 * fixed order. */
int acac_ras_apply(acac_handle *h, const void *r, void *z);

/* Solve J(X1) x = b by restarted right-preconditioned GMRES (Sec. 3.1, Eq.
 * hjacobi) with the Schwarz/ILU(0) preconditioner factored from J(X1), x0 = 0,
 * stopping when the residual estimate <= max(gmres_rtol ||b||, gmres_atol).
 * b, x: double state vectors (device).  *its, *resid: host.  ACAC_E_DIVERGED if
 * gmres_maxit is reached. */
int acac_gmres(acac_handle *h, const double *X1, const double *X0, double dt,
               const double *b, double *x, int *its, double *resid);

/* One inexact-Newton solve of F(X) = 0 at fixed dt from X_0 = U0 (Sec. 3.1, Eq.
 * newton), without time-step control.  U0, U1: double state vectors (device);
 * U1 receives the root.  *info (host) receives fnorm0, fnorm, newton_its,
 * gmres_its, line_search_cuts, ilu_factorizations and status (t, dt, eta,
 * energy, mass are not filled). */
int acac_nks_solve(acac_handle *h, const double *U0, double dt, double *U1,
                   acac_step_info *info);

/* ---- autotuning of the Schwarz partition ---------------------------------------- */

/* Time acac_step for candidate Schwarz partitions of the problem *p and return the
 * fastest in *best (a copy of *p with ras_parts and ras_overlap replaced).  The
 * candidates are *p itself and near-cubic boxes of owned width 12, 16, 24, 32, 48, 64,
 * 96, 128, 192 or 240 cells per direction, each with overlap 1 and 2, that acac_create
 * accepts.  The box shape trades the preconditioner's strength (GMRES iterations)
 * against the length of the triangular sweeps and the parallelism across boxes, so
 * each candidate is timed end to end: one untimed step from (u, v) (device, B*N
 * doubles each for an ensemble of batch B, not modified), then trial_steps timed steps
 * continuing from it (an ensemble is timed as a whole, every member with the
 * coefficients of *p).  *best_ms_per_step and *ncandidates (host, may be NULL) report
 * the best time and the number of candidates tried.  ACAC_E_ARG on bad arguments,
 * ACAC_E_DIVERGED when no candidate completes its steps.  Synchronises. */
int acac_autotune(const acac_params *p, const double *u, const double *v, int trial_steps,
                  void *cuda_stream, acac_params *best, double *best_ms_per_step,
                  int *ncandidates);

/* ---- adjoint of the implicit step (FP64 handles) -------------------------------- */
/* There is no adjoint in the paper; these entry points differentiate its fixed-dt
 * scheme (NSOA-1, Sec. 2) in reverse mode.  With F(U^{n+1}, U^n; p) = 0 per step and
 * J1 = dF/dU^{n+1}, J0 = dF/dU^n:
 *     J1^T mu = lambda^{n+1},   lambda^n = -J0^T mu,   dL/dp += -mu^T dF/dp,
 * for p = (alpha, beta, theta, gamma).  J1^T mu = lambda is solved by GMRES on the
 * transposed assembled Jacobian, preconditioned by the Schwarz/ILU(0) preconditioner
 * of params.ras_type factored from the subdomain blocks of J1^T, to relative residual
 * rtol.  Vectors are double state vectors [u | v] on the device.  ACAC_E_ARG on an
 * ensemble or mixed-precision handle. */

/* dF/dX0 at (X1, X0, dt) in the storage of acac_jacobian (Krylov precision). */
int acac_jacobian_x0(acac_handle *h, const double *X1, const double *X0, double dt, void *J);

/* y = J^T w for J in the storage of acac_jacobian (Krylov precision, device). */
int acac_spmv_t(acac_handle *h, const void *J, const void *w, void *y);

/* Loss L = w_energy E~(X) + (w_misfit / 2) sum ((u - u*)^2 + (v - v*)^2) dx dy of a
 * state X against target = [u* | v*]: *loss (host), dX = dL/dX (device, 2N) and
 * grad[0..3] (host, may be NULL) = dL/d(alpha, beta, theta, gamma) at fixed X.
 * ACAC_E_DOMAIN if some u+v or u-v of X lies outside (0, 1).  Synchronises. */
int acac_loss(acac_handle *h, const double *X, const double *target, double w_energy,
              double w_misfit, double *loss, double *dX, double *grad);

/* One adjoint step at (X1, X0, dt): lam0 = -J0^T mu with J1^T mu = lam1 (lam0 may
 * alias lam1), grad[0..3] (host, may be NULL) = -mu^T dF/d(alpha, beta, theta, gamma),
 * *gmres_its (host, may be NULL).  Synchronises. */
int acac_adjoint_step(acac_handle *h, const double *X1, const double *X0, double dt,
                      const double *lam1, double *lam0, double *grad, double rtol,
                      int *gmres_its);

/* Gradient of L(U^K) (as acac_loss) after nsteps fixed-dt steps from (u0, v0), by the
 * adjoint recursion with a checkpoint every checkpoint_every steps: the forward run
 * keeps those states (and U^K), the backward run recomputes each segment from its
 * checkpoint.  Device: u0, v0, u_target, v_target (N each), du0, dv0 (N each,
 * receive dL/du0, dL/dv0).  Host: *loss, grad[0..3] = dL/d(alpha, beta, theta,
 * gamma), *gmres_its (may be NULL).  Working memory: (nsteps/checkpoint_every + 2 +
 * checkpoint_every) states, allocated for the call.  The handle's time-step history
 * is not used or changed.  Errors as acac_nks_solve and acac_loss.  Synchronises. */
int acac_adjoint(acac_handle *h, const double *u0, const double *v0, int nsteps, double dt,
                 int checkpoint_every, const double *u_target, const double *v_target,
                 double w_energy, double w_misfit, double rtol, double *loss, double *du0,
                 double *dv0, double *grad, int *gmres_its);

/* ---- residual without a handle and without device allocation ------------------- */

/* F(X1) and ||F|| exactly as acac_residual computes them, for callers that may not
 * allocate device memory when they need a residual (code inside a framework that
 * owns every device allocation, allocation-free latency-critical loops, plugins
 * that are handed only their buffers).  There is no counterpart of this entry
 * point in the paper: it is a deployment convenience.
 *   p: validated like acac_create; the grid may have at most 512 x 512 cells
 *      (ACAC_E_ARG beyond that).  X1, X0, F: device state vectors (double, 2N);
 *      *fnorm: host, may be NULL.  cuda_stream: cudaStream_t (NULL = default).
 *   Working memory: file-scope device arrays of about 6 MB, present on every GPU
 *      that loads the library until the process exits; nothing is allocated or
 *      freed per call.
 *   The first call on a device looks up those arrays' device addresses (once per
 *      device, cached for the life of the process); make that first call before any
 *      stream capture.  Every call copies ||F||^2 and a flag back to the host and
 *      synchronises cuda_stream before it returns.  Calls share the arrays: calls
 *      whose work overlaps on the GPU (other streams, other host threads) race.
 *      X1, X0 and F must live on the current device.  After cudaDeviceReset the
 *      cached addresses (and the library's constant tables) are stale: the library
 *      does not support use across a device reset.
 *   Returns ACAC_OK, ACAC_E_ARG, ACAC_E_DOMAIN (a midpoint outside the
 *      admissible set) or ACAC_E_CUDA. */
int acac_residual_noalloc(const acac_params *p, const double *X1, const double *X0, double dt,
                          double *F, double *fnorm, void *cuda_stream);

/* y[i] = ln x[i] (device arrays, n values) with the logarithm the residual and energy
 * kernels use (a table-driven reduction: Tang, ACM TOMS 1990).  Enqueued on
 * cuda_stream; exposed so that its accuracy can be checked against a reference. */
int acac_log(const double *x, double *y, long long n, void *cuda_stream);

/* ---- instrumentation ---------------------------------------------------------- */

/* Kernel classes counted and timed by the handle (one __global__ each, except
 * ACAC_K_VECTOR, which gathers the small vector kernels of GMRES and Newton). */
#define ACAC_K_RESIDUAL_G    0    /* G~^S and mobility per cell (pass A of F)        */
#define ACAC_K_RESIDUAL_F    1    /* F and ||F||^2 partials (pass B of F)             */
#define ACAC_K_LINEARIZE     2    /* per-cell derivative cache                        */
#define ACAC_K_ASSEMBLE      3    /* stencil-diagonal Jacobian                        */
#define ACAC_K_SPMV          4    /* assembled y = J w                                */
#define ACAC_K_JVP_G         5    /* matrix-free J w, pass 1                          */
#define ACAC_K_JVP_F         6    /* matrix-free J w, pass 2                          */
#define ACAC_K_RAS_FACTOR    7    /* batched subdomain ILU(0)                         */
#define ACAC_K_RAS_APPLY     8    /* batched restriction, triangular sweeps, extension */
#define ACAC_K_DOT           9    /* Gram–Schmidt block dot products                  */
#define ACAC_K_CGS_UPDATE   10    /* Gram–Schmidt update (and norm)                   */
#define ACAC_K_REPACK       11    /* Jacobian rows repacked per subdomain cell        */
#define ACAC_K_VECTOR       12    /* other vector kernels                             */
#define ACAC_K_ENERGY       13    /* energy and mass                                  */
#define ACAC_NKERNEL        14

/* Reset the per-kernel counters; enable != 0 also brackets every launch with CUDA
 * events on the handle's stream (durations are collected at the next
 * synchronisation).  Launch counts are kept whether or not timing is enabled.
 * Synchronises the stream. */
int acac_profile(acac_handle *h, int enable);

/* As acac_profile, timing only the launches of the kernel classes whose bit
 * (1 << ACAC_K_*) is set in mask (0: no timing).  Two events per timed launch cost host
 * time; a mask with only the class of interest keeps that cost off the other launches. */
int acac_profile_mask(acac_handle *h, unsigned mask);

/* Since the last acac_profile: launches of kernel class `kernel`, their summed
 * event-timed duration in ms (0 unless timing was enabled), and their summed
 * algorithmic HBM bytes and floating-point operations (the minimum traffic and
 * arithmetic of the operation, from the launch sizes; 0 where not modelled).
 * Any output pointer may be NULL.  Synchronises. */
int acac_kernel_stats(acac_handle *h, int kernel, long long *launches, double *total_ms,
                      double *bytes, double *flops);

/* Static name of a kernel class. */
const char *acac_kernel_name(int kernel);

/* Self-check of the bounded device-side waits (the Schwarz apply's mbarrier waits,
 * mode 0; the dataflow factorization's row waits, mode 1): one warp waits, with the
 * production wait helper, on an mbarrier phase / a done bit that nothing completes.  The
 * wait gives up after its limit (0.5 s / 0.2 s) and the kernel reports it.  Returns
 * ACAC_E_TIMEOUT when the wait gave up (the expected result; the CUDA context stays
 * usable), ACAC_OK if it completed, ACAC_E_ARG for another mode, ACAC_E_CUDA /
 * ACAC_E_NOMEM on a runtime failure.  Enqueued on `stream` (NULL: the default stream);
 * synchronises it. */
int acac_wait_selftest(void *stream, int mode);

/* Measured fused multiply-add rate of the device (instrumentation: the arithmetic peak that
 * the FP64 kernels' rooflines are taken against).  A full-occupancy grid whose threads run
 * eight independent multiply-add chains of `iters` steps each, in double (kind 0) or float
 * (kind 1), timed with CUDA events after one warm-up launch.  Kinds 2..6: double with only
 * the first 16, 8, 4, 2 or 1 lanes of every warp working (what a partly filled warp costs
 * the FP64 pipe).  *tflops receives 2 x chains x iters x working threads / time in TFLOP/s,
 * *ms the timed launch's duration (either may be NULL).
 * Allocates and frees one small output buffer; enqueued on cuda_stream (NULL: the default
 * stream), which it synchronises.  ACAC_E_ARG for another kind or iters < 1.  No
 * counterpart in the paper. */
int acac_peak_probe(int kind, int iters, double *tflops, double *ms, void *cuda_stream);

/* Block pattern of a subdomain factorization with fill (Sec. 4.2, Table 2), host only (no
 * GPU, no handle): the box of W x H (x D) cells in natural order (x fastest), the radius-2
 * stencil of dimension dim, solver ACAC_SUB_ILU1, ACAC_SUB_ILU2 or ACAC_SUB_LU.  One
 * entry per kept 2x2 block (cell pair): row ptr[c]..ptr[c+1]-1 of col holds the kept
 * columns (cell indices) of cell c, sorted.  ptr has n + 1 = W H D + 1 entries and col
 * room for cap entries; *nnz receives the count.  ILU: levels of fill as described at
 * acac_params.subdomain_solver; LU: the profile of each row, a superset of the exact
 * factorization's fill.  ACAC_E_ARG on bad sizes or a cap below *nnz (then only *nnz is
 * written). */
int acac_subdomain_pattern(int dim, int W, int H, int D, int solver, int *ptr, int *col, long long cap,
                           long long *nnz);

#ifdef __cplusplus
}
#endif
#endif /* ACAC_H */
