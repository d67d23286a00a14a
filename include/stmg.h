/*
 * stmg.h -- C ABI of the GB300 (sm_103a) hp space-time multigrid Newton-Krylov library.
 *
 * The library solves the local slab problem of a tensor-product space-time finite element
 * discretisation of the incompressible Navier-Stokes equations: mapped Q_{r+1}^d / P_r^disc
 * in space (Sec. 2.2, Def. VKQK), DG(k) in time with the Lagrange basis at the right
 * Gauss-Radau points (Sec. 3.1, Eq. GF, BasYk), Nitsche boundary conditions on the whole
 * boundary (Eq. def-b-gam, def-a-gam-tp), convection in divergence form (Eq. ns-form-tp)
 * integrated in time by the reduced Radau rule (Eq. QuadNL, AlgFconv).  The slab residual
 * is Problem LocAlgNS (Eq. InAlgNS), its Jacobian Eq. JacobianLocal0-1.
 *
 * Vector layout (one slab, Eq. DefSubvec): [V^1 .. V^{k+1} | P^1 .. P^{k+1}].
 *   V^a: velocity at Radau node a, component-major: all x-components over the global node
 *        grid N1^d (N1 = (r+1) n + 1, lexicographic, x fastest), then y, then z.
 *   P^a: pressure modes, cell-major (cells lexicographic, x fastest), C(r+d,d) modes per
 *        cell: tensor Legendre P_i(2x-1) P_j(2y-1) [P_l(2z-1)] with i+j(+l) <= r, ordered by
 *        total degree, then ascending degree of the last coordinate.
 *
 * Ownership: every vector argument is a DEVICE pointer owned by the caller unless stated
 * otherwise; its element type follows the precision argument (double for STMG_FP64, float
 * for STMG_FP32).  The handle owns meshes, level data, smoother factors and Krylov scratch.
 * Work is enqueued on the handle's stream; a call returns after enqueueing unless it needs a
 * device scalar (norms, Krylov control), in which case it synchronises that stream.
 * Errors: every call returns a stmg_status; stmg_last_error() describes the last failure of a
 * handle.  No C++ exception crosses the ABI.  A handle is used by one host thread at a time;
 * distinct handles are independent.
 */
#ifndef STMG_H
#define STMG_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stmg_handle stmg_handle;
typedef void* stmg_stream; /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
  STMG_OK = 0,
  STMG_ERR_ARG = 1,           /* invalid argument or unsupported size */
  STMG_ERR_OOM = 2,           /* device allocation failed */
  STMG_ERR_CUDA = 3,          /* a CUDA call failed */
  STMG_ERR_NOT_CONVERGED = 4, /* Newton reached its iteration cap (or stalled, newton_stall_steps) */
  STMG_ERR_NUMERIC = 5,       /* NaN / Inf detected */
  STMG_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
  STMG_ERR_UNSUPPORTED = 7    /* configuration not compiled in */
} stmg_status;

typedef enum { STMG_FP64 = 0, STMG_FP32 = 1 } stmg_precision;

/* Analytic data sets of the bundled workloads (f, g, v0).  STMG_CAV3D: the lid-driven cavity of
   Sec. 5.2 on [0,1]^3 -- f = 0, v0 = 0, no-slip walls, and on the lid z = 1 the tangential
   velocity (sin(pi t / 4), 0, 0) (the paper prints the scalar profile; the lid moves along x). */
typedef enum { STMG_TG2D = 0, STMG_MMS2D = 1, STMG_TG3D = 2, STMG_MMS3D = 3, STMG_CAV3D = 4,
               STMG_USER = 5 /* f, g, v0 from caller callbacks (stmg_set_data, stmg_initial_condition);
                                zero until stmg_set_data is called */ } stmg_problem;

/* A vector field given by the caller (Sec. 2, Problem 2.1: the body force f, the Dirichlet data g
 * and the initial velocity v0 are data of the problem).  The library calls it on the host with
 * npts points x (dim x npts doubles, structure of arrays: x[i * npts + p] is coordinate i of point
 * p) at time t and expects the field in out (dim x npts doubles, same layout; out is zeroed before
 * the call).  user is the pointer given with the callback.  Values must be finite. */
typedef void (*stmg_field_fn)(void* user, int64_t npts, const double* x, double t, double* out);

typedef struct {
  int dim;             /* d in {2, 3} */
  int n_cells_1d;      /* n: the finest mesh has n^d cells */
  int r;               /* pressure degree; velocity Q_{r+1}; 1 <= r <= 3 */
  int k;               /* DG(k) in time, 0 <= k <= 2 */
  double nu;           /* kinematic viscosity (1/Re) */
  double tau;          /* slab length */
  double gamma1, gamma2;   /* Nitsche penalties (Sec. 5: 10, 10) */
  int problem;         /* stmg_problem */
  int bconv;           /* 1: include the boundary convection pairing of Eq. bttp */
  int n_levels_h;      /* number of h-coarsenings; -1: coarsen while n even and n/2 >= 2 */
  int precond_precision; /* stmg_precision of the multigrid preconditioner */
  int nu1, nu2;        /* Vanka pre/post sweeps (Sec. 5.1: 1, 1) */
  double omega;        /* Vanka damping of the velocity DoFs (Eq. vanka0); <= 0 (default):
                          1.2 / 2^d, i.e. 0.3 in 2D, 0.15 in 3D (a vertex lies in 2^d patches) */
  double newton_rtol, newton_atol; int newton_maxit;            /* Sec. 5: 1e-8, 1e-12 */
  double ew_eta0, ew_c, ew_theta, ew_min, ew_max;               /* Alg. 1: 0.4, 0.5, 1.5, 1e-3, 0.8 */
  double ls_lambda0, ls_c, ls_tau, ls_alpha_min; int ls_maxbt, ls_window; /* Alg. 2 */
  int gmres_restart, gmres_maxit;                               /* 30, 50 */
  double rebuild_thetaN, rebuild_thetaL; int rebuild_kappa_abs; /* Alg. 1 rebuild triggers */
  int stag_s; double stag_theta;                                /* FGMRES stagnation window */
  double omega_p;      /* Vanka relaxation of the pressure DoFs (velocity DoFs use omega) */
  int vanka_fp16;      /* 1: store the Vanka patch inverses as FP16 with one FP32 scale per patch
                          (half the smoother's memory traffic; the apply still accumulates in
                          the preconditioner precision).  0 (default): preconditioner precision. */
  int build_chunk_cells; /* the smoother build computes the per-cell element matrices in chunks of
                          whole cell planes of at most this many cells (at least three planes),
                          bounding its scratch memory; <= 0 (default): 262144 */
  int keep_time_degree; /* 0 (default): the paper's coarsening order, p in space and time
                          ((k, r) -> (k/2, r/2), Sec. 4.2).  1: p-coarsen in space only and keep
                          DG(k) on every level (a variant; the coarse levels cost (k+1)/(k/2+1)
                          times more, the V-cycle contracts faster when k >= 2) */
  int smoother;        /* 0 (default): the inexact space-time Vanka of Sec. 4.3 (midpoint-surrogate
                          patch matrices, exact patch inverse).  1: diagonal space-time Vanka, the
                          cheaper smoother the paper's closing section proposes: the patch's velocity
                          block keeps only the (k+1) x (k+1) temporal block of each spatial velocity
                          DoF with itself, the pressure coupling stays whole, and the modified patch
                          is solved exactly through its (k+1) C(r+d,d) pressure Schur complement
                          (storage per cell (k+1)^2 m_v + C(r+d,d) m_v + ((k+1) C(r+d,d))^2 reals,
                          m_v = d (r+2)^d; vanka_fp16 does not apply).  2: exact space-time patches
                          R_K J R_K^T, the convection of each time node at its own velocity (the
                          matrix the surrogate approximates): k+1 element-matrix passes and one
                          (k+1) m_s square Gauss-Jordan per cell; where the patch fits shared memory
                          (2D; 3D Q2/P1 with k <= 1), else STMG_ERR_UNSUPPORTED at the build */
  int nu_tc;           /* > 0: pre- and post-sweeps on the levels whose next coarser level has a
                          lower time degree (the DG(k) levels of the paper's p-coarsening), in place
                          of nu1 / nu2 there; <= 0 (default): nu1 / nu2 on every level.  The temporal
                          modes that DG(k) -> DG(k/2) drops are left to the smoother of those levels */
  int newton_stall_steps;    /* > 0: stop with STMG_ERR_NOT_CONVERGED once ||R||_M after a Newton step
                                exceeds newton_stall_ratio times its value newton_stall_steps steps
                                earlier (a solve that makes no progress releases the GPU early;
                                a serving policy, not part of Alg. 1).  <= 0 (default): off */
  double newton_stall_ratio; /* e.g. 0.9 */
} stmg_params;

/* Fill *p with the paper's defaults (Sec. 5, Alg. 1-2) for a d-dimensional problem. */
void stmg_params_default(stmg_params* p);

/* Create a handle: mesh, mapping, multigrid hierarchy and reference tables.
 *   vertices: HOST array of (n+1)^d * d doubles, vertex-major (x,y[,z] per vertex), vertices
 *             lexicographic with x fastest; NULL = the uniform Cartesian grid.  Boundary
 *             vertices must lie on the boundary of the unit square / cube.
 *   stream:   the cudaStream_t all work of this handle is enqueued on.
 * Returns STMG_ERR_ARG for unsupported sizes, STMG_ERR_OOM if the device memory is short. */
stmg_status stmg_create(const stmg_params* p, const double* vertices, stmg_stream stream,
                        stmg_handle** out);
void stmg_destroy(stmg_handle* h);

/* Device bytes a handle with these parameters needs once its slab solver is set up (mesh
 * hierarchy, level vectors, Vanka patch inverses, transfer and coarse work space, FGMRES basis),
 * computed without allocating: the admission test of the serving loop. */
stmg_status stmg_footprint(const stmg_params* p, uint64_t* bytes);

/* Change viscosity, slab length and analytic data of an existing handle; the mesh hierarchy
 * and all device work space stay resident (serving requests of one shape reuse a handle).
 * The next slab solve rebuilds the smoother. */
stmg_status stmg_set_physics(stmg_handle* h, double nu, double tau, int problem);
const char* stmg_last_error(const stmg_handle* h);

/* Number of levels of the hp hierarchy (level 0 = finest) and the sizes of one level. */
stmg_status stmg_num_levels(const stmg_handle* h, int* n_levels);
stmg_status stmg_level_info(const stmg_handle* h, int level, int* n_cells_1d, int* r, int* k,
                            int64_t* n_v, int64_t* n_p, int64_t* n_st);

/* y = J_n(U) x: matrix-free application of the slab Jacobian (Eq. JacobianLocal0-1) on a level,
 * column-wise in time with dense temporal mixing (Sec. 4.4, "matrix-free application of the
 * slab Jacobian").  U_state, x, y: device vectors of that level's n_st entries in the given
 * precision (the pressure part of U_state is not read).  y may not alias x or U_state. */
stmg_status stmg_apply(stmg_handle* h, int level, int precision, const void* U_state,
                       const void* x, void* y);

/* R = R_n(U; V_prev) of Eq. InAlgNS on the finest level, FP64, slab (t_start, t_start + tau].
 * U: n_st doubles; V_prev: n_v doubles (velocity at the end of the previous slab, or the
 * initial velocity for the first slab); R: n_st doubles. */
stmg_status stmg_residual(stmg_handle* h, double t_start, const double* U, const double* V_prev,
                          double* R);

/* Data of the slab problem given by the caller (Sec. 2, Problem 2.1; Eq. DefFn, DefLn): the body
 * force f (the term F_n of the residual) and the Dirichlet data g of the Nitsche terms (L_n and
 * the boundary convection pairing, Eq. bttp), both host callbacks, either may be NULL (zero field).
 * Switches the handle to problem STMG_USER.  Before each residual of a slab (t_start, t_start +
 * tau] the library evaluates f at the (r+2)^d Gauss points of every finest-level cell and g at the
 * (r+2)^(d-1) Gauss points of every boundary face, at the k+1 Radau times of the slab, and keeps
 * the values on the device (d (k+1) n^d (r+2)^d + 2 d^2 (k+1) n^(d-1) (r+2)^(d-1) doubles,
 * allocated by the first call; the evaluation is repeated only when t_start or tau change).  The
 * callbacks run on the calling host thread inside stmg_residual / stmg_slab_solve; user must stay
 * valid while the handle uses them.  STMG_ERR_NUMERIC from those calls if a callback returns a
 * non-finite value, STMG_ERR_OOM if the tables do not fit. */
stmg_status stmg_set_data(stmg_handle* h, stmg_field_fn f, stmg_field_fn g, void* user);

/* Nodal interpolation of the initial velocity at the velocity nodes of the finest level (the
 * mapped Gauss-Lobatto nodes): V0 receives n_v doubles (device, component-major).  v0 != NULL:
 * the caller's field, evaluated on the host at t = 0 and copied to V0 (the call returns when the
 * copy is complete); v0 == NULL: the problem's own initial velocity (zero for STMG_USER). */
stmg_status stmg_initial_condition(stmg_handle* h, stmg_field_fn v0, void* user, double* V0);

/* Newton initial guess: U (n_st doubles, device) gets V_prev (n_v doubles, device) at every
 * time node and zero pressure. */
stmg_status stmg_initial_guess(stmg_handle* h, const double* V_prev, double* U);

/* y = diag(M^tau (x) M_h, M^tau (x) M_h^p) x on the finest level, FP64: the matrix of the
 * mass-weighted norm of Sec. 4.1.  x, y: n_st doubles (device), y may not alias x. */
stmg_status stmg_mass(stmg_handle* h, const double* x, double* y);

/* Build the hp-STMG preconditioner at the Newton state U (n_st doubles, device, finest level):
 * level states by interpolation, the inexact Vanka patch inverses of every smoothed level
 * (midpoint surrogate, Eq. DefTildeHn / DefVnAst, patches = all DoFs of a cell at all time
 * nodes, Eq. LVS) and the coarsest-level factorisation.  Work space is allocated on the first
 * call and kept by the handle.  STMG_ERR_UNSUPPORTED if a patch does not fit on-chip memory
 * for this (d, r, k); STMG_ERR_NUMERIC on a singular patch. */
stmg_status stmg_smoother_build(stmg_handle* h, const double* U);

/* nsweeps additive Vanka sweeps on a level (Eq. vanka0): d <- d + omega sum_K R_K^T S~_K^{-1}
 * R_K (rhs - J d), with J the level Jacobian at the level state.  rhs, d: that level's n_st
 * entries in the preconditioner precision (float for STMG_FP32, double for STMG_FP64);
 * zero_start = 1 sets d = 0 first.  The level must have a smoother (not the coarsest). */
stmg_status stmg_smoother_sweep(stmg_handle* h, int level, const void* rhs, void* d, int nsweeps,
                                int zero_start);

/* The same sweep as stmg_smoother_sweep, for callers that must not allocate device memory
 * during the call: real-time loops that forbid allocator calls once they run, and applications
 * that reserve all device memory in a fixed pool at start-up and may not grow it later.  The
 * paper has no counterpart; this is a property of the library, not of the method.
 * The residual r - J d of each sweep is kept in a fixed 4 MiB device array that every GPU
 * loading this library holds until the process exits; the level's n_st entries in the
 * preconditioner precision must fit in it (at most 524288 doubles or 1048576 floats), else the
 * call returns STMG_ERR_ARG and does nothing.  Nothing is allocated: the handle's patch inverses
 * and level state come from an earlier stmg_smoother_build.  The first call on a device looks up
 * the array's device address with that device current; make that first call before any stream
 * capture.  The current device must be the one the handle was created on (else STMG_ERR_ARG).
 * The array is shared by all calls and keeps the last call's contents (each sweep overwrites it
 * fully before reading it); calls that overlap on the GPU, e.g. from two streams, race on it and
 * must be serialised by the caller.  Like stmg_smoother_sweep, the call ends by reading the
 * device flag of the bounded waits, so it synchronises the handle's stream before it returns
 * (STMG_ERR_TIMEOUT if a wait ran out).  Arguments and results as in stmg_smoother_sweep. */
stmg_status stmg_smoother_sweep_noalloc(stmg_handle* h, int level, const void* rhs, void* d, int nsweeps,
                                        int zero_start);

/* One V-cycle of the preconditioner on the finest level: z = B^{-1} r (Sec. 4.2; p-coarsening
 * first, then h; nu1 / nu2 sweeps; restriction = transpose of prolongation; direct coarse
 * solve).  r, z: n_st doubles (device); cast to the preconditioner precision internally. */
stmg_status stmg_vcycle(stmg_handle* h, const double* r, double* z);

/* Grid transfer between `level` and `level + 1`, preconditioner precision:
 *   op 0: out(level) = P in(level+1)          (prolongation, Sec. 4.2 canonical embedding)
 *   op 1: out(level+1) = P^T in(level)        (restriction)
 *   op 2: out(level+1) = I in(level)          (velocity state: fine field at coarse nodes and
 *                                              Radau points; only the velocity part is written) */
stmg_status stmg_transfer(stmg_handle* h, int level, int op, const void* in, void* out);

/* Copy the level state of the last smoother build (n_st entries of that level, preconditioner
 * precision) into out. */
stmg_status stmg_level_state(stmg_handle* h, int level, void* out);

typedef struct {
  int newton_its, gmres_its_total, rebuilds, armijo_backtracks;
  double res0, res_final;                       /* ||R||_M at the start and the end */
  double t_rebuild, t_vanka, t_mg_other, t_other; /* seconds; filled when timing is on */
} stmg_stats;

/* Record device time of the four phases of the paper's breakdown (rebuild Vanka, apply Vanka,
 * rest of multigrid, other) during stmg_slab_solve (adds a few event records per phase). */
stmg_status stmg_set_timing(stmg_handle* h, int on);

/* Failure-handling test hook.  With on != 0, every following Vanka sweep of this handle outside
 * a captured V-cycle arms the shared-memory barrier of its patch staging for 16 bytes more than
 * it copies, so that the kernel's bounded wait runs out: the kernel flags the timeout, waits once
 * more (also bounded) and leaves the correction of that cell unchanged; the call returns
 * STMG_ERR_TIMEOUT.  No copy is left in flight and the GPU is not faulted, so the handle stays
 * usable; on = 0 restores normal operation.  Each sweep launch takes up to a few seconds while
 * the hook is on.  Not part of the method (no counterpart in the paper). */
stmg_status stmg_test_wait_timeout(stmg_handle* h, int on);

/* Restrict the per-kernel-class timers of stmg_set_timing to the classes whose bit is set in
 * mask (bit c = class c of stmg_kernel_profile; default: all).  Every timed launch adds two
 * event records (graph nodes inside the captured V-cycle), so timing one class perturbs the
 * solve less than timing all of them; the phase times are recorded either way. */
stmg_status stmg_set_timing_classes(stmg_handle* h, unsigned mask);

/* Device time (ms), launches and algorithmic bytes accumulated per kernel class while timing is
 * on (collected at the end of each stmg_slab_solve).  Classes: 0 FP64 Jacobian apply (outer
 * FGMRES), 1 preconditioner-precision Jacobian apply (level residuals), 2 residual, 3 Vanka
 * patch apply (one launch per colour; bytes = patch inverses + patch vectors), 4 Vanka build
 * (element matrices, patch assembly and inversion), 5 mass apply, 6 Vanka patch apply on the
 * finest level only (a subset of class 3). */
stmg_status stmg_kernel_profile(const stmg_handle* h, int cls, double* ms, long long* launches,
                                double* bytes);
stmg_status stmg_kernel_profile_reset(stmg_handle* h);

/* Number of kernels this library has launched in this process (all handles). */
long long stmg_launch_count(void);

/* Newton-FGMRES solve of one slab (Alg. 1-2): U (n_st doubles, device) is the initial guess on
 * entry and the solution on return; V_prev (n_v doubles, device) is the velocity at t_start.
 * Stops at ||R||_M <= max(newton_atol, newton_rtol ||R_0||_M).  STMG_ERR_NOT_CONVERGED when
 * newton_maxit is reached (U holds the last iterate), STMG_ERR_NUMERIC on NaN / Inf.  stats
 * may be NULL. */
stmg_status stmg_slab_solve(stmg_handle* h, double t_start, const double* V_prev, double* U,
                            stmg_stats* stats);

/* ---- Batched preconditioning across same-shape solves (continuous batching of requests) ----
 * A group holds one hp-STMG hierarchy with `slots` slots for handles of one shape (the same
 * stmg_params except viscosity and problem data, the same vertices).  An attached handle's
 * smoother builds fill its own slot, and each preconditioner application (one per FGMRES
 * iteration) joins the next batched V-cycle of the group: every kernel of the V-cycle chain
 * (level residuals, Vanka sweeps, transfers, coarse solve) is launched once for all ready slots.
 * Batching is the serving pattern of concurrent same-shape requests; the paper has no
 * counterpart (its solver runs one problem at a time).  A round starts as soon as every attached
 * handle that is inside stmg_slab_solve is waiting, or 200 microseconds after the first one
 * arrived.  Each slot computes exactly what a handle without a group computes, so results are
 * bitwise the same alone and in a batch.  Slab solves of attached handles must run on different
 * host threads (they wait for each other); stmg_smoother_sweep / stmg_vcycle / stmg_transfer /
 * stmg_level_state are not available on attached handles (STMG_ERR_ARG).  The group runs on a
 * non-blocking stream that it creates and owns (a stream shared with any other user could be
 * touched by another thread while a V-cycle graph is being captured on it), ordered against the
 * handles' streams by events.  Device memory: the hierarchy of `slots` handles (an attached
 * handle allocates no hierarchy of its own). */
typedef struct stmg_group stmg_group;

/* Create a group for handles shaped like p / vertices (as stmg_create), 1 <= slots <= 16, on the
 * current device.  *out is NULL on any error. */
stmg_status stmg_group_create(const stmg_params* p, const double* vertices, int slots, stmg_group** out);
/* Destroy a group; attached handles are detached first (their next solve allocates their own
 * hierarchy).  No solve of an attached handle may be running. */
void stmg_group_destroy(stmg_group* g);
/* Attach a handle to a free slot; STMG_ERR_ARG if the shape differs or no slot is free.  Attach
 * before the handle's first smoother build or slab solve. */
stmg_status stmg_group_attach(stmg_group* g, stmg_handle* h);
stmg_status stmg_group_detach(stmg_group* g, stmg_handle* h);
/* Counters: batched V-cycle rounds, slot V-cycles served (the V-cycles the handles asked for),
 * kernel launches of the rounds' V-cycles (the per-handle path would launch about
 * launches / rounds * slot_vcycles). */
stmg_status stmg_group_stats(const stmg_group* g, long long* rounds, long long* slot_vcycles,
                             long long* launches);

#ifdef __cplusplus
}
#endif

#endif /* STMG_H */
