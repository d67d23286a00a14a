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
  STMG_ERR_NOT_CONVERGED = 4, /* Newton reached its iteration cap */
  STMG_ERR_NUMERIC = 5,       /* NaN / Inf detected */
  STMG_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
  STMG_ERR_UNSUPPORTED = 7    /* configuration not compiled in */
} stmg_status;

typedef enum { STMG_FP64 = 0, STMG_FP32 = 1 } stmg_precision;

/* Analytic data sets of the bundled workloads (f, g, v0). */
typedef enum { STMG_TG2D = 0, STMG_MMS2D = 1, STMG_TG3D = 2, STMG_MMS3D = 3 } stmg_problem;

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
  double omega;        /* Vanka damping (Eq. vanka0) */
  double newton_rtol, newton_atol; int newton_maxit;            /* Sec. 5: 1e-8, 1e-12 */
  double ew_eta0, ew_c, ew_theta, ew_min, ew_max;               /* Alg. 1: 0.4, 0.5, 1.5, 1e-3, 0.8 */
  double ls_lambda0, ls_c, ls_tau, ls_alpha_min; int ls_maxbt, ls_window; /* Alg. 2 */
  int gmres_restart, gmres_maxit;                               /* 30, 50 */
  double rebuild_thetaN, rebuild_thetaL; int rebuild_kappa_abs; /* Alg. 1 rebuild triggers */
  int stag_s; double stag_theta;                                /* FGMRES stagnation window */
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

/* Nodal interpolation of the problem's initial velocity v0 at the velocity nodes (finest
 * level): V0 receives n_v doubles (device). */
stmg_status stmg_initial_condition(stmg_handle* h, double* V0);

#ifdef __cplusplus
}
#endif

#endif /* STMG_H */
