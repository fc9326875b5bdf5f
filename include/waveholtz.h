/*
 * waveholtz.h -- C ABI of libwaveholtz: one WaveHoltz iteration (and the solvers that
 * drive it) on an overset grid, on one NVIDIA GB300 (sm_103a).
 *
 * The method (Appelo, Banks, Henshaw, Schwendeman, "An optimal O(N) Helmholtz solver for
 * complex geometry using WaveHoltz and overset grids"):
 *   Solve  c(x)^2 Lap u + omega^2 u = f  in Omega,  B u = 0 on the boundary
 *   (Eq. HelmholtzBVP, Sec. 2.1) by iterating the WaveHoltz map (Algorithm 1, Sec. 2.2)
 *       v <- W_h(v, f) = (2/Tbar) sum_n sigma_n dt (cos(omega_e t^n) - alpha/2) W^n
 *   where W^n solves the explicit scheme D+tD-t W = c^2 L_h W - f cos(omega_e t)
 *   (Eq. WaveSchemeexplicit, Sec. 4.2) with W^0 = v, marched over Np periods by
 *   Algorithm 2 (advance every grid, apply boundary conditions, interpolate; Sec. 3.2),
 *   with the explicit time correction of Recipe OmegaTildeExplicit (App. B.1) and the
 *   adjusted filter parameter alpha_d (Eq. alphad).  The fixed point is the discrete
 *   Helmholtz solution; it is reached by the fixed-point iteration or by GMRES on
 *   (I - S) v = b, A v = v - W_h(v, 0), b = W_h(0, f) (Eqs. WaveHoltzLinearSystem and
 *   MevalII, Sec. 4.3).
 *
 * Conventions (every entry point):
 *   - Every function returns a wh_status; negative values are errors and
 *     wh_last_error(ctx) then holds a one-line message.  No call aborts the process.
 *   - A context owns every device allocation it makes; wh_destroy frees them.  Calls on
 *     one context are not thread-safe.  Work is issued on the context's stream
 *     (wh_set_stream); calls that return host data synchronise that stream.
 *   - Grid arrays passed to wh_add_grid / wh_set_forcing are HOST arrays that the
 *     library copies; the caller keeps ownership.
 *   - "Compact vectors" are the concatenation over grids (in wh_add_grid order) of
 *     n0*n1 values per grid, row-major with axis 0 fastest (index j*n0 + i).  Values at
 *     unused points are ignored on input and written as 0 on output.
 *   - Ghost width is order/2 on non-periodic axes and 0 on periodic axes.  "Extended"
 *     arrays cover indices i in [-g0, n0+g0), j in [-g1, n1+g1), same ordering.
 *   - Boundary data g is zero (homogeneous Dirichlet / Neumann conditions).
 */
#ifndef WAVEHOLTZ_H
#define WAVEHOLTZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wh_ctx wh_ctx;

typedef enum {
  WH_OK = 0,
  WH_ERR_ARG = -1,           /* invalid argument (null pointer, bad size or code) */
  WH_ERR_CUDA = -2,          /* a CUDA runtime call failed */
  WH_ERR_STATE = -3,         /* call out of order (e.g. wh_iterate before wh_prepare) */
  WH_ERR_DIVERGED = -4,      /* residual became NaN/Inf or grew without bound */
  WH_ERR_TIMEOUT = -5,       /* a bounded device-side wait gave up */
  WH_ERR_NOT_CONVERGED = -6, /* solver hit its iteration limit above tolerance */
  WH_ERR_GRID = -7,          /* inconsistent grid description or interpolation data */
  WH_ERR_NOMEM = -8          /* device or host allocation failed */
} wh_status;

/* Point classification (Sec. 3.1).  Dirichlet points are boundary points whose value
 * the boundary condition sets. */
enum { WH_UNUSED = 0, WH_DISC = 1, WH_INTERP = 2, WH_DIRICHLET = 3 };
/* Boundary condition of a side; sides are [axis0-lo, axis0-hi, axis1-lo, axis1-hi]. */
enum { WH_BC_NONE = 0, WH_BC_DIRICHLET = 1, WH_BC_NEUMANN = 2, WH_BC_PERIODIC = 3 };
/* Grid kinds: axis-aligned Cartesian, or curvilinear given by inverse metrics. */
enum { WH_CARTESIAN = 0, WH_CURVILINEAR = 1 };
/* Arithmetic of the wave march.  WH_FP32 keeps the state, forcing and stencil weights in
 * FP32; the filter accumulator, interpolation weights and all reductions stay FP64. */
enum { WH_FP64 = 0, WH_FP32 = 1 };
/* Solvers for wh_solve. */
enum { WH_FPI = 0, WH_GMRES = 1 };
/* How an iteration is launched.  WH_LAUNCH_GRAPH (default): a CUDA graph of per-phase
 * kernels (2M + 1 launches).  WH_LAUNCH_PERSISTENT: one cooperative kernel per WaveHoltz
 * iteration, bounded grid-wide barriers between the march and the ghost-rule +
 * interpolation phase of every time step.  Both compute the same values. */
enum { WH_LAUNCH_PERSISTENT = 0, WH_LAUNCH_GRAPH = 1 };

typedef struct {
  int32_t order;      /* spatial order p: 2 or 4 (Sec. 3.2) */
  int32_t periods;    /* Np >= 1: Tbar = Np * T (Algorithm 1) */
  double cfl;         /* fraction of the explicit stability limit: (0, 1] is stable; values
                         in (1, 2] are accepted only so that the divergence checks of
                         wh_solve can be exercised (the march then grows without bound) */
  int32_t alpha_mode; /* 0: alpha_d of Eq. alphad (default); 1: alpha = 1/2 */
  int32_t precision;  /* WH_FP64 (default) or WH_FP32 */
  int32_t launch_mode;  /* WH_LAUNCH_GRAPH (default) or WH_LAUNCH_PERSISTENT */
  uint64_t barrier_spin_limit;  /* polls before a grid barrier of the persistent kernel
                                   gives up (WH_ERR_TIMEOUT); 0 = default (2^22, ~1 s) */
  uint64_t trajectory_bytes;    /* wh_adjoint keeps the whole forward trajectory (M + 1
                                   states) in device memory when it needs at most this
                                   many bytes, else recomputes it from checkpoints every
                                   16 steps; 0 = default (half the free device memory) */
  int32_t resident_blocks;      /* launch layouts whose blocks wait on one another (the
                                   march with the ghost rules and interpolation folded into
                                   it; the persistent kernel) need all their blocks on the
                                   GPU at once.  0 (default): the occupancy query's figure for
                                   the whole device; > 0: assume at most this many (a GPU
                                   shared with other streams or processes): the folded
                                   layout is then used only when its grid fits, and the
                                   persistent kernel's grid is capped.  Independently, a
                                   folded launch whose bounded wait expires makes the context
                                   stop folding (that call reports WH_ERR_TIMEOUT). */
} wh_options;

/* One component grid (Sec. 3.1).  All pointers are host pointers, read during the call.
 *   n[2]        points per axis, boundary points included, ghosts excluded; a periodic
 *               axis lists each point once.  n >= 2*order + 1 on non-periodic axes.
 *   kind        WH_CARTESIAN: spacing h[] is physical, metrics are the identity.
 *               WH_CURVILINEAR: h[] is the parameter spacing, rx gives the metrics.
 *   bc[4]       per-side WH_BC_*; periodic sides come in pairs.  A Neumann side may only
 *               meet periodic or interpolation sides.
 *   orthogonal  1 if the grid lines are orthogonal (the mixed coefficient a12 is then
 *               identically zero and dropped); grids with a Dirichlet or Neumann side
 *               must be orthogonal.
 *   mask        n0*n1 int8 WH_UNUSED / WH_DISC / WH_INTERP / WH_DIRICHLET.
 *   rx          curvilinear only: 4 extended arrays, dr1/dx, dr1/dy, dr2/dx, dr2/dy.
 *   c2          n0*n1 values of c(x)^2 > 0, or NULL for c = 1. */
typedef struct {
  int32_t n[2];
  int32_t kind;
  int32_t bc[4];
  int32_t orthogonal;
  int32_t instance;  /* independent problem this grid belongs to (batching): 0 for the
                        first grid, then equal to or one more than the previous grid's */
  double h[2];
  const int8_t *mask;
  const double *rx;
  const double *c2;
} wh_grid_desc;

/* Interpolation data (Sec. 3.1): receiver k in grid recv_grid[k] at (recv_i, recv_j)
 * takes sum_{a,b} wx[k][a] wy[k][b] u_donor(i0 + a, j0 + b), a, b = 0..order, from grid
 * donor_grid[k] with lower corner (donor_i0, donor_j0) (wrapping on periodic axes).
 * Every donor must be a WH_DISC or WH_DIRICHLET point (explicit interpolation); every
 * receiver must be a WH_INTERP point; each WH_INTERP point must be listed once.  Host
 * pointers; wx, wy are [n][order+1] FP64. */
typedef struct {
  int64_t n;
  const int32_t *recv_grid, *recv_i, *recv_j;
  const int32_t *donor_grid, *donor_i0, *donor_j0;
  const double *wx, *wy;
} wh_interp_desc;

/* Three-dimensional grids (Sec. 3 in three space dimensions).  A context takes either
 * two-dimensional grids (wh_add_grid / wh_set_interp) or three-dimensional ones
 * (wh_add_grid3 / wh_set_interp3), fixed by the first grid added; 3D contexts hold one
 * instance and take opt.order = 2 on any grid or opt.order = 4 on Cartesian grids only
 * (second difference D+D-(1 - h^2/12 D+D-) per axis, Eq. SecondDerivOrderp; two ghost
 * layers filled per boundary point of a Dirichlet face by the compatibility condition
 * c^2 D_nn W_b = f_b cos(omega_e t) and of a Neumann face by the centred fourth-order
 * D_n W = 0, each with the extrapolation D+^5 W_{-2} = 0; time-step constant sqrt(3)/2).
 * Compact 3D vectors hold n0*n1*n2 values per grid with axis 0 fastest (index
 * (k*n1 + j)*n0 + i); the ghost width is order/2 on non-periodic axes and 0 on periodic
 * ones, and extended arrays cover [-g_a, n_a + g_a) per axis in the same order.  Sides are [axis0-lo, axis0-hi, axis1-lo, axis1-hi, axis2-lo, axis2-hi].
 *   n[3]    points per axis (boundary points included; a periodic axis lists each point
 *           once); n >= 5 on non-periodic axes, >= 3 on periodic ones.
 *   kind    WH_CARTESIAN (h physical) or WH_CURVILINEAR (h the parameter spacing; order 2
 *           only).
 *   bc[6]   per-side WH_BC_*; periodic sides come in pairs.  Discretization points may lie
 *           on a non-periodic side only if it is a Neumann side, and their inward neighbour
 *           must be a discretization or Dirichlet point.
 *   ortho   bit mask of axis pairs whose grid lines are orthogonal: bit 0 (0,1), bit 1
 *           (0,2), bit 2 (1,2).  The mixed term 2 a_kl u_{r_k r_l} of such a pair is dropped
 *           (a_kl = 0).  The normal axis of a Neumann side must be orthogonal to the other
 *           two (the centred rule W_{-1} = W_{+1} is then the normal derivative).  Ignored
 *           on Cartesian grids.
 *   mask    n0*n1*n2 int8 point classes (WH_UNUSED ... WH_DIRICHLET).  A discretization
 *           point's stencil (the 7-point cross and the edge points of non-orthogonal pairs;
 *           at order 4 the 13-point cross) must read no unused point.  At order 4 every
 *           ghost it reads must be filled by a rule (the boundary point of that grid line is
 *           a discretization point of a Neumann face or a Dirichlet point of a Dirichlet
 *           face), the rules' three inward points may not be interpolation points, and a
 *           Neumann face may only meet periodic or interpolation faces.
 *   rx      curvilinear: 9 extended arrays, array 3k+m = dr_k/dx_m.
 *   c2      n0*n1*n2 values of c(x)^2 > 0, or NULL for c = 1.
 * Host pointers, copied during the call.  Errors: WH_ERR_ARG (bad sizes, codes, spacing,
 * orthogonality of a Neumann axis; at order 4 a curvilinear grid or a Neumann face meeting
 * another physical face), WH_ERR_GRID (stencils reading unused points or unfilled ghosts,
 * Neumann inward neighbours), WH_ERR_STATE (a two-dimensional context). */
typedef struct {
  int32_t n[3];
  int32_t kind;
  int32_t bc[6];
  int32_t ortho;
  int32_t instance;  /* must be 0 */
  double h[3];
  const int8_t *mask;
  const double *rx;
  const double *c2;
} wh_grid3_desc;

/* Three-dimensional interpolation data (Sec. 3.1): receiver k of grid recv_grid[k] at
 * (recv_i, recv_j, recv_k) takes sum_{a,b,c} wx[k][a] wy[k][b] wz[k][c]
 * u_donor(i0 + a, j0 + b, k0 + c), a, b, c = 0..p (p the order: stencils of width p + 1),
 * from grid donor_grid[k] with lower corner (donor_i0, donor_j0, donor_k0), wrapping on
 * periodic axes.  Every donor must be a WH_DISC or WH_DIRICHLET point (explicit
 * interpolation), every receiver a WH_INTERP point, and each WH_INTERP point listed exactly
 * once (else WH_ERR_GRID).  Host pointers; wx, wy, wz are [n][p + 1] FP64. */
typedef struct {
  int64_t n;
  const int32_t *recv_grid, *recv_i, *recv_j, *recv_k;
  const int32_t *donor_grid, *donor_i0, *donor_j0, *donor_k0;
  const double *wx, *wy, *wz;
} wh_interp3_desc;

/* Time setup of one frequency (Recipe OmegaTildeExplicit, Eq. alphad). */
typedef struct {
  double omega;      /* requested frequency */
  double dt;         /* (2/omega) sin(pi/Nt) */
  double omega_e;    /* 2 pi / (Nt dt) */
  double alpha;      /* alpha_d or 1/2 */
  double dt_max;     /* cfl * largest stable dt (frozen coefficients) */
  double Tbar;       /* Np * Nt * dt */
  int32_t Nt;        /* time steps per period */
  int32_t M;         /* Np * Nt time steps per WaveHoltz iteration */
  int64_t n_active;  /* discretization + interpolation + Dirichlet points */
  int64_t n_total;   /* length of a compact vector */
} wh_time_info;

typedef struct {
  int32_t iterations;   /* WaveHoltz iterations (FPI) or matrix-vector products (GMRES):
                           products_fp64 + products_fp32 */
  int32_t converged;    /* 1 if the tolerance was met */
  double residual;      /* final relative residual: FPI ||v_k - v_{k-1}|| / ||v_k||,
                           GMRES ||b - A v|| / ||b|| with the FP64 march (Sec. 6.1) */
  double seconds;       /* wall time of the solve */
  int32_t n_history;    /* entries written to history (<= history_cap) */
  int32_t products_fp64;  /* wave solves with the FP64 march */
  int32_t products_fp32;  /* wave solves with the FP32 march */
} wh_stats;

/* Fill *opt with order 4, Np = 1, cfl 0.9, alpha_d, FP64, graph launch. */
wh_status wh_options_default(wh_options *opt);

/* Create a context on the current CUDA device.  *out receives the handle. */
wh_status wh_create(const wh_options *opt, wh_ctx **out);

/* Free every device and host resource of ctx (NULL is a no-op). */
void wh_destroy(wh_ctx *ctx);

/* Message of the last failing call on ctx (never NULL). */
const char *wh_last_error(const wh_ctx *ctx);

/* Issue all further work on this cudaStream_t (NULL = legacy default stream). */
wh_status wh_set_stream(wh_ctx *ctx, void *stream);

/* Add one component grid (Sec. 3.1); *grid_id receives its index (0, 1, ...).
 * Errors: WH_ERR_ARG, WH_ERR_GRID (unsupported boundary combination or bad mask). */
wh_status wh_add_grid(wh_ctx *ctx, const wh_grid_desc *grid, int32_t *grid_id);

/* Set the interpolation data for all receivers (replaces earlier data).  Validated
 * against the masks: WH_ERR_GRID on any violation. */
wh_status wh_set_interp(wh_ctx *ctx, const wh_interp_desc *interp);
/* Add a three-dimensional grid / set three-dimensional interpolation data (see
 * wh_grid3_desc, wh_interp3_desc).  wh_set_forcing, wh_prepare, wh_iterate,
 * wh_iterate_host, wh_solve, wh_dot, wh_eigs, the deflation calls, wh_get_state /
 * wh_set_state, wh_profile_kernels and wh_get_time_info work on 3D contexts unchanged;
 * batches, differentiation, wh_set_coefficient and the launch tuning calls return
 * WH_ERR_STATE there.  One 3D iteration is an input kernel, a CUDA graph of
 * 2M + 1 kernels (level-0 ghost rules and interpolation, then per step the march and the
 * next level's ghost rules and interpolation) and an output kernel. */
wh_status wh_add_grid3(wh_ctx *ctx, const wh_grid3_desc *grid, int32_t *grid_id);
wh_status wh_set_interp3(wh_ctx *ctx, const wh_interp3_desc *interp);

/* Forcing f(x) of grid grid_id (host, n0*n1): the right-hand side of
 * c^2 Lap u + omega^2 u = f; the scheme applies -f cos(omega_e t). */
wh_status wh_set_forcing(wh_ctx *ctx, int32_t grid_id, const double *f);

/* Dirichlet boundary data g of grid grid_id (host, n0*n1 compact values, copied; read at
 * the grid's WH_DIRICHLET points, ignored elsewhere; NULL removes them): the Helmholtz
 * solution takes u = g there (the paper's problem statement with g != 0, which its
 * experiments leave at g = 0).  The wave march holds W = g cos(omega_e t) at those points
 * while the forcing is on (the map W_h(., 0) keeps g = 0, so GMRES and the eigensolver are
 * unchanged); at order 4 the compatibility ghost rule's right side becomes
 * f_b - omega^2 g_b - c^2 (D_tt g)_b with D_tt the fourth-order second difference along
 * the side (centred; wrapped on a periodic side; six-point one-sided at the ends), since
 * the scheme's second time difference of g cos(omega_e t) is exactly -omega^2 g cos.
 * Takes effect at the next wh_prepare.  On three-dimensional contexts (order 2, no
 * Dirichlet ghost rule) the data are set per level by a small kernel before the level's
 * ghost rules and interpolation, and the temporally blocked FP32 march keeps the units
 * near such points in single steps.  Differentiation and wh_set_deflation (Algorithm 3's
 * inflation) then return WH_ERR_STATE, while wh_set_deflation_basis stays exact.
 * Errors: WH_ERR_ARG (bad grid, non-finite data, a three-dimensional context of order 4),
 * WH_ERR_GRID (order 4: a curvilinear grid with a Dirichlet side, or a Dirichlet side of
 * fewer than 6 points). */
wh_status wh_set_boundary_data(wh_ctx *ctx, int32_t grid_id, const double *g);

/* Prepare one frequency per instance (batching: several independent Helmholtz problems,
 * each with its own grids, omega, time step, Nt and alpha, advanced by the same kernel
 * launches; an instance stops after its own M steps).  omegas: host array of one value per
 * instance; infos (host, may be NULL) receives one time setup per instance. */
wh_status wh_prepare_batch(wh_ctx *ctx, const double *omegas, wh_time_info *infos);

/* Prepare frequency omega (every instance): the operator coefficients of the mapping method
 * (a_kl, b_k; Sec. 3.1) and the stability bound on the device, the time setup, the
 * per-point stencil weights, and the per-step tables.  Must follow the last
 * wh_add_grid / wh_set_interp / wh_set_forcing.  *info (may be NULL) receives the
 * time setup. */
wh_status wh_prepare(wh_ctx *ctx, double omega, wh_time_info *info);

/* ONE WaveHoltz iteration v_out = W_h(v_in, f) (forcing = 1) or W_h(v_in, 0)
 * (forcing = 0): the hot path.  v_in, v_out: DEVICE compact vectors of n_total FP64
 * values (may not alias).  Asynchronous on the context stream.  A persistent launch whose
 * grid barrier timed out is reported as WH_ERR_TIMEOUT by a later call on the context
 * (the next synchronising call at the latest); the context stays usable. */
wh_status wh_iterate(wh_ctx *ctx, int32_t forcing, const double *v_in, double *v_out);

/* Same as wh_iterate with HOST vectors: copies v_in to the device, iterates, copies the
 * result back and synchronises. */
wh_status wh_iterate_host(wh_ctx *ctx, int32_t forcing, const double *v_in, double *v_out);

/* Solve to relative tolerance tol with WH_FPI (Algorithm 1) or WH_GMRES (restarted,
 * classical Gram-Schmidt applied twice, Sec. 4.3).  u: DEVICE compact vector, the
 * initial guess on entry and the solution on exit.  history (host, may be NULL)
 * receives up to history_cap relative residuals.  max_it bounds the wave solves.
 * On a WH_FP32 context, WH_GMRES runs in two phases: b uses the FP64 march; GMRES(restart)
 * cycles whose wave solves use the FP32 march take the residual to max(tol, 1e-4) (or
 * until a cycle no longer halves it), then FP64-march cycles continue from that iterate to
 * tol, confirmed by a true FP64 residual.  The orthogonalisation, the updates and all
 * reductions are FP64 throughout.  WH_FPI iterates with the context's march.
 * With a deflation set (wh_set_deflation) both methods solve the deflated problem of
 * Algorithm 3 and, on return (converged or not), add back the Helmholtz solution's
 * components along the set: WH_FPI removes the set's components after every iteration;
 * WH_GMRES (Sec. 4.3 applied to the deflated fixed-point iteration) solves
 * (I - P S) v = P b with P = I - sum_m phi_m phi_m^T, starting from P u.  Residuals are
 * those of the deflated iterates.  Returns WH_ERR_NOT_CONVERGED (u holds the last iterate)
 * when max_it is reached; WH_ERR_DIVERGED on a NaN/Inf residual, on FPI differences
 * ||v_{k+1} - v_k|| growing past 10x their smallest value, or on a GMRES product with
 * ||A q|| > 25 ||q|| (a stable march keeps it near 2): the signs of an unstable march. */
wh_status wh_solve(wh_ctx *ctx, int32_t method, double tol, int32_t max_it, int32_t restart,
                   double *u, wh_stats *stats, double *history, int32_t history_cap);

/* Deflation set of wh_solve (Algorithm 3, Sec. 4.4): k discrete eigenpairs (phi_m,
 * lambda_m^2) of the spatial operator (c^2 L_h phi = -lambda^2 phi with the boundary and
 * interpolation constraints; wh_eigs computes them).  After every WaveHoltz iteration of
 * wh_solve(WH_FPI) the iterate loses its components along the set,
 * v <- v - sum_m (v, phi_m) phi_m (wh_solve(WH_GMRES) solves for the fixed point of that
 * deflated iteration); on return the solution gains
 * u = v + sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m, where (f, phi_m) pairs phi_m
 * with f at discretization points only (the forcing enters the discrete system on those
 * rows).  Inner products are plain sums over the compact vector, so the rows must be
 * orthonormal in it (exact for self-adjoint discretizations; an approximation on overset
 * grids, whose discrete operator is not symmetric).  phi: DEVICE pointer to
 * k compact vectors, row m at phi + m * n_total; the context keeps the pointer (not a copy):
 * the caller owns the memory and keeps it alive and unchanged while the set is in use.
 * lambda2: HOST array of k values, copied.  k = 0 removes the set.  Single-instance
 * contexts (2D or 3D).  Errors: WH_ERR_ARG (k < 0 or > 4000, null pointers,
 * non-finite lambda2; at solve time |omega^2 - lambda_m^2| <= 1e-12 omega^2 for some m,
 * where the inflation would divide by a near-zero difference), WH_ERR_STATE (at solve time
 * a batch). */
wh_status wh_set_deflation(wh_ctx *ctx, int32_t k, const double *phi, const double *lambda2);

/* Checkpoint and resume of a solve.  When wh_solve stops at its max_it wave solves
 * (WH_ERR_NOT_CONVERGED), the context keeps what continuing it needs: the iterate (for
 * GMRES stopped inside a restart cycle: the cycle's starting iterate, the Krylov basis built
 * so far, the Hessenberg matrix, the Givens rotations and the residual vector), the
 * right-hand side b, the product counts and the FP32/FP64 phase.  wh_get_state writes it
 * into the HOST buffer buf (*bytes: its size on entry, the bytes written on return); with
 * buf NULL it only returns the size in *bytes.  wh_set_state loads such a state into a
 * context prepared for the same problem and frequency (checked: sizes, omega, dt, M); the
 * next wh_solve with the same method (and restart) then continues that solve instead of
 * starting one: its u receives the saved iterate (the initial guess is ignored) and max_it
 * keeps counting the products made before the save.  A solve stopped at N products and
 * resumed with max_it = N_total gives bit for bit the result of one uninterrupted solve with
 * max_it = N_total.  The deflation set and tuning must be the same as when the state was
 * saved (not checked).  Another wh_solve on the context discards a state not yet saved.
 * Errors: WH_ERR_STATE (no stopped solve; another problem; an FP32 phase state on an FP64
 * context), WH_ERR_ARG (buffer too small or not a saved state). */
wh_status wh_get_state(wh_ctx *ctx, void *buf, size_t *bytes);
wh_status wh_set_state(wh_ctx *ctx, const void *buf, size_t bytes);

/* Deflation set as an orthonormal basis Q of an S-invariant subspace (S = W_h(., 0)) with
 * its Rayleigh matrix T = Q^T S Q, as wh_eigs returns them.  wh_solve then deflates with
 * P = I - Q Q^T like wh_set_deflation's set and inflates exactly: the Helmholtz solution is
 * U = v + Q c with (I - T) c = Q^T W_h(v, f) (from U = S U + b, Sec. 4.3, projected on Q;
 * one extra FP64 wave solve).  Algorithm 3's inflation with (f, phi_m) / (omega^2 -
 * lambda_m^2) is exact only for self-adjoint discretizations; this one also holds on
 * overset grids, where interpolation makes the discrete operator non-symmetric (on a
 * nearly resonant overset disk: 8e-11 against the direct solve, where the printed formula
 * was off by 42%).  The paper has no counterpart of this form.  Q: DEVICE, k compact
 * vectors (row m at Q + m * n_total), kept by pointer like wh_set_deflation's; T: HOST,
 * k x k row-major, copied.  Errors: WH_ERR_ARG (k outside [1, 4000], null or non-finite
 * input; at solve time I - T singular), WH_ERR_STATE (at solve time a batch).  wh_set_deflation with
 * k = 0 removes either kind of set. */
wh_status wh_set_deflation_basis(wh_ctx *ctx, int32_t k, const double *Q, const double *T);

/* Eigenpairs for the deflation set on the GPU (Sec. 4.4; the paper calls SLEPc's
 * Krylov-Schur method on the spatial pencil and notes that WaveHoltz itself can provide
 * them): a Krylov-Schur-style iteration (Arnoldi with classical Gram-Schmidt twice, thick
 * restarts that keep the Schur-like basis of the wanted Ritz values) on the zero-forcing map
 * S with the FP64 march.  S has the eigenvectors of the constrained spatial operator with
 * eigenvalues beta_d(lambda~) (Theorem FullyDiscreteExplicitWaveHoltzConvergenceRate), so
 * its k eigenvalues of largest modulus are the k modes the fixed-point iteration reduces
 * most slowly.  With passes = 2 a second run on (I - Q1 Q1^T) S (I - Q1 Q1^T) from another
 * start vector finds the copies of repeated eigenvalues that one Krylov sequence misses
 * (symmetric geometries), and the k largest of the union are kept (k more products for the
 * coupling block Q1^T S Q2); it runs only when the first pass converged and a whole basis
 * of products remains, and its result is kept only if it converged too.
 *   k      eigenpairs wanted; m: basis size (0 = max(3k, k + 60), at most 2048);
 *   tol    relative residual ||S y - beta y|| <= tol |beta| of every wanted Ritz pair;
 *   max_products  wave solves allowed (all passes);  seed: start vectors (splitmix64).
 * Outputs: Q (DEVICE, k compact vectors, row i at Q + i * n_total): an orthonormal basis of
 * the invariant subspace of the k eigenvalues, in decreasing |beta| (for a self-adjoint
 * discretization, the eigenvectors themselves); T (HOST k x k row-major, may be NULL):
 * Q^T S Q (for wh_set_deflation_basis); beta (HOST k): the eigenvalues, decreasing modulus;
 * lambda2 (HOST k, may be NULL): lambda^2 = -(y, c^2 L_h y) / (y, y) over discretization
 * points for each eigenvector y (ghost rules applied first; c^2 L_h y from one first step
 * of the march), for wh_set_deflation.  stats (may be NULL): products, converged, the
 * largest relative residual, seconds.  Single-instance contexts (2D or 3D) after
 * wh_prepare.  Allocates its basis ((m + 1) + max(m, 2k) + 3k vectors) for the call.
 * Errors: WH_ERR_ARG, WH_ERR_STATE; WH_ERR_NOT_CONVERGED when the products run out first
 * (the outputs then hold the current approximations). */
wh_status wh_eigs(wh_ctx *ctx, int32_t k, int32_t m, double tol, int32_t max_products,
                  int32_t passes, uint64_t seed, double *Q, double *T, double *beta,
                  double *lambda2, wh_stats *stats);

/* Testing aid for the host side of wh_eigs: eigenvalues w (2m: re, im) and unit
 * eigenvectors V (may be NULL; 2 m^2: element (r, i), i the eigenvalue's index, at
 * V[2 (r m + i)] re, +1 im) of the real m x m row-major matrix A, by Householder reduction
 * to Hessenberg form and the shifted QR algorithm in complex arithmetic.  No device work.
 * WH_ERR_ARG for m outside [1, 4096] or null pointers; WH_ERR_NOT_CONVERGED if the QR
 * algorithm does not converge.  The paper has no counterpart. */
wh_status wh_dense_eig(int32_t m, const double *A, double *w, double *V);
/* Testing aid, the same host routine's invariant subspace: a real orthonormal basis Q
 * (column-major m x p, room for m x (want + 1)) of the invariant subspace of the `want`
 * eigenvalues of largest modulus of A (row-major m x m; a complex pair is kept whole, so
 * *p is want or want + 1), from the complex Schur form reordered by unitary swaps.  No
 * device work.  WH_ERR_ARG on bad sizes or null pointers. */
wh_status wh_dense_invariant(int32_t m, const double *A, int32_t want, double *Q, int32_t *p);

/* Batched solve: one GMRES per instance (restart cycles of the same length), all advancing
 * in lockstep around one batched wave solve per Arnoldi step; an instance that reaches
 * ||b_k - A_k u_k|| <= tol ||b_k|| (checked with the FP64 march) is switched off in the
 * kernels.  FP32 contexts run the two phases of wh_solve per instance (FP32 wave solves to
 * max(tol, 1e-4), then FP64 ones).  u: DEVICE compact vector
 * of all instances (initial guess in, solutions out); stats: host array of one entry per
 * instance (seconds is the whole batch's).  max_it bounds the batched wave solves. */
wh_status wh_solve_batch(wh_ctx *ctx, double tol, int32_t max_it, int32_t restart, double *u,
                         wh_stats *stats);

/* Differentiation (single-instance contexts; FP64 march, also on WH_FP32 contexts).
 * The paper has no adjoint; this is the exact transpose of the implemented discrete map:
 * with C the constraint map (ghost rules and interpolation), D the restriction to
 * discretization points and A the march stencil, W_h(v, 0) = S v = sum_n w_n M X^n with
 * X^0 = C E v, X^1 = C D (A X^0 / 2), X^{n+1} = C D (A X^n - X^{n-1}).
 *
 * wh_apply_adjoint: w_out = S^T w_in (DEVICE compact vectors; <S v, w> = <v, S^T w>).
 *
 * wh_adjoint: for a converged solution u of (I - S) u = b(f) and the gradient g = dJ/du of
 * a scalar misfit J(u) (DEVICE compact vectors), solves (I - S)^T lam = g by GMRES(restart)
 * to relative residual tol (lam: DEVICE compact, output), then returns
 *   grad_c2 = dJ/d(c^2) and grad_f = dJ/df  (DEVICE compact, one value per grid point)
 * from one reverse sweep over the forward states (the march from u with forcing): all of
 * them kept in device memory (see wh_options.trajectory_bytes; the buffer stays with the
 * context), else recomputed from checkpoints every 16 time steps.  The time step is held fixed (it changes only when
 * Nt does); the fixed point is the discrete Helmholtz solution at omega whatever the time
 * step (Sec. 2, the omega-tilde recipe), so these are also the gradients of that solution.
 * Errors: WH_ERR_NOT_CONVERGED when max_it products end above tol (lam then holds the last
 * iterate and grad_c2, grad_f the gradients for it); WH_ERR_STATE before wh_prepare;
 * WH_ERR_ARG on a context with several instances.  Synchronises. */
wh_status wh_apply_adjoint(wh_ctx *ctx, const double *w_in, double *w_out);
wh_status wh_adjoint(wh_ctx *ctx, const double *u, const double *g, double tol, int32_t max_it,
                     int32_t restart, double *lam, double *grad_c2, double *grad_f,
                     wh_stats *stats);

/* Replace c(x)^2 of grid grid_id (host, n0*n1, > 0; NULL: c = 1).  Takes effect at the next
 * wh_prepare. */
wh_status wh_set_coefficient(wh_ctx *ctx, int32_t grid_id, const double *c2);

/* How an iteration is laid out in launches (none of it changes the results beyond rounding
 * order; every configuration is tested against the oracle).  -1 in a field: the library's
 * own choice, which depends on the problem (see each field).
 *   launch_mode   WH_LAUNCH_GRAPH or WH_LAUNCH_PERSISTENT.
 *   fold_gather   graph path: 1 = each march launch (plain or TMA-staged) also does the
 *                 next level's ghost rules and interpolation (library: for the plain march
 *                 when their work units are at most half the march blocks); 0 = a separate
 *                 kernel after each march launch.
 *   tile_tickets  graph path without folding: 1 = march tiles by atomic ticket (library),
 *                 0 = by fixed grid stride.
 *   tma           FP32 march sets: 1 = TMA-staged march for constant-weight grids (library,
 *                 when such grids exist), 0 = the plain march kernel.
 *   pdl           graph path: 1 = the graph's kernels use programmatic dependent launch
 *                 (library), 0 = plain stream order.
 *   temporal_depth  three-dimensional FP32 march: time steps per launch of the temporally
 *                 blocked march, 1..4 (1 = one step per launch); library: 4.  Blocks of
 *                 kTX x 16 x unit_depth points whose box widened by depth - 1 points holds no
 *                 receiver and no Neumann ghost advance that many steps per launch from
 *                 shared memory and registers (recomputing a halo of depth points); the
 *                 rest (the overset coupling region) advances one step at a time with the
 *                 ghost rules and interpolation after each.  Results are bit-identical to
 *                 depth 1.  Ignored by the FP64 march, by fourth-order three-dimensional
 *                 contexts (no point is blocked: blocked_points stays 0) and by
 *                 two-dimensional contexts (-1 or 1 there).
 *   unit_depth    planes along axis 2 of a blocked unit: a multiple of 8 in [8, 256];
 *                 library: 64.
 *   ms_per_iteration, candidates: filled by wh_autotune; blocked_points (points that
 *                 advance temporal_depth steps per launch): filled by wh_autotune and
 *                 wh_get_tuning. */
typedef struct {
  int32_t launch_mode;
  int32_t fold_gather;
  int32_t tile_tickets;
  int32_t tma;
  int32_t pdl;
  double ms_per_iteration;
  int32_t candidates;
  int32_t temporal_depth;
  int32_t unit_depth;
  int64_t blocked_points;
} wh_tuning;

/* Fix the launch layout (fields of -1 leave the library's choice; launch_mode -1 keeps the
 * current mode).  Takes effect at the next iteration.  On three-dimensional contexts only
 * temporal_depth and unit_depth apply and the other layout fields must be -1. */
wh_status wh_set_tuning(wh_ctx *ctx, const wh_tuning *tuning);

/* The launch layout in use, resolved to the values the library applies (after wh_prepare;
 * ms_per_iteration and candidates are 0). */
wh_status wh_get_tuning(const wh_ctx *ctx, wh_tuning *out);

/* Autotuner: after wh_prepare, times `reps` forced WaveHoltz iterations (after one untimed)
 * of every valid launch layout on the prepared problem — persistent; graph with the gather
 * folded; graph with a separate gather and tiles by ticket or by stride; for FP32 contexts
 * also with and without the TMA-staged march; each graph layout with and without
 * programmatic dependent launch; on three-dimensional FP32 contexts the temporal depth
 * 1..4 with unit depths 32, 64 and 128 — keeps the fastest, and reports it (resolved
 * to 0/1 values) with its time and the number of layouts timed in *out (host, may be NULL).
 * Uses the context's working vectors only.  Synchronises. */
wh_status wh_autotune(wh_ctx *ctx, int32_t reps, wh_tuning *out);

/* FP64 inner product <x, y> over n entries of two DEVICE vectors (the GMRES reduction:
 * warp-shuffle partial sums, then one deterministic pass).  *out is a host scalar.  n = 0
 * gives 0 (x, y may then be NULL). */
wh_status wh_dot(wh_ctx *ctx, const double *x, const double *y, int64_t n, double *out);

/* Measurement aid: the device time of each kernel of the iteration, from graph-captured
 * bursts of `reps` back-to-back launches (warm L2, no host gaps) on the prepared problem.
 * ms[4] and counts[4] (host) receive the average milliseconds per launch and the launches
 * per iteration of: [0] the march kernel (with the next level's ghost rules and
 * interpolation when the iteration folds them into its launches), [1] the separate
 * ghost-rule + interpolation kernel, [2] the input kernel, [3] the output kernel.  The bursts run on the context's internal
 * working buffers and leave them unspecified (every wh_iterate rebuilds them from its
 * input).  On three-dimensional contexts [0] is the single-step march, [1] the ghost-rule +
 * interpolation kernel and [2] the temporally blocked march (0 launches when blocking is
 * off), each launch timed on its own with events over `reps` iterations, and [3] is 0.
 * Synchronises. */
wh_status wh_profile_kernels(wh_ctx *ctx, int32_t reps, double *ms, int32_t *counts);

/* Allocation-free inner products.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc -- code whose device memory belongs to another allocator with a
 * fixed budget, and latency-critical loops where cudaMalloc/cudaFree (which synchronise
 * the device) are not acceptable.
 *   out[k] = <X_k, y>, k = 0..nv-1, X_k = X + k*ldx, each vector n FP64 values; X, y and
 *   out (nv doubles) are DEVICE pointers owned by the caller; stream is a cudaStream_t
 *   (NULL = legacy default stream).  Asynchronous on that stream; needs no context.
 * It allocates nothing: the per-block partial sums live in a fixed file-scope device
 * array of WH_NOALLOC_MAX_VECTORS x WH_NOALLOC_BLOCKS doubles (256 KiB) that every GPU
 * loading the library holds until the process exits.  The first call on a device looks up
 * that array's device address; make it before any stream capture on that device.  All
 * calls on a device share the array (it keeps the last call's contents; each call writes
 * every entry it reads), so calls that overlap on the GPU race and must be serialised.
 * The looked-up address is kept for the life of the process: it does not survive
 * cudaDeviceReset on that device (the array is then reloaded at another address), so do
 * not call this function again on a device after resetting it.
 * Returns WH_ERR_ARG, without touching the device, if nv is outside
 * [1, WH_NOALLOC_MAX_VECTORS], n < 0, ldx < n (nv > 1) or a needed pointer is NULL;
 * WH_ERR_CUDA if a CUDA call fails. */
#define WH_NOALLOC_MAX_VECTORS 64
#define WH_NOALLOC_BLOCKS 512
wh_status wh_multidot_noalloc(const double *X, int64_t ldx, int32_t nv, const double *y,
                              int64_t n, double *out, void *stream);

/* Testing aid: out[i] = x[i] widened from FP32 to FP64 by the integer routine the FP32 march
 * uses for its FP64 filter (every normal number and signed zero assembled from its bits by
 * IEEE 754's binary32 -> binary64 rule; subnormals, infinities and NaNs by the hardware
 * conversion), so that it can be checked bit for bit against the hardware conversion.
 * x, out: DEVICE arrays of n values owned by the caller; stream a cudaStream_t (NULL =
 * legacy default stream); asynchronous.  The paper has no counterpart.  WH_ERR_ARG on
 * n < 0 or null pointers with n > 0. */
wh_status wh_widen_f32(const float *x, double *out, int64_t n, void *stream);

/* Measurement aid: the FP64 FMA throughput of the current device (the ALU roofline of the
 * FP64 march), from a kernel of independent dependent FMA chains and nothing else, timed
 * with CUDA events; *tflops receives the best of `reps` launches in TFLOP/s (an FMA counts
 * as 2 FLOP) and *ms (may be NULL) that launch's milliseconds.  Allocates and frees its own
 * small output buffer and stream; synchronises.  The paper has no counterpart. */
wh_status wh_probe_fp64(int32_t reps, double *tflops, double *ms);

/* Time setup of the last wh_prepare. */
wh_status wh_get_time_info(const wh_ctx *ctx, wh_time_info *info);

/* Number of kernel launches issued by the last wh_iterate / wh_solve call. */
int64_t wh_last_launch_count(const wh_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* WAVEHOLTZ_H */
