/*
 * waveholtz_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of one WaveHoltz iteration on
 * an overset grid, written from the paper (Appelo, Banks, Henshaw, Schwendeman,
 * "An optimal O(N) Helmholtz solver for complex geometry using WaveHoltz and overset
 * grids").  Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (each step cites the passage it follows):
 *   - time-step setup: the explicit CFL bound (Eq. dtForCartesian, Sec. 3.2, with frozen
 *     coefficients on curvilinear grids) and the explicit time correction
 *     (Recipe OmegaTildeExplicit: dt = (2/omega) sin(pi/Nt), omega_e = 2 pi/(Nt dt));
 *     the adjusted filter parameter alpha_d = tan(omega_e dt/2)/tan(omega_e dt)
 *     (Eq. alphad, Sec. 4.2);
 *   - the mapped Laplacian (Sec. 3.1, mapping method): coefficients
 *     a_kl = sum_m dr_k/dx_m dr_l/dx_m and b_k = sum_m sum_l dr_l/dx_m d/dr_l(dr_k/dx_m),
 *     the latter by finite differences of the metrics; second differences
 *     D+D- sum_mu b_mu (-h^2 D+D-)^mu truncated at mu < p/2 with b_mu = 2 (mu!)^2/(2mu+2)!
 *     (Theorem uxxCoeff and Eq. SecondDerivOrderp, Sec. 5 and App. C);
 *   - the explicit scheme D+tD-t W = c^2 L_h W - f cos(omega_e t) with the first step
 *     W^1 = W^0 + dt^2/2 (c^2 L_h W^0 - f) (Eq. WaveSchemeexplicit, Sec. 4.2);
 *   - Algorithm 2 ordering per step: advance every grid, apply boundary conditions,
 *     then interpolate (Sec. 3.2);
 *   - tensor-product Lagrange interpolation from donor stencils (Sec. 3.1);
 *   - the trapezoid-rule time filter (Eq. updateDiscreteExplicit, Sec. 4.2) with
 *     T-bar = Np Nt dt, weights sigma_0 = sigma_M = 1/2.
 * Readings where the paper is silent (ghost-point rules, fourth-order first and mixed
 * derivatives, frozen-coefficient CFL on curvilinear grids) are listed in the design
 * notes and restated at each function below.
 *
 * Boundary data: Dirichlet sides carry W_b = g_b cos(omega_e t) with g given per boundary
 * point (or_set_boundary; 0 when not given), switched off with the forcing (the map
 * W_h(., 0) has g = 0).  The Helmholtz solution then takes the value g on those sides.
 * Neumann sides likewise take dW/dn = gn_b cos(omega_e t) (or_set_neumann; outward normal),
 * so that the solution's normal derivative is gn there.
 *
 * Ghost-point rules (the paper defers them to its reference on high-order overset wave
 * solvers):
 *   order 2, Dirichlet: W_b = g_b cos(omega_e t); ghosts are never read and stay 0.
 *   order 2, Neumann:   centred normal derivative D0 W = 0  =>  W_{-1} = W_{+1}.
 *   order 4, Dirichlet: W_b = g_b cos(omega_e t); ghosts G1, G2 from the compatibility
 *     condition (the scheme at the boundary point, where D+tD-t of g cos(omega_e t) is
 *     -omega^2 g cos(omega_e t) exactly by the time-step recipe)
 *       c^2 (a_nn D_nn W + b_n D_n W)_b = (f_b - omega^2 g_b - c^2 D_tt g_b) cos(omega_e t)
 *     with D_tt the fourth-order second difference of g along the side (centred, wrapped
 *     on a periodic side, one-sided with six points at the two ends: exact for quintics),
 *     Cartesian grids only when g is given, and the extrapolation D+^5 W_{-2} = 0.
 *   order 4, Neumann: fourth-order centred normal derivative D_n W = 0 and the same
 *     extrapolation.
 * Non-orthogonal grids with physical sides (order 2 only): a Dirichlet side reads no
 * ghost; a Neumann side's rule is the normal derivative with its tangential term (see
 * apply_bc), along a periodic side.
 * The boundary grid lines must otherwise be orthogonal to the boundary, and a Neumann side may
 * only meet periodic or interpolation sides (both checked).
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { OR_UNUSED = 0, OR_DISC = 1, OR_INTERP = 2, OR_DIRICHLET = 3 };
enum { OR_BC_NONE = 0, OR_BC_DIRICHLET = 1, OR_BC_NEUMANN = 2, OR_BC_PERIODIC = 3 };
enum { OR_CARTESIAN = 0, OR_CURVILINEAR = 1 };
#define OR_MAX_GRIDS 64

typedef struct {
  int n[2];      /* points per axis */
  int g[2];      /* ghost width per axis (0 on a periodic axis) */
  int e[2];      /* extended extent n + 2g */
  int kind, orthogonal, bc[4];
  double h[2];   /* Cartesian: physical spacing; curvilinear: parameter spacing */
  signed char *mask; /* extended; ghosts and unused are OR_UNUSED */
  double *rx;    /* curvilinear: 4 extended arrays dr1/dx, dr1/dy, dr2/dx, dr2/dy */
  double *c2;    /* extended; c(x)^2 */
  double *f;     /* extended */
  double *gb;    /* extended; Dirichlet boundary data g (used at Dirichlet points) */
  int has_g;
  double *gn;    /* extended; Neumann data dU/dn (outward normal) at Neumann boundary points */
  double *coef;  /* curvilinear: 5 extended arrays c^2 a11, c^2 a12, c^2 a22, c^2 b1, c^2 b2 */
  long offset;   /* offset of this grid in the concatenated compact vector */
} or_grid;

typedef struct {
  int order, ngrids;
  or_grid G[OR_MAX_GRIDS];
  long nrecv;
  int *rg, *ri, *rj, *dg, *di, *dj;
  double *wx, *wy;
  /* time setup */
  double omega, dt, omega_e, alpha, cfl;
  int Nt, Np, M, prepared;
  double nu;     /* dissipation of the deviation from the periodic motion (0: none) */
  char err[256];
} or_problem;

/* ---------------------------------------------------------------- helpers */

static long at(const or_grid *G, int i, int j) {
  if (G->bc[0] == OR_BC_PERIODIC) i = ((i % G->n[0]) + G->n[0]) % G->n[0];
  if (G->bc[2] == OR_BC_PERIODIC) j = ((j % G->n[1]) + G->n[1]) % G->n[1];
  if (i < -G->g[0] || i >= G->n[0] + G->g[0] || j < -G->g[1] || j >= G->n[1] + G->g[1]) {
    fprintf(stderr, "oracle: index (%d,%d) outside grid\n", i, j);
    abort();
  }
  return (long)(j + G->g[1]) * G->e[0] + (i + G->g[0]);
}

static long ext_size(const or_grid *G) { return (long)G->e[0] * G->e[1]; }

/* b_mu = 2 (mu!)^2 / (2 mu + 2)!  (Theorem uxxCoeff, Eq. uxxCoeff) */
static double b_mu(int mu) {
  double num = 1.0, den = 1.0;
  for (int k = 1; k <= mu; ++k) num *= k;
  num = 2.0 * num * num;
  for (int k = 1; k <= 2 * mu + 2; ++k) den *= k;
  return num / den;
}

/* Value of W at offset k along axis a from (i, j). */
static double nb(const or_grid *G, const double *W, int i, int j, int a, int k) {
  return a == 0 ? W[at(G, i + k, j)] : W[at(G, i, j + k)];
}

/* (D+D-)^q W at (i, j) along axis a, times h^(2q) (undivided), by recursion. */
static double dpdm_pow(const or_grid *G, const double *W, int i, int j, int a, int q) {
  if (q == 0) return W[at(G, i, j)];
  int di = a == 0, dj = a == 1;
  return dpdm_pow(G, W, i + di, j + dj, a, q - 1) - 2.0 * dpdm_pow(G, W, i, j, a, q - 1) +
         dpdm_pow(G, W, i - di, j - dj, a, q - 1);
}

/* Second derivative along axis a: D+D- sum_{mu=0}^{p/2-1} b_mu (-h^2 D+D-)^mu W
 * (Eq. SecondDerivOrderp truncated at mu = p/2 - 1, as in App. C's order-p form). */
static double d2(const or_grid *G, const double *W, int i, int j, int a, int order) {
  double h = G->h[a], s = 0.0;
  for (int mu = 0; mu < order / 2; ++mu) {
    double sign = (mu % 2) ? -1.0 : 1.0;
    s += b_mu(mu) * sign * dpdm_pow(G, W, i, j, a, mu + 1);
  }
  return s / (h * h);
}

/* First derivative along axis a: D0 (order 2) or D0 (1 - h^2/6 D+D-) (order 4). */
static double d1(const or_grid *G, const double *W, int i, int j, int a, int order) {
  double h = G->h[a];
  double d0 = (nb(G, W, i, j, a, 1) - nb(G, W, i, j, a, -1)) / (2.0 * h);
  if (order == 2) return d0;
  /* D0 D+D- W = (W_{+2} - 2 W_{+1} + 2 W_{-1} - W_{-2}) / (2 h^3) */
  double d0dpdm = (nb(G, W, i, j, a, 2) - 2.0 * nb(G, W, i, j, a, 1) +
                   2.0 * nb(G, W, i, j, a, -1) - nb(G, W, i, j, a, -2)) / (2.0 * h * h * h);
  return d0 - h * h / 6.0 * d0dpdm;
}

/* Mixed derivative d^2/dr1 dr2: D0r1 D0r2 (order 2) or the product of the fourth-order
 * first-derivative operators (order 4). */
static double d12(const or_grid *G, const double *W, int i, int j, int order) {
  int r = order / 2;
  double w1[5]; /* D_r2 W at columns i-r..i+r */
  for (int k = -r; k <= r; ++k) w1[k + r] = d1(G, W, i + k, j, 1, order);
  double h = G->h[0];
  if (order == 2) return (w1[2] - w1[0]) / (2.0 * h);
  return (8.0 * (w1[3] - w1[1]) - (w1[4] - w1[0])) / (12.0 * h);
}

/* c^2 L_h W at (i, j) (Sec. 3.1, mapping method; Cartesian grids: c^2 sum D_xx). */
static double lap(const or_problem *P, const or_grid *G, const double *W, int i, int j) {
  long k = at(G, i, j);
  if (G->kind == OR_CARTESIAN)
    return G->c2[k] * (d2(G, W, i, j, 0, P->order) + d2(G, W, i, j, 1, P->order));
  long E = ext_size(G);
  const double *c = G->coef;
  double L = c[k] * d2(G, W, i, j, 0, P->order) + c[2 * E + k] * d2(G, W, i, j, 1, P->order) +
             c[3 * E + k] * d1(G, W, i, j, 0, P->order) +
             c[4 * E + k] * d1(G, W, i, j, 1, P->order);
  if (!G->orthogonal) L += 2.0 * c[E + k] * d12(G, W, i, j, P->order);
  return L;
}

/* ----------------------------------------------------- operator precompute */

/* a_kl and b_k at every point where the stencil of a discretization or Dirichlet
 * point needs them (c^2 folded in).  b_k = sum_m sum_l rx_lm D_l(rx_km). */
static void precompute_coeffs(or_problem *P, or_grid *G) {
  long E = ext_size(G);
  free(G->coef);
  G->coef = (double *)calloc(5 * E, sizeof(double));
  const double *rx = G->rx; /* rx[(2k + m) * E + idx] = dr_k / dx_m */
  for (int j = 0; j < G->n[1]; ++j)
    for (int i = 0; i < G->n[0]; ++i) {
      long q = at(G, i, j);
      signed char m = G->mask[q];
      if (m != OR_DISC && m != OR_DIRICHLET) continue;
      double a[2][2], b[2];
      for (int k = 0; k < 2; ++k)
        for (int l = 0; l < 2; ++l)
          a[k][l] = rx[(2 * k + 0) * E + q] * rx[(2 * l + 0) * E + q] +
                    rx[(2 * k + 1) * E + q] * rx[(2 * l + 1) * E + q];
      for (int k = 0; k < 2; ++k) {
        b[k] = 0.0;
        for (int mm = 0; mm < 2; ++mm)
          for (int l = 0; l < 2; ++l)
            b[k] += rx[(2 * l + mm) * E + q] * d1(G, rx + (2 * k + mm) * E, i, j, l, P->order);
      }
      double c2 = G->c2[q];
      G->coef[q] = c2 * a[0][0];
      G->coef[E + q] = c2 * a[0][1];
      G->coef[2 * E + q] = c2 * a[1][1];
      G->coef[3 * E + q] = c2 * b[0];
      G->coef[4 * E + q] = c2 * b[1];
    }
}

/* ------------------------------------------------------- time-step setup */

/* Largest stable dt of the explicit scheme, frozen coefficients:
 * c dt sqrt(sum_k a_kk / dr_k^2 + 2|a_12|/(dr_1 dr_2)) < C_{2,p}, with C_{2,2} = 1,
 * C_{2,4} = sqrt(3)/2 (Eq. dtForCartesian, Sec. 3.2, read as a bound on c dt, not its
 * square). */
static double dt_bound(const or_problem *P) {
  double Cp = P->order == 2 ? 1.0 : sqrt(3.0) / 2.0;
  double smax = 0.0;
  for (int g = 0; g < P->ngrids; ++g) {
    const or_grid *G = &P->G[g];
    long E = ext_size(G);
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long q = at(G, i, j);
        if (G->mask[q] != OR_DISC) continue;
        double s;
        if (G->kind == OR_CARTESIAN)
          s = G->c2[q] * (1.0 / (G->h[0] * G->h[0]) + 1.0 / (G->h[1] * G->h[1]));
        else {
          s = G->coef[q] / (G->h[0] * G->h[0]) + G->coef[2 * E + q] / (G->h[1] * G->h[1]);
          if (!G->orthogonal) s += 2.0 * fabs(G->coef[E + q]) / (G->h[0] * G->h[1]);
        }
        if (s > smax) smax = s;
      }
  }
  return Cp / sqrt(smax);
}

/* ------------------------------------------------------ boundary conditions */

/* Point (i,j) stepped k units inward from side s (k < 0: into the ghost region). */
static void side_point(const or_grid *G, int s, int t, int k, int *i, int *j) {
  int a = s / 2, hi = s % 2;
  int nrm = hi ? (G->n[a] - 1 - k) : k;
  if (a == 0) { *i = nrm; *j = t; } else { *i = t; *j = nrm; }
}

/* Fourth-order second difference of the boundary data along side s at tangential index t
 * (undivided by h^2 * 12): centred where the five points exist (wrapping on a periodic
 * side), else the six-point one-sided formulas exact for polynomials of degree 5. */
static double side_d2_g(const or_grid *G, int s, int t) {
  int ta = 1 - s / 2, n = G->n[ta];
  int periodic = G->bc[2 * ta] == OR_BC_PERIODIC;
  double v[6];
  if (periodic || (t >= 2 && t <= n - 3)) {
    static const double c[5] = {-1.0, 16.0, -30.0, 16.0, -1.0};
    double acc = 0.0;
    for (int k = -2; k <= 2; ++k) {
      int i, j;
      side_point(G, s, t + k, 0, &i, &j);
      acc += c[k + 2] * G->gb[at(G, i, j)];
    }
    return acc;
  }
  static const double e0[6] = {45.0, -154.0, 214.0, -156.0, 61.0, -10.0};
  static const double e1[6] = {10.0, -15.0, -4.0, 14.0, -6.0, 1.0};
  const int lo = t < 2;
  for (int k = 0; k < 6; ++k) {
    int i, j;
    side_point(G, s, lo ? k : n - 1 - k, 0, &i, &j);
    v[k] = G->gb[at(G, i, j)];
  }
  const double *c = (lo ? t : n - 1 - t) == 0 ? e0 : e1;
  double acc = 0.0;
  for (int k = 0; k < 6; ++k) acc += c[k] * v[k];
  return acc;
}

/* Fill the ghost points of every physical side at time t; fcos = cos(omega_e t) when the
 * forcing is on and 0 when it is off (the compatibility condition carries f and g). */
static void apply_bc(const or_problem *P, int gidx, double *W, double fcos) {
  const or_grid *G = &P->G[gidx];
  long E = ext_size(G);
  for (int s = 0; s < 4; ++s) {
    int a = s / 2, code = G->bc[s];
    if (code != OR_BC_DIRICHLET && code != OR_BC_NEUMANN) continue;
    int ta = 1 - a;
    for (int t = 0; t < G->n[ta]; ++t) {
      int i, j;
      side_point(G, s, t, 0, &i, &j);
      long qb = at(G, i, j);
      signed char m = G->mask[qb];
      double U[4];
      long gq[2];
      for (int k = 0; k < 4; ++k) {
        int ii, jj;
        side_point(G, s, t, k, &ii, &jj);
        U[k] = W[at(G, ii, jj)];
      }
      for (int k = 1; k <= P->order / 2; ++k) {
        int ii, jj;
        side_point(G, s, t, -k, &ii, &jj);
        gq[k - 1] = at(G, ii, jj);
      }
      if (code == OR_BC_NEUMANN) {
        if (m != OR_DISC) continue;
        /* Neumann data: dW/dn = gn cos(omega_e t) along the outward unit normal
         * -+ grad r_a / |grad r_a|; with |grad r_a| = sqrt(a_aa) (c^2 taken out) the
         * normal-axis difference gains 2 h gn fcos / sqrt(a_aa) (order 2) or
         * -12 h gn fcos / sqrt(a_aa) on the undivided fourth-order row, on either side */
        double gnq = 0.0;
        if (G->gn[qb] != 0.0) {
          const double aa = G->kind == OR_CARTESIAN ? 1.0
                            : G->coef[(a == 0 ? 0 : 2) * E + qb] / G->c2[qb];
          gnq = G->gn[qb] * fcos / sqrt(aa);
        }
        if (P->order == 2) {
          /* D0 W = 0 along the normal axis a; on a non-orthogonal grid the normal
           * derivative grad r_a . grad W = a_aa W_{r_a} + a_at W_{r_t} (a_kl =
           * grad r_k . grad r_l) keeps its tangential term, D0 along the (periodic) side:
           * G1 = U1 +- 2 h_a (a_at / a_aa) D0_t W_b (+ on a low side, - on a high one) */
          double corr = 0.0;
          if (!G->orthogonal) {
            int ip, jp, im, jm;
            side_point(G, s, t + 1, 0, &ip, &jp);
            side_point(G, s, t - 1, 0, &im, &jm);
            const double ann = G->coef[(a == 0 ? 0 : 2) * E + qb], ant = G->coef[E + qb];
            const double T = (W[at(G, ip, jp)] - W[at(G, im, jm)]) / (2.0 * G->h[ta]);
            corr = ((s % 2) ? -2.0 : 2.0) * G->h[a] * ant / ann * T;
          }
          W[gq[0]] = U[1] + corr + 2.0 * G->h[a] * gnq;
        } else {
          /* Solve  8(U1 - G1) - (U2 - G2) = 0  and  G2 - 5G1 + 10U0 - 10U1 + 5U2 - U3 = 0. */
          double A[2][2] = {{-8.0, 1.0}, {-5.0, 1.0}};
          double r[2] = {-(8.0 * U[1] - U[2]) - 12.0 * G->h[a] * gnq,
                         -(10.0 * U[0] - 10.0 * U[1] + 5.0 * U[2] - U[3])};
          double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
          W[gq[0]] = (r[0] * A[1][1] - A[0][1] * r[1]) / det;
          W[gq[1]] = (A[0][0] * r[1] - r[0] * A[1][0]) / det;
        }
      } else { /* Dirichlet */
        if (m != OR_DIRICHLET || P->order == 2) continue;
        /* c^2 (a_nn D_nn W + b_n D_n W)_b = f_b cos t, with D_n taken along +r_n.
         * Inward index k runs against +r_n on a high side: sgn = -1 there. */
        double h = G->h[a], ann, bn;
        if (G->kind == OR_CARTESIAN) { ann = G->c2[qb]; bn = 0.0; }
        else { ann = G->coef[(a == 0 ? 0 : 2) * E + qb]; bn = G->coef[(3 + a) * E + qb]; }
        double sgn = (s % 2) ? -1.0 : 1.0;
        double A2 = ann / (12.0 * h * h), B1 = sgn * bn / (12.0 * h);
        /* D_nn: (-G2 + 16G1 - 30U0 + 16U1 - U2) / (12 h^2);
         * D_n : sgn (8(U1 - G1) - (U2 - G2)) / (12 h) */
        double A[2][2] = {{16.0 * A2 - 8.0 * B1, -A2 + B1}, {-5.0, 1.0}};
        double rhs_b = G->f[qb];
        if (G->has_g) {
          double ht = G->h[1 - a];
          rhs_b -= P->omega * P->omega * G->gb[qb] +
                   G->c2[qb] * side_d2_g(G, s, t) / (12.0 * ht * ht);
        }
        double r[2] = {rhs_b * fcos - A2 * (-30.0 * U[0] + 16.0 * U[1] - U[2]) -
                           B1 * (8.0 * U[1] - U[2]),
                       -(10.0 * U[0] - 10.0 * U[1] + 5.0 * U[2] - U[3])};
        double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        W[gq[0]] = (r[0] * A[1][1] - A[0][1] * r[1]) / det;
        W[gq[1]] = (A[0][0] * r[1] - r[0] * A[1][0]) / det;
      }
    }
  }
}

/* Dissipation of the march's deviation from the periodic motion of the iterate (the
 * paper's upwind-dissipation variant leaves the form to its reference; this is the reading
 * used here): sum_a (-D+D-)^(p/2) h_a^p applied to Y = (W^n - W^{n-1}) - V0 (cos(omega_e
 * t^n) - cos(omega_e t^{n-1})), V0 the level-0 state after its boundary rules and
 * interpolation.  The operator is positive semi-definite and damps the grid-scale modes;
 * Y vanishes on W^n = V0 cos(omega_e t^n), so a fixed point of the iteration -- the
 * discrete Helmholtz solution -- stays one (the "additional correction" the paper asks for
 * to keep the exact match with the direct solve). */
static double dissipation(const or_problem *P, const or_grid *G, const double *Wn,
                          const double *Wm, const double *V0, int i, int j, double dc) {
  static const double c1[3] = {-1.0, 2.0, -1.0}, c2[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
  const int r = P->order / 2;
  const double *c = r == 1 ? c1 : c2;
  double s = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int k = -r; k <= r; ++k) {
      const long q = a == 0 ? at(G, i + k, j) : at(G, i, j + k);
      s += c[k + r] * ((Wn[q] - Wm[q]) - V0[q] * dc);
    }
  return s;
}

/* Interpolate every receiver from its donor stencil (Sec. 3.1). */
static void interpolate(const or_problem *P, double **W) {
  int w = P->order + 1;
  for (long r = 0; r < P->nrecv; ++r) {
    const or_grid *D = &P->G[P->dg[r]];
    double s = 0.0;
    for (int b = 0; b < w; ++b)
      for (int a = 0; a < w; ++a)
        s += P->wx[r * w + a] * P->wy[r * w + b] *
             W[P->dg[r]][at(D, P->di[r] + a, P->dj[r] + b)];
    W[P->rg[r]][at(&P->G[P->rg[r]], P->ri[r], P->rj[r])] = s;
  }
}

/* ------------------------------------------------------------ public API */

or_problem *or_new(int order) {
  if (order != 2 && order != 4) return NULL;
  or_problem *P = (or_problem *)calloc(1, sizeof(or_problem));
  P->order = order;
  return P;
}

const char *or_error(const or_problem *P) { return P->err; }

/* mask, c2 and f are compact (n1 x n0, i fastest); rx is over the extended extent. */
int or_add_grid(or_problem *P, int n0, int n1, int kind, const int *bc, int orthogonal,
                double h0, double h1, const signed char *mask, const double *rx,
                const double *c2) {
  if (P->ngrids >= OR_MAX_GRIDS) return -1;
  if ((bc[0] == OR_BC_PERIODIC) != (bc[1] == OR_BC_PERIODIC) ||
      (bc[2] == OR_BC_PERIODIC) != (bc[3] == OR_BC_PERIODIC)) {
    snprintf(P->err, sizeof P->err, "periodic must pair");
    return -1;
  }
  int phys = 0, neu = 0;
  for (int s = 0; s < 4; ++s) {
    phys |= bc[s] == OR_BC_DIRICHLET || bc[s] == OR_BC_NEUMANN;
    neu |= bc[s] == OR_BC_NEUMANN;
  }
  if (kind == OR_CURVILINEAR && !orthogonal && phys) {
    /* order 2 only: a Dirichlet side reads no ghost there, and a Neumann side's normal
     * derivative takes its tangential term along the side, which must be periodic */
    int ok = P->order == 2;
    for (int s = 0; s < 4; ++s)
      if (bc[s] == OR_BC_NEUMANN && bc[2 * (1 - s / 2)] != OR_BC_PERIODIC) ok = 0;
    if (!ok) {
      snprintf(P->err, sizeof P->err,
               "non-orthogonal grid with a physical boundary: order 2 only, Neumann sides "
               "along a periodic axis");
      return -1;
    }
  }
  if (neu) {
    /* a Neumann side may only meet periodic or interpolation sides: the fourth-order
     * Neumann ghost rule is unstable at corners shared with another physical side */
    for (int s = 0; s < 4; ++s)
      for (int s2 = 0; s2 < 4; ++s2)
        if (s / 2 != s2 / 2 && bc[s] == OR_BC_NEUMANN &&
            (bc[s2] == OR_BC_DIRICHLET || bc[s2] == OR_BC_NEUMANN)) {
          snprintf(P->err, sizeof P->err, "a Neumann side meets another physical side");
          return -1;
        }
  }
  or_grid *G = &P->G[P->ngrids];
  memset(G, 0, sizeof *G);
  G->n[0] = n0; G->n[1] = n1;
  for (int s = 0; s < 4; ++s) G->bc[s] = bc[s];
  for (int a = 0; a < 2; ++a) {
    G->g[a] = bc[2 * a] == OR_BC_PERIODIC ? 0 : P->order / 2;
    G->e[a] = G->n[a] + 2 * G->g[a];
  }
  G->kind = kind; G->orthogonal = orthogonal; G->h[0] = h0; G->h[1] = h1;
  long E = ext_size(G);
  G->mask = (signed char *)calloc(E, 1);
  G->c2 = (double *)malloc(E * sizeof(double));
  G->f = (double *)calloc(E, sizeof(double));
  G->gb = (double *)calloc(E, sizeof(double));
  G->gn = (double *)calloc(E, sizeof(double));
  for (long q = 0; q < E; ++q) G->c2[q] = 1.0;
  for (int j = 0; j < n1; ++j)
    for (int i = 0; i < n0; ++i) {
      long q = at(G, i, j);
      G->mask[q] = mask[(long)j * n0 + i];
      if (c2) G->c2[q] = c2[(long)j * n0 + i];
    }
  if (kind == OR_CURVILINEAR) {
    G->rx = (double *)malloc(4 * E * sizeof(double));
    memcpy(G->rx, rx, 4 * E * sizeof(double));
  }
  long off = 0;
  for (int g = 0; g < P->ngrids; ++g) off += (long)P->G[g].n[0] * P->G[g].n[1];
  G->offset = off;
  P->prepared = 0;
  return P->ngrids++;
}

int or_set_forcing(or_problem *P, int gidx, const double *f) {
  or_grid *G = &P->G[gidx];
  for (int j = 0; j < G->n[1]; ++j)
    for (int i = 0; i < G->n[0]; ++i) G->f[at(G, i, j)] = f[(long)j * G->n[0] + i];
  return 0;
}

int or_set_boundary(or_problem *P, int gidx, const double *g) {
  or_grid *G = &P->G[gidx];
  for (int j = 0; j < G->n[1]; ++j)
    for (int i = 0; i < G->n[0]; ++i) G->gb[at(G, i, j)] = g[(long)j * G->n[0] + i];
  G->has_g = 1;
  P->prepared = 0;
  return 0;
}

/* Neumann data of grid gidx (compact n1 x n0, read at the discretization points of its
 * Neumann sides): the outward normal derivative of the Helmholtz solution there. */
/* Dissipation coefficient nu >= 0 of the march (0: the plain scheme). */
int or_set_dissipation(or_problem *P, double nu) {
  if (!(nu >= 0.0)) return -1;
  P->nu = nu;
  return 0;
}

int or_set_neumann(or_problem *P, int gidx, const double *gn) {
  or_grid *G = &P->G[gidx];
  for (int j = 0; j < G->n[1]; ++j)
    for (int i = 0; i < G->n[0]; ++i) G->gn[at(G, i, j)] = gn[(long)j * G->n[0] + i];
  P->prepared = 0;
  return 0;
}

int or_set_interp(or_problem *P, long n, const int *rg, const int *ri, const int *rj,
                  const int *dg, const int *di, const int *dj, const double *wx,
                  const double *wy) {
  int w = P->order + 1;
  P->nrecv = n;
  int **dst[6] = {&P->rg, &P->ri, &P->rj, &P->dg, &P->di, &P->dj};
  const int *src[6] = {rg, ri, rj, dg, di, dj};
  for (int k = 0; k < 6; ++k) {
    free(*dst[k]);
    *dst[k] = (int *)malloc((n ? n : 1) * sizeof(int));
    if (n) memcpy(*dst[k], src[k], n * sizeof(int));
  }
  free(P->wx); free(P->wy);
  P->wx = (double *)malloc((n ? n : 1) * w * sizeof(double));
  P->wy = (double *)malloc((n ? n : 1) * w * sizeof(double));
  if (n) { memcpy(P->wx, wx, n * w * sizeof(double)); memcpy(P->wy, wy, n * w * sizeof(double)); }
  return 0;
}

/* Time setup for frequency omega (Recipe OmegaTildeExplicit; Eq. alphad).
 * alpha_mode 0: alpha_d; 1: alpha = 1/2.  out[0..6] = dt, omega_e, alpha, Nt, M, dt_max, Tbar. */
int or_prepare(or_problem *P, double omega, double cfl, int Np, int alpha_mode, double *out) {
  for (int g = 0; g < P->ngrids; ++g) {
    const or_grid *G = &P->G[g];
    if (!G->has_g || P->order != 4) continue;
    for (int s = 0; s < 4; ++s) {
      if (G->bc[s] != OR_BC_DIRICHLET) continue;
      if (G->kind != OR_CARTESIAN) {
        snprintf(P->err, sizeof P->err, "boundary data on a curvilinear Dirichlet side (order 4)");
        return -1;
      }
      if (G->n[1 - s / 2] < 6) {
        snprintf(P->err, sizeof P->err, "a side with boundary data needs 6 points (order 4)");
        return -1;
      }
    }
  }
  for (int g = 0; g < P->ngrids; ++g)
    if (P->G[g].kind == OR_CURVILINEAR) precompute_coeffs(P, &P->G[g]);
  double dtmax = cfl * dt_bound(P);
  int Nt = (int)ceil(2.0 * M_PI / (omega * dtmax));
  if (Nt < 2) Nt = 2;
  double dt = 2.0 / omega * sin(M_PI / Nt);
  while (dt > dtmax) { ++Nt; dt = 2.0 / omega * sin(M_PI / Nt); }
  P->omega = omega; P->cfl = cfl; P->Nt = Nt; P->Np = Np; P->M = Np * Nt; P->dt = dt;
  P->omega_e = 2.0 * M_PI / (Nt * dt);
  P->alpha = alpha_mode ? 0.5 : tan(P->omega_e * dt / 2.0) / tan(P->omega_e * dt);
  P->prepared = 1;
  if (out) {
    out[0] = dt; out[1] = P->omega_e; out[2] = P->alpha; out[3] = Nt; out[4] = P->M;
    out[5] = dtmax; out[6] = P->M * dt;
  }
  return 0;
}

/* One WaveHoltz iteration v_out = W_h(v_in, f) (forcing = 1) or W_h(v_in, 0)
 * (forcing = 0, Eq. MevalII).  Vectors are concatenated compact per-grid arrays. */
int or_iterate(or_problem *P, int forcing, const double *v_in, double *v_out) {
  if (!P->prepared) return -1;
  int ng = P->ngrids, M = P->M;
  double dt = P->dt, we = P->omega_e, fs = forcing ? 1.0 : 0.0;
  double *Wm[OR_MAX_GRIDS], *W0[OR_MAX_GRIDS], *Wp[OR_MAX_GRIDS], *V[OR_MAX_GRIDS];
  double *Vr[OR_MAX_GRIDS]; /* level 0 after its boundary rules and interpolation */
  for (int g = 0; g < ng; ++g) {
    long E = ext_size(&P->G[g]);
    Vr[g] = (double *)calloc(E, sizeof(double));
    Wm[g] = (double *)calloc(E, sizeof(double));
    W0[g] = (double *)calloc(E, sizeof(double));
    Wp[g] = (double *)calloc(E, sizeof(double));
    V[g] = (double *)calloc(E, sizeof(double));
  }
  /* time-filter weight of level n: (2/Tbar) sigma_n dt (cos(omega_e t^n) - alpha/2) */
#define FILTER_W(n) ((2.0 / (M * dt)) * (((n) == 0 || (n) == M) ? 0.5 : 1.0) * dt * \
                     (cos(we * (n) * dt) - P->alpha / 2.0))
  /* W^0 = v on active points; BC and interpolation at t = 0 */
  for (int g = 0; g < ng; ++g) {
    or_grid *G = &P->G[g];
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long q = at(G, i, j);
        signed char m = G->mask[q];
        double v = v_in[G->offset + (long)j * G->n[0] + i];
        W0[g][q] = (m == OR_DISC || m == OR_INTERP) ? v : (m == OR_DIRICHLET ? fs * G->gb[q] : 0.0);
      }
    apply_bc(P, g, W0[g], fs);
  }
  interpolate(P, W0);
  for (int g = 0; g < ng; ++g) memcpy(Vr[g], W0[g], ext_size(&P->G[g]) * sizeof(double));
  for (int n = 0; n < M; ++n) {
    double tn = n * dt;
    double wn = FILTER_W(n);
    for (int g = 0; g < ng; ++g) {
      or_grid *G = &P->G[g];
      long E = ext_size(G);
      /* OpenMP builds (timing only) split the point loops across threads; every point's
         arithmetic is the same, so the results are the same bits */
#pragma omp parallel for schedule(static)
      for (long q = 0; q < E; ++q)
        if (G->mask[q] != OR_UNUSED) V[g][q] += wn * W0[g][q];
    }
    /* advance every grid (Algorithm 2) */
    for (int g = 0; g < ng; ++g) {
      or_grid *G = &P->G[g];
      memset(Wp[g], 0, ext_size(G) * sizeof(double));
#pragma omp parallel for schedule(static)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          long q = at(G, i, j);
          if (G->mask[q] != OR_DISC) continue;
          double L = lap(P, G, W0[g], i, j);
          if (n == 0) /* W^1 = W^0 + dt^2/2 (c^2 L W^0 - f) */
            Wp[g][q] = W0[g][q] + 0.5 * dt * dt * (L - fs * G->f[q]);
          else /* W^{n+1} = 2W^n - W^{n-1} + dt^2 (c^2 L W^n - f cos(omega_e t^n)) */
            Wp[g][q] = 2.0 * W0[g][q] - Wm[g][q] + dt * dt * (L - fs * G->f[q] * cos(we * tn));
          if (n > 0 && P->nu > 0.0)
            Wp[g][q] -= P->nu * dissipation(P, G, W0[g], Wm[g], Vr[g], i, j,
                                            cos(we * tn) - cos(we * (tn - dt)));
        }
      /* Dirichlet points: the boundary data at t^{n+1} */
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          long q = at(G, i, j);
          if (G->mask[q] == OR_DIRICHLET) Wp[g][q] = fs * G->gb[q] * cos(we * (n + 1) * dt);
        }
      apply_bc(P, g, Wp[g], fs * cos(we * (n + 1) * dt));
    }
    interpolate(P, Wp);
    for (int g = 0; g < ng; ++g) {
      double *t = Wm[g]; Wm[g] = W0[g]; W0[g] = Wp[g]; Wp[g] = t;
    }
  }
  {
    double wn = FILTER_W(M);
    for (int g = 0; g < ng; ++g) {
      or_grid *G = &P->G[g];
      long E = ext_size(G);
#pragma omp parallel for schedule(static)
      for (long q = 0; q < E; ++q)
        if (G->mask[q] != OR_UNUSED) V[g][q] += wn * W0[g][q];
    }
  }
#undef FILTER_W
  for (int g = 0; g < ng; ++g) {
    or_grid *G = &P->G[g];
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        v_out[G->offset + (long)j * G->n[0] + i] = V[g][at(G, i, j)];
    free(Wm[g]); free(W0[g]); free(Wp[g]); free(V[g]); free(Vr[g]);
  }
  return 0;
}

/* ---- pieces exposed for the tests (pins check them one by one) ---- */

/* c^2 L_h applied to an extended array u of grid g, written at discretization points of
 * the extended array out (other entries untouched). */
int or_apply_lap(or_problem *P, int gidx, const double *u, double *out) {
  or_grid *G = &P->G[gidx];
  for (int j = 0; j < G->n[1]; ++j)
    for (int i = 0; i < G->n[0]; ++i) {
      long q = at(G, i, j);
      if (G->mask[q] == OR_DISC || G->mask[q] == OR_DIRICHLET) out[q] = lap(P, G, u, i, j);
    }
  return 0;
}

/* Ghost rules on an extended array; fcos multiplies f in the compatibility condition. */
int or_apply_bc(or_problem *P, int gidx, double *u, double fcos) {
  apply_bc(P, gidx, u, fcos);
  return 0;
}

/* Copy one of the five coefficient arrays (extended extent). */
int or_get_coef(or_problem *P, int gidx, int which, double *out) {
  or_grid *G = &P->G[gidx];
  if (!G->coef) return -1;
  memcpy(out, G->coef + which * ext_size(G), ext_size(G) * sizeof(double));
  return 0;
}

/* Interpolate receivers in a set of extended arrays (one pointer per grid). */
int or_interpolate(or_problem *P, double **u) {
  interpolate(P, u);
  return 0;
}

double or_b_mu(int mu) { return b_mu(mu); }

void or_free(or_problem *P) {
  if (!P) return;
  for (int g = 0; g < P->ngrids; ++g) {
    or_grid *G = &P->G[g];
    free(G->mask); free(G->rx); free(G->c2); free(G->f); free(G->gb); free(G->gn); free(G->coef);
  }
  free(P->rg); free(P->ri); free(P->rj); free(P->dg); free(P->di); free(P->dj);
  free(P->wx); free(P->wy);
  free(P);
}
