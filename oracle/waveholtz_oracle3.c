/*
 * waveholtz_oracle3.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of one WaveHoltz iteration on a
 * three-dimensional overset grid at second order (and at fourth order),
 * written from the paper (Appelo, Banks,
 * Henshaw, Schwendeman, "An optimal O(N) Helmholtz solver for complex geometry using
 * WaveHoltz and overset grids").  Only tests/, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header or table with the CUDA library
 * nor with the two-dimensional oracle.
 *
 * What it computes (each step cites the passage it follows):
 *   - time-step setup: the explicit CFL bound c dt sqrt(sum_k a_kk / dr_k^2 +
 *     2 sum_{k<l} |a_kl| / (dr_k dr_l)) <= 1 (Eq. dtForCartesian, Sec. 3.2, C = 1 at second
 *     order, frozen coefficients on curvilinear grids), then Recipe OmegaTildeExplicit
 *     (dt = (2/omega) sin(pi/Nt), omega_e = 2 pi/(Nt dt)) and alpha_d (Eq. alphad, Sec. 4.2);
 *   - the mapped Laplacian in three dimensions (Sec. 3.1, mapping method):
 *       L u = sum_k a_kk u_{r_k r_k} + 2 sum_{k<l} a_kl u_{r_k r_l} + sum_k b_k u_{r_k},
 *       a_kl = sum_m dr_k/dx_m dr_l/dx_m,  b_k = sum_m sum_l dr_l/dx_m d/dr_l(dr_k/dx_m),
 *     discretised with D+D- for the second derivatives, D0 for first derivatives and
 *     D0 D0 for mixed ones (Sec. 3.2, order 2); b_k from D0 differences of the metrics;
 *   - the explicit scheme D+tD-t W = c^2 L_h W - f cos(omega_e t) with the first step
 *     W^1 = W^0 + dt^2/2 (c^2 L_h W^0 - f) (Eq. WaveSchemeexplicit, Sec. 4.2);
 *   - Algorithm 2 per step: advance every grid, apply boundary conditions, interpolate;
 *   - tensor-product Lagrange interpolation from 3 x 3 x 3 donor stencils (Sec. 3.1);
 *   - the trapezoid-rule filter (Eq. updateDiscreteExplicit, Sec. 4.2), T-bar = Np Nt dt.
 *
 * Boundary data: Dirichlet points carry W_b = g_b cos(omega_e t) with g given per point
 * (o3_set_boundary; 0 when not given), switched off with the forcing.
 *
 * Ghost rules at second order (the paper defers them to its reference on overset wave
 * solvers):
 *   Dirichlet: W_b = g_b cos(omega_e t); ghosts are never read.
 *   Neumann:   centred normal derivative D0 W = 0 along the boundary's normal grid axis,
 *              i.e. W_{-1} = W_{+1}.  This is the normal derivative when the normal grid
 *              axis is orthogonal to the two tangential axes, which is required.
 * Grid lines of a pair of axes declared orthogonal drop the mixed term (a_kl = 0).
 *
 * Fourth order (o3_new_order(4)): two ghost layers, the second difference
 * D+D-(1 - h^2/12 D+D-) per axis (Eq. SecondDerivOrderp with mu < 2), on curvilinear grids
 * also the first difference D0(1 - h^2/6 D+D-) and its tensor product for the mixed terms
 * (and for b_k from the metrics), the stability constant C = sqrt(3)/2 in the time-step
 * bound, Lagrange interpolation of width 5, and the two-dimensional fourth-order ghost
 * rules applied along each face's normal axis (on a curvilinear grid a Dirichlet face's
 * compatibility condition takes c^2 (a_nn D_nn + b_n D_n); its normal axis must be
 * orthogonal to the others):
 *   Dirichlet: W_b = 0 (no boundary data at this order); c^2 D_nn W_b = f_b cos(omega_e t)
 *     (the tangential second differences of the zero boundary values vanish) and
 *     D+^5 W_{-2} = 0;
 *   Neumann: fourth-order centred D_n W = 0 and the same extrapolation; a Neumann face
 *     may only meet periodic or interpolation faces.
 */
#include <math.h>
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

enum { O3_UNUSED = 0, O3_DISC = 1, O3_INTERP = 2, O3_DIRICHLET = 3 };
enum { O3_BC_NONE = 0, O3_BC_DIRICHLET = 1, O3_BC_NEUMANN = 2, O3_BC_PERIODIC = 3 };
enum { O3_CARTESIAN = 0, O3_CURVILINEAR = 1 };
#define O3_MAX_GRIDS 64

/* Coefficient arrays (c^2 folded in), in this order. */
enum { C_A00 = 0, C_A11, C_A22, C_A01, C_A02, C_A12, C_B0, C_B1, C_B2, C_N };

typedef struct {
  int n[3], g[3], e[3];
  int kind;
  int fourth;      /* fourth-order differences (Cartesian grids of an order-4 problem) */
  int ortho;       /* bit 0: axes (0,1) orthogonal, bit 1: (0,2), bit 2: (1,2) */
  int bc[6];       /* [axis0 lo, axis0 hi, axis1 lo, axis1 hi, axis2 lo, axis2 hi] */
  double h[3];
  signed char *mask; /* extended */
  double *rx;      /* curvilinear: 9 extended arrays, rx[(3 k + m) E + q] = dr_k / dx_m */
  double *c2, *f;  /* extended */
  double *gb;      /* extended; Dirichlet boundary data (read at Dirichlet points) */
  double *gn;      /* extended; Neumann data du/dn along the outward normal (read at the
                      discretization points of Neumann faces) */
  double *coef;    /* curvilinear: C_N extended arrays */
  long offset;
} o3_grid;

typedef struct {
  int ngrids, order;
  o3_grid G[O3_MAX_GRIDS];
  long nrecv;
  int *rg, *ri, *rj, *rk, *dg, *di, *dj, *dk;
  double *wx, *wy, *wz;
  double omega, dt, omega_e, alpha, cfl;
  int Nt, Np, M, prepared;
  double nu;  /* dissipation of the deviation from the periodic motion (0: none) */
  char err[256];
} o3_problem;

/* pair index of axes a < b: (0,1) -> 0, (0,2) -> 1, (1,2) -> 2 */
static int pair_of(int a, int b) { return a + b - 1; }

static long ext_size(const o3_grid *G) { return (long)G->e[0] * G->e[1] * G->e[2]; }

static long at(const o3_grid *G, int i, int j, int k) {
  int ix[3] = {i, j, k};
  for (int a = 0; a < 3; ++a) {
    if (G->bc[2 * a] == O3_BC_PERIODIC) ix[a] = ((ix[a] % G->n[a]) + G->n[a]) % G->n[a];
    if (ix[a] < -G->g[a] || ix[a] >= G->n[a] + G->g[a]) {
      fprintf(stderr, "oracle3: index (%d,%d,%d) outside grid\n", i, j, k);
      abort();
    }
  }
  return ((long)(ix[2] + G->g[2]) * G->e[1] + (ix[1] + G->g[1])) * G->e[0] + (ix[0] + G->g[0]);
}

/* Value of W at (i, j, k) + d. */
static double val(const o3_grid *G, const double *W, int i, int j, int k, const int *d) {
  return W[at(G, i + d[0], j + d[1], k + d[2])];
}

/* D+D- W along axis a (divided); with two ghost layers (fourth order) the fourth-order
 * difference D+D-(1 - h^2/12 D+D-) = (-W_-2 + 16 W_-1 - 30 W + 16 W_+1 - W_+2) / (12 h^2). */
static double d2(const o3_grid *G, const double *W, int i, int j, int k, int a) {
  int p[3] = {0, 0, 0}, m[3] = {0, 0, 0}, z[3] = {0, 0, 0};
  p[a] = 1; m[a] = -1;
  const double s1 = val(G, W, i, j, k, p) - 2.0 * val(G, W, i, j, k, z) + val(G, W, i, j, k, m);
  if (G->fourth) {
    int p2[3] = {0, 0, 0}, m2[3] = {0, 0, 0};
    p2[a] = 2; m2[a] = -2;
    const double s2 = val(G, W, i, j, k, p2) - 4.0 * val(G, W, i, j, k, p) +
                      6.0 * val(G, W, i, j, k, z) - 4.0 * val(G, W, i, j, k, m) +
                      val(G, W, i, j, k, m2);
    return (s1 - s2 / 12.0) / (G->h[a] * G->h[a]);
  }
  return s1 / (G->h[a] * G->h[a]);
}

/* First-difference weights of offsets -2..2: D0 (second order) and, with two ghost layers,
 * D0(1 - h^2/6 D+D-) = (W_-2 - 8 W_-1 + 8 W_+1 - W_+2) / (12 h) (fourth order). */
static const double D1W2[5] = {0.0, -0.5, 0.0, 0.5, 0.0};
static const double D1W4[5] = {1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0};

/* First difference of W along axis a (divided). */
static double d1(const o3_grid *G, const double *W, int i, int j, int k, int a) {
  const double *w = G->fourth ? D1W4 : D1W2;
  double s = 0.0;
  for (int o = -2; o <= 2; ++o) {
    if (w[o + 2] == 0.0) continue;
    int d[3] = {0, 0, 0};
    d[a] = o;
    s += w[o + 2] * val(G, W, i, j, k, d);
  }
  return s / G->h[a];
}

/* Mixed difference along axes a != b: the product of the two first differences above
 * (D0_a D0_b at second order, its fourth-order counterpart with two ghost layers). */
static double d11(const o3_grid *G, const double *W, int i, int j, int k, int a, int b) {
  const double *w = G->fourth ? D1W4 : D1W2;
  double s = 0.0;
  for (int oa = -2; oa <= 2; ++oa)
    for (int ob = -2; ob <= 2; ++ob) {
      if (w[oa + 2] == 0.0 || w[ob + 2] == 0.0) continue;
      int d[3] = {0, 0, 0};
      d[a] = oa;
      d[b] = ob;
      s += w[oa + 2] * w[ob + 2] * val(G, W, i, j, k, d);
    }
  return s / (G->h[a] * G->h[b]);
}

/* c^2 L_h W at (i, j, k) (Sec. 3.1 mapping method; Cartesian: c^2 sum D+D-). */
static double lap(const o3_grid *G, const double *W, int i, int j, int k) {
  long q = at(G, i, j, k);
  if (G->kind == O3_CARTESIAN)
    return G->c2[q] * (d2(G, W, i, j, k, 0) + d2(G, W, i, j, k, 1) + d2(G, W, i, j, k, 2));
  long E = ext_size(G);
  const double *c = G->coef;
  double L = 0.0;
  for (int a = 0; a < 3; ++a) L += c[(C_A00 + a) * E + q] * d2(G, W, i, j, k, a);
  const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
  for (int p = 0; p < 3; ++p)
    if (!(G->ortho >> p & 1)) L += 2.0 * c[(C_A01 + p) * E + q] * d11(G, W, i, j, k, pa[p], pb[p]);
  for (int a = 0; a < 3; ++a) L += c[(C_B0 + a) * E + q] * d1(G, W, i, j, k, a);
  return L;
}

/* a_kl, b_k (c^2 folded in) at discretization and Dirichlet points. */
static void precompute_coeffs(o3_grid *G) {
  long E = ext_size(G);
  free(G->coef);
  G->coef = (double *)calloc(C_N * E, sizeof(double));
  const double *rx = G->rx;
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long q = at(G, i, j, k);
        signed char m = G->mask[q];
        if (m != O3_DISC && m != O3_DIRICHLET) continue;
        double a[3][3], b[3];
        for (int r = 0; r < 3; ++r)
          for (int s = 0; s < 3; ++s) {
            a[r][s] = 0.0;
            for (int mm = 0; mm < 3; ++mm) a[r][s] += rx[(3 * r + mm) * E + q] * rx[(3 * s + mm) * E + q];
          }
        for (int r = 0; r < 3; ++r) {
          b[r] = 0.0;
          for (int mm = 0; mm < 3; ++mm)
            for (int l = 0; l < 3; ++l)
              b[r] += rx[(3 * l + mm) * E + q] * d1(G, rx + (3 * r + mm) * E, i, j, k, l);
        }
        double c2 = G->c2[q];
        G->coef[C_A00 * E + q] = c2 * a[0][0];
        G->coef[C_A11 * E + q] = c2 * a[1][1];
        G->coef[C_A22 * E + q] = c2 * a[2][2];
        G->coef[C_A01 * E + q] = (G->ortho & 1) ? 0.0 : c2 * a[0][1];
        G->coef[C_A02 * E + q] = (G->ortho & 2) ? 0.0 : c2 * a[0][2];
        G->coef[C_A12 * E + q] = (G->ortho & 4) ? 0.0 : c2 * a[1][2];
        for (int r = 0; r < 3; ++r) G->coef[(C_B0 + r) * E + q] = c2 * b[r];
      }
}

/* Largest stable dt at second order, frozen coefficients (Eq. dtForCartesian). */
static double dt_bound(const o3_problem *P) {
  double smax = 0.0;
  for (int g = 0; g < P->ngrids; ++g) {
    const o3_grid *G = &P->G[g];
    long E = ext_size(G);
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          long q = at(G, i, j, k);
          if (G->mask[q] != O3_DISC) continue;
          double s = 0.0;
          if (G->kind == O3_CARTESIAN) {
            for (int a = 0; a < 3; ++a) s += 1.0 / (G->h[a] * G->h[a]);
            s *= G->c2[q];
          } else {
            for (int a = 0; a < 3; ++a) s += G->coef[(C_A00 + a) * E + q] / (G->h[a] * G->h[a]);
            const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
            for (int p = 0; p < 3; ++p)
              s += 2.0 * fabs(G->coef[(C_A01 + p) * E + q]) / (G->h[pa[p]] * G->h[pb[p]]);
          }
          if (s > smax) smax = s;
        }
  }
  return 1.0 / sqrt(smax);
}

/* Ghost points of every physical face at time t; fcos = cos(omega_e t) with the forcing on,
 * 0 with it off.  Second order: Neumann W_{-1} = W_{+1} next to discretization points.
 * Fourth order: the rules of the header, per boundary point along the face's normal axis
 * (U0..U3 the boundary point and three inward, G1, G2 the two ghosts). */
static void apply_bc(const o3_problem *P, int gidx, double *W, double fcos) {
  const o3_grid *G = &P->G[gidx];
  const long E = ext_size(G);
  for (int s = 0; s < 6; ++s) {
    const int code = G->bc[s];
    if (code != O3_BC_NEUMANN && !(code == O3_BC_DIRICHLET && G->fourth)) continue;
    int a = s / 2, hi = s % 2, t1 = (a + 1) % 3, t2 = (a + 2) % 3;
    for (int v = 0; v < G->n[t2]; ++v)
      for (int u = 0; u < G->n[t1]; ++u) {
        int ip[6][3];  /* offsets -2, -1, 0, 1, 2, 3 along the inward normal */
        for (int o = 0; o < 6; ++o) {
          ip[o][t1] = u;
          ip[o][t2] = v;
          ip[o][a] = hi ? G->n[a] - 1 - (o - 2) : (o - 2);
        }
        const long qb = at(G, ip[2][0], ip[2][1], ip[2][2]);
        const signed char m = G->mask[qb];
        /* Neumann data: du/dn = gn cos along the outward normal -+grad r_a / |grad r_a| is
         * du/dr_a = -+gq, gq = gn cos / |grad r_a| (|grad r_a| = 1 on Cartesian grids) */
        double gq = 0.0;
        if (code == O3_BC_NEUMANN && G->gn[qb] != 0.0) {
          double nrm = 1.0;
          if (G->kind == O3_CURVILINEAR) {
            double s2 = 0.0;
            for (int mm = 0; mm < 3; ++mm) s2 += G->rx[(3 * a + mm) * E + qb] * G->rx[(3 * a + mm) * E + qb];
            nrm = sqrt(s2);
          }
          gq = G->gn[qb] * fcos / nrm;
        }
        if (!G->fourth) {
          if (m != O3_DISC) continue;
          /* centred D0 along the inward direction: (U1 - G1) / (2 h) = -gq */
          W[at(G, ip[1][0], ip[1][1], ip[1][2])] = W[at(G, ip[3][0], ip[3][1], ip[3][2])] +
                                                   2.0 * G->h[a] * gq;
          continue;
        }
        if ((code == O3_BC_NEUMANN && m != O3_DISC) || (code == O3_BC_DIRICHLET && m != O3_DIRICHLET))
          continue;
        double U[4];
        for (int k = 0; k < 4; ++k) U[k] = W[at(G, ip[2 + k][0], ip[2 + k][1], ip[2 + k][2])];
        const long g1 = at(G, ip[1][0], ip[1][1], ip[1][2]), g2 = at(G, ip[0][0], ip[0][1], ip[0][2]);
        /* second row, D+^5 W_{-2} = 0:  G2 - 5 G1 + 10 U0 - 10 U1 + 5 U2 - U3 = 0 */
        double A[2][2], r[2];
        A[1][0] = -5.0; A[1][1] = 1.0;
        r[1] = -(10.0 * U[0] - 10.0 * U[1] + 5.0 * U[2] - U[3]);
        if (code == O3_BC_NEUMANN) {
          /* 8 (U1 - G1) - (U2 - G2) = -12 h gq (the fourth-order D_n inward, undivided) */
          A[0][0] = -8.0; A[0][1] = 1.0;
          r[0] = -(8.0 * U[1] - U[2]) - 12.0 * G->h[a] * gq;
        } else {
          /* c^2 (a_nn D_nn W + b_n D_n W)_b = f_b cos, D_nn = (-G2 + 16 G1 - 30 U0 +
           * 16 U1 - U2) / (12 h^2) and D_n along +r_a, i.e. +-(-U2 + 8 U1 - 8 G1 + G2) /
           * (12 h) with + on a low side (Cartesian grids: a_nn = 1, b_n = 0) */
          double ann = G->c2[qb], bn = 0.0;
          if (G->kind == O3_CURVILINEAR) {
            ann = G->coef[(C_A00 + a) * E + qb];
            bn = G->coef[(C_B0 + a) * E + qb];
          }
          const double A2 = ann / (12.0 * G->h[a] * G->h[a]);
          const double B1 = (hi ? -1.0 : 1.0) * bn / (12.0 * G->h[a]);
          A[0][0] = 16.0 * A2 - 8.0 * B1; A[0][1] = -A2 + B1;
          r[0] = G->f[qb] * fcos - A2 * (-30.0 * U[0] + 16.0 * U[1] - U[2]) -
                 B1 * (8.0 * U[1] - U[2]);
        }
        const double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
        W[g1] = (r[0] * A[1][1] - A[0][1] * r[1]) / det;
        W[g2] = (A[0][0] * r[1] - r[0] * A[1][0]) / det;
      }
  }
}

/* Every receiver from its (p + 1)^3 donor stencil (Sec. 3.1). */
static void interpolate(const o3_problem *P, double **W) {
  const int w = P->order + 1;
  for (long r = 0; r < P->nrecv; ++r) {
    const o3_grid *D = &P->G[P->dg[r]];
    double s = 0.0;
    for (int c = 0; c < w; ++c)
      for (int b = 0; b < w; ++b)
        for (int a = 0; a < w; ++a)
          s += P->wx[r * w + a] * P->wy[r * w + b] * P->wz[r * w + c] *
               W[P->dg[r]][at(D, P->di[r] + a, P->dj[r] + b, P->dk[r] + c)];
    W[P->rg[r]][at(&P->G[P->rg[r]], P->ri[r], P->rj[r], P->rk[r])] = s;
  }
}

/* ------------------------------------------------------------ public API */

o3_problem *o3_new_order(int order) {
  if (order != 2 && order != 4) return NULL;
  o3_problem *P = (o3_problem *)calloc(1, sizeof(o3_problem));
  if (P) P->order = order;
  return P;
}

o3_problem *o3_new(void) { return o3_new_order(2); }

const char *o3_error(const o3_problem *P) { return P->err; }

/* mask, c2 are compact (n2 x n1 x n0, axis 0 fastest); rx covers the extended extent. */
int o3_add_grid(o3_problem *P, int n0, int n1, int n2, int kind, const int *bc, int ortho,
                double h0, double h1, double h2, const signed char *mask, const double *rx,
                const double *c2) {
  if (P->ngrids >= O3_MAX_GRIDS) return -1;
  for (int a = 0; a < 3; ++a)
    if ((bc[2 * a] == O3_BC_PERIODIC) != (bc[2 * a + 1] == O3_BC_PERIODIC)) {
      snprintf(P->err, sizeof P->err, "periodic must pair");
      return -1;
    }
  for (int s = 0; s < 6; ++s) {
    if (bc[s] != O3_BC_NEUMANN) continue;
    int a = s / 2;
    for (int b = 0; b < 3; ++b) {
      if (b == a) continue;
      int p = pair_of(a < b ? a : b, a < b ? b : a);
      if (kind == O3_CURVILINEAR && !(ortho >> p & 1)) {
        snprintf(P->err, sizeof P->err, "Neumann axis not orthogonal to the tangential axes");
        return -1;
      }
    }
  }
  if (P->order == 4) {
    /* a Dirichlet face's fourth-order rule on a curvilinear grid takes the normal axis's
     * own terms only: that axis must be orthogonal to the two others */
    if (kind != O3_CARTESIAN)
      for (int s = 0; s < 6; ++s) {
        if (bc[s] != O3_BC_DIRICHLET) continue;
        for (int b = 0; b < 3; ++b) {
          const int a = s / 2;
          if (b == a) continue;
          if (!(ortho >> pair_of(a < b ? a : b, a < b ? b : a) & 1)) {
            snprintf(P->err, sizeof P->err,
                     "fourth order: a Dirichlet face's normal axis must be orthogonal to the others");
            return -1;
          }
        }
      }
    /* the fourth-order Neumann rule is unstable at corners with another physical side */
    for (int s = 0; s < 6; ++s)
      for (int s2 = 0; s2 < 6; ++s2)
        if (s / 2 != s2 / 2 && bc[s] == O3_BC_NEUMANN &&
            (bc[s2] == O3_BC_DIRICHLET || bc[s2] == O3_BC_NEUMANN)) {
          snprintf(P->err, sizeof P->err, "a Neumann face meets another physical face");
          return -1;
        }
  }
  o3_grid *G = &P->G[P->ngrids];
  memset(G, 0, sizeof *G);
  G->n[0] = n0; G->n[1] = n1; G->n[2] = n2;
  G->fourth = P->order == 4;
  for (int s = 0; s < 6; ++s) G->bc[s] = bc[s];
  for (int a = 0; a < 3; ++a) {
    G->g[a] = bc[2 * a] == O3_BC_PERIODIC ? 0 : P->order / 2;
    G->e[a] = G->n[a] + 2 * G->g[a];
  }
  G->kind = kind; G->ortho = kind == O3_CARTESIAN ? 7 : ortho;
  G->h[0] = h0; G->h[1] = h1; G->h[2] = h2;
  long E = ext_size(G);
  G->mask = (signed char *)calloc(E, 1);
  G->c2 = (double *)malloc(E * sizeof(double));
  G->f = (double *)calloc(E, sizeof(double));
  G->gb = (double *)calloc(E, sizeof(double));
  G->gn = (double *)calloc(E, sizeof(double));
  for (long q = 0; q < E; ++q) G->c2[q] = 1.0;
  for (int k = 0; k < n2; ++k)
    for (int j = 0; j < n1; ++j)
      for (int i = 0; i < n0; ++i) {
        long q = at(G, i, j, k), c = ((long)k * n1 + j) * n0 + i;
        G->mask[q] = mask[c];
        if (c2) G->c2[q] = c2[c];
      }
  if (kind == O3_CURVILINEAR) {
    G->rx = (double *)malloc(9 * E * sizeof(double));
    memcpy(G->rx, rx, 9 * E * sizeof(double));
  }
  long off = 0;
  for (int g = 0; g < P->ngrids; ++g) off += (long)P->G[g].n[0] * P->G[g].n[1] * P->G[g].n[2];
  G->offset = off;
  P->prepared = 0;
  return P->ngrids++;
}

int o3_set_forcing(o3_problem *P, int gidx, const double *f) {
  o3_grid *G = &P->G[gidx];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        G->f[at(G, i, j, k)] = f[((long)k * G->n[1] + j) * G->n[0] + i];
  return 0;
}

int o3_set_boundary(o3_problem *P, int gidx, const double *g) {
  o3_grid *G = &P->G[gidx];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        G->gb[at(G, i, j, k)] = g[((long)k * G->n[1] + j) * G->n[0] + i];
  return 0;
}

/* Neumann data (compact; read at the discretization points of Neumann faces): the ghost
 * rule makes the outward normal derivative gn cos(omega_e t) instead of 0, switched off with
 * the forcing. */
int o3_set_neumann(o3_problem *P, int gidx, const double *gn) {
  o3_grid *G = &P->G[gidx];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i)
        G->gn[at(G, i, j, k)] = gn[((long)k * G->n[1] + j) * G->n[0] + i];
  return 0;
}

int o3_set_interp(o3_problem *P, long n, const int *rg, const int *ri, const int *rj,
                  const int *rk, const int *dg, const int *di, const int *dj, const int *dk,
                  const double *wx, const double *wy, const double *wz) {
  P->nrecv = n;
  int **dst[8] = {&P->rg, &P->ri, &P->rj, &P->rk, &P->dg, &P->di, &P->dj, &P->dk};
  const int *src[8] = {rg, ri, rj, rk, dg, di, dj, dk};
  for (int q = 0; q < 8; ++q) {
    free(*dst[q]);
    *dst[q] = (int *)malloc((n ? n : 1) * sizeof(int));
    if (n) memcpy(*dst[q], src[q], n * sizeof(int));
  }
  double **wd[3] = {&P->wx, &P->wy, &P->wz};
  const double *ws[3] = {wx, wy, wz};
  for (int q = 0; q < 3; ++q) {
    free(*wd[q]);
    const int w = P->order + 1;
    *wd[q] = (double *)malloc((n ? n : 1) * w * sizeof(double));
    if (n) memcpy(*wd[q], ws[q], n * w * sizeof(double));
  }
  return 0;
}

/* Time setup (Recipe OmegaTildeExplicit; Eq. alphad).
 * out[0..6] = dt, omega_e, alpha, Nt, M, dt_max, Tbar. */
int o3_prepare(o3_problem *P, double omega, double cfl, int Np, int alpha_mode, double *out) {
  for (int g = 0; g < P->ngrids; ++g)
    if (P->G[g].kind == O3_CURVILINEAR) precompute_coeffs(&P->G[g]);
  if (P->order == 4)
    for (int g = 0; g < P->ngrids; ++g) {
      const o3_grid *G = &P->G[g];
      for (long q = 0; q < ext_size(G); ++q)
        if (G->mask[q] == O3_DIRICHLET && G->gb[q] != 0.0) {
          snprintf(P->err, sizeof P->err, "boundary data at fourth order in 3D");
          return -1;
        }
    }
  /* Eq. dtForCartesian: C = 1 at second order, sqrt(3)/2 at fourth */
  double dtmax = cfl * (P->order == 4 ? sqrt(3.0) / 2.0 : 1.0) * dt_bound(P);
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

/* Dissipation of the march's deviation from the periodic motion of the iterate (the
 * paper's upwind-dissipation variant leaves the form to its reference; the same reading as
 * in two dimensions): sum_a (-D+D-)^(p/2) h_a^p applied to Y = (W^n - W^{n-1}) -
 * V0 (cos(omega_e t^n) - cos(omega_e t^{n-1})), V0 the level-0 state after its boundary
 * rules and interpolation.  Positive semi-definite, it damps grid-scale modes; Y vanishes
 * on W^n = V0 cos(omega_e t^n), so the discrete Helmholtz solution stays a fixed point. */
static double dissipation(const o3_problem *P, const o3_grid *G, const double *Wn,
                          const double *Wm, const double *V0, int i, int j, int k, double dc) {
  static const double c1[3] = {-1.0, 2.0, -1.0}, c2[5] = {1.0, -4.0, 6.0, -4.0, 1.0};
  const int r = P->order / 2;
  const double *c = r == 1 ? c1 : c2;
  double s = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int o = -r; o <= r; ++o) {
      const long q = at(G, i + (a == 0 ? o : 0), j + (a == 1 ? o : 0), k + (a == 2 ? o : 0));
      s += c[o + r] * ((Wn[q] - Wm[q]) - V0[q] * dc);
    }
  return s;
}

int o3_set_dissipation(o3_problem *P, double nu) {
  if (!(nu >= 0.0)) return -1;
  P->nu = nu;
  return 0;
}

/* One WaveHoltz iteration v_out = W_h(v_in, f) (forcing = 1) or W_h(v_in, 0). */
int o3_iterate(o3_problem *P, int forcing, const double *v_in, double *v_out) {
  if (!P->prepared) return -1;
  int ng = P->ngrids, M = P->M;
  double dt = P->dt, we = P->omega_e, fs = forcing ? 1.0 : 0.0;
  double *Wm[O3_MAX_GRIDS], *W0[O3_MAX_GRIDS], *Wp[O3_MAX_GRIDS], *V[O3_MAX_GRIDS];
  double *Vr[O3_MAX_GRIDS]; /* level 0 after its boundary rules and interpolation */
  for (int g = 0; g < ng; ++g) {
    long E = ext_size(&P->G[g]);
    Wm[g] = (double *)calloc(E, sizeof(double));
    W0[g] = (double *)calloc(E, sizeof(double));
    Wp[g] = (double *)calloc(E, sizeof(double));
    V[g] = (double *)calloc(E, sizeof(double));
    Vr[g] = (double *)calloc(E, sizeof(double));
  }
  /* filter weight of level n: (2/Tbar) sigma_n dt (cos(omega_e t^n) - alpha/2) */
#define FILTER_W(n) ((2.0 / (M * dt)) * (((n) == 0 || (n) == M) ? 0.5 : 1.0) * dt * \
                     (cos(we * (n) * dt) - P->alpha / 2.0))
  for (int g = 0; g < ng; ++g) {
    o3_grid *G = &P->G[g];
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i) {
          long q = at(G, i, j, k);
          signed char m = G->mask[q];
          double v = v_in[G->offset + ((long)k * G->n[1] + j) * G->n[0] + i];
          W0[g][q] = (m == O3_DISC || m == O3_INTERP) ? v : (m == O3_DIRICHLET ? fs * G->gb[q] : 0.0);
        }
    apply_bc(P, g, W0[g], fs);
  }
  interpolate(P, W0);
  for (int g = 0; g < ng; ++g) memcpy(Vr[g], W0[g], ext_size(&P->G[g]) * sizeof(double));
  for (int n = 0; n < M; ++n) {
    double tn = n * dt, wn = FILTER_W(n);
    for (int g = 0; g < ng; ++g) {
      o3_grid *G = &P->G[g];
      long E = ext_size(G);
      /* OpenMP builds (timing only) split the point loops across threads; every point's
         arithmetic is the same, so the results are the same bits */
#pragma omp parallel for schedule(static)
      for (long q = 0; q < E; ++q)
        if (G->mask[q] != O3_UNUSED) V[g][q] += wn * W0[g][q];
    }
    for (int g = 0; g < ng; ++g) {
      o3_grid *G = &P->G[g];
      memset(Wp[g], 0, ext_size(G) * sizeof(double));
#pragma omp parallel for schedule(static)
      for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
          for (int i = 0; i < G->n[0]; ++i) {
            long q = at(G, i, j, k);
            if (G->mask[q] != O3_DISC) continue;
            double L = lap(G, W0[g], i, j, k);
            if (n == 0)
              Wp[g][q] = W0[g][q] + 0.5 * dt * dt * (L - fs * G->f[q]);
            else
              Wp[g][q] = 2.0 * W0[g][q] - Wm[g][q] + dt * dt * (L - fs * G->f[q] * cos(we * tn));
            if (n > 0 && P->nu > 0.0)
              Wp[g][q] -= P->nu * dissipation(P, G, W0[g], Wm[g], Vr[g], i, j, k,
                                              cos(we * tn) - cos(we * (tn - dt)));
          }
      /* Dirichlet points: the boundary data at t^{n+1} */
      for (int k = 0; k < G->n[2]; ++k)
        for (int j = 0; j < G->n[1]; ++j)
          for (int i = 0; i < G->n[0]; ++i) {
            long q = at(G, i, j, k);
            if (G->mask[q] == O3_DIRICHLET) Wp[g][q] = fs * G->gb[q] * cos(we * (n + 1) * dt);
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
      o3_grid *G = &P->G[g];
      long E = ext_size(G);
#pragma omp parallel for schedule(static)
      for (long q = 0; q < E; ++q)
        if (G->mask[q] != O3_UNUSED) V[g][q] += wn * W0[g][q];
    }
  }
#undef FILTER_W
  for (int g = 0; g < ng; ++g) {
    o3_grid *G = &P->G[g];
    for (int k = 0; k < G->n[2]; ++k)
      for (int j = 0; j < G->n[1]; ++j)
        for (int i = 0; i < G->n[0]; ++i)
          v_out[G->offset + ((long)k * G->n[1] + j) * G->n[0] + i] = V[g][at(G, i, j, k)];
    free(Wm[g]); free(W0[g]); free(Wp[g]); free(V[g]); free(Vr[g]);
  }
  return 0;
}

/* ---- pieces exposed for the tests ---- */

/* c^2 L_h of an extended array of grid g at discretization and Dirichlet points. */
int o3_apply_lap(o3_problem *P, int gidx, const double *u, double *out) {
  o3_grid *G = &P->G[gidx];
  for (int k = 0; k < G->n[2]; ++k)
    for (int j = 0; j < G->n[1]; ++j)
      for (int i = 0; i < G->n[0]; ++i) {
        long q = at(G, i, j, k);
        if (G->mask[q] == O3_DISC || G->mask[q] == O3_DIRICHLET) out[q] = lap(G, u, i, j, k);
      }
  return 0;
}

int o3_apply_bc(o3_problem *P, int gidx, double *u) {
  apply_bc(P, gidx, u, 0.0);  /* zero forcing */
  return 0;
}

/* The ghost rules with the forcing factor fcos (the order-4 Dirichlet compatibility
 * condition's f_b cos(omega t) term), for the implicit scheme's level systems. */
int o3_apply_bc_forced(o3_problem *P, int gidx, double *u, double fcos) {
  apply_bc(P, gidx, u, fcos);
  return 0;
}

int o3_get_coef(o3_problem *P, int gidx, int which, double *out) {
  o3_grid *G = &P->G[gidx];
  if (!G->coef || which < 0 || which >= C_N) return -1;
  memcpy(out, G->coef + which * ext_size(G), ext_size(G) * sizeof(double));
  return 0;
}

int o3_interpolate(o3_problem *P, double **u) {
  interpolate(P, u);
  return 0;
}

void o3_free(o3_problem *P) {
  if (!P) return;
  for (int g = 0; g < P->ngrids; ++g) {
    o3_grid *G = &P->G[g];
    free(G->mask); free(G->rx); free(G->c2); free(G->f); free(G->gb); free(G->gn); free(G->coef);
  }
  free(P->rg); free(P->ri); free(P->rj); free(P->rk);
  free(P->dg); free(P->di); free(P->dj); free(P->dk);
  free(P->wx); free(P->wy); free(P->wz);
  free(P);
}
