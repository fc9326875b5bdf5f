// wh_kernels3.cu -- CUDA kernels of the three-dimensional WaveHoltz path (sm_103a): second
// order on any grid, fourth order on Cartesian grids (march3o4 / gather3o4 at the end).
//
// One WaveHoltz iteration (Algorithm 1) on a 3D overset grid is
//   init3 -> gather3(level 0) -> [march3(n) -> gather3(level n + 1)] for n < M -> finish3:
//   - march3: the explicit scheme of Eq. WaveSchemeexplicit (Sec. 4.2) at every
//     discretization point of every grid, the stencil of the mapped Laplacian (Sec. 3.1,
//     second order: D+D-, D0, D0 D0) with dt^2 c^2 folded into per-point or constant
//     weights, the forcing term, and the filter accumulation of Eq. updateDiscreteExplicit
//     fused into the write of W^{n+1}.  W^{n+1} overwrites W^{n-1} in place.
//   - gather3: the ghost rules (Neumann: centred normal derivative, a copy of the inward
//     value) and the explicit interpolation of every receiver from its 3 x 3 x 3 donor
//     stencil (Sec. 3.1, Algorithm 2: boundary conditions and interpolation after every
//     grid has advanced), one thread per receiver evaluating the tensor product axis by
//     axis (the FP64 pipe, not memory, bounds a lane-per-donor form on GB300).  Receivers
//     add their filter term too.
// Setup kernels compute the mapped-Laplacian coefficients a_kl, b_k from the metrics with
// the CFL bound (Eq. dtForCartesian), and the stencil weights for one dt.
#include <cuda_runtime.h>

#include <cstdint>

#include "wh3_internal.h"
#include "wh_widen.cuh"

namespace wh3 {
namespace {

constexpr int8_t kDisc = WH_DISC, kInterpPt = WH_INTERP, kDirichlet = WH_DIRICHLET;

__device__ __forceinline__ int wrap(int i, int n, int per) {
  if (!per) return i;
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

__device__ __forceinline__ int64_t at3(const Grid3Dev &G, int i, int j, int k) {
  return G.base + ((int64_t)(k + G.g2) * G.e1 + (j + G.g1)) * G.e0 + (i + G.g0);
}

// Index of (i + di, j + dj, k + dk), wrapping periodic axes.
__device__ __forceinline__ int64_t nb3(const Grid3Dev &G, int i, int j, int k, int di, int dj,
                                       int dk) {
  return at3(G, wrap(i + di, G.n0, G.per & 1), wrap(j + dj, G.n1, G.per & 2),
             wrap(k + dk, G.n2, G.per & 4));
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *a, double v) {
  // positive doubles order like their bit patterns
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------- setup kernels

// Coefficients c^2 a_kl, c^2 b_k at discretization and Dirichlet points of a curvilinear
// grid (Sec. 3.1: a_kl = sum_m dr_k/dx_m dr_l/dx_m, b_k = sum_m sum_l dr_l/dx_m
// D0_l(dr_k/dx_m)); mixed coefficients of pairs declared orthogonal are 0.  At
// discretization points of every grid, the frozen-coefficient CFL quantity
// sum_k a_kk / h_k^2 + 2 sum_{k<l} |a_kl| / (h_k h_l) goes into smax.
__global__ void coef3_kernel(const Grid3Dev *grids, int gidx, const int8_t *mask,
                             const double *rx, const double *c2, double *coef,
                             unsigned long long *smax) {
  const Grid3Dev G = grids[gidx];
  const int64_t npts = (int64_t)G.n0 * G.n1 * G.n2;
  const int64_t E = G.ext;
  double local = 0.0;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % G.n0), j = (int)((t / G.n0) % G.n1), k = (int)(t / ((int64_t)G.n0 * G.n1));
    const int64_t q = at3(G, i, j, k), ql = q - G.base;
    const int8_t m = mask[q];
    if (m != kDisc && m != kDirichlet) continue;
    const double c2q = c2[q];
    if (G.kind == WH_CARTESIAN) {
      if (m == kDisc) {
        double s = 1.0 / (G.h[0] * G.h[0]) + 1.0 / (G.h[1] * G.h[1]) + 1.0 / (G.h[2] * G.h[2]);
        local = fmax(local, c2q * s);
      }
      continue;
    }
    const double *R = rx + G.rbase;
    double r[9];
#pragma unroll
    for (int p = 0; p < 9; ++p) r[p] = R[p * E + ql];
    double a[3][3];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) a[u][v] = r[3 * u] * r[3 * v] + r[3 * u + 1] * r[3 * v + 1] +
                                            r[3 * u + 2] * r[3 * v + 2];
    // neighbour offsets (relative to the grid's base) along each parameter axis
    int64_t qp[3], qm[3];
    qp[0] = nb3(G, i, j, k, 1, 0, 0) - G.base;
    qm[0] = nb3(G, i, j, k, -1, 0, 0) - G.base;
    qp[1] = nb3(G, i, j, k, 0, 1, 0) - G.base;
    qm[1] = nb3(G, i, j, k, 0, -1, 0) - G.base;
    qp[2] = nb3(G, i, j, k, 0, 0, 1) - G.base;
    qm[2] = nb3(G, i, j, k, 0, 0, -1) - G.base;
    double b[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      double s = 0.0;
#pragma unroll
      for (int mm = 0; mm < 3; ++mm) {
        const double *P = R + (3 * u + mm) * E;
#pragma unroll
        for (int l = 0; l < 3; ++l) s += r[3 * l + mm] * ((P[qp[l]] - P[qm[l]]) / (2.0 * G.h[l]));
      }
      b[u] = s;
    }
    double *C = coef + G.kbase;
    const double A01 = (G.ortho & 1) ? 0.0 : c2q * a[0][1];
    const double A02 = (G.ortho & 2) ? 0.0 : c2q * a[0][2];
    const double A12 = (G.ortho & 4) ? 0.0 : c2q * a[1][2];
    C[kA00 * E + ql] = c2q * a[0][0];
    C[kA11 * E + ql] = c2q * a[1][1];
    C[kA22 * E + ql] = c2q * a[2][2];
    C[kA01 * E + ql] = A01;
    C[kA02 * E + ql] = A02;
    C[kA12 * E + ql] = A12;
    C[kB0 * E + ql] = c2q * b[0];
    C[kB1 * E + ql] = c2q * b[1];
    C[kB2 * E + ql] = c2q * b[2];
    if (m == kDisc) {
      double s = c2q * a[0][0] / (G.h[0] * G.h[0]) + c2q * a[1][1] / (G.h[1] * G.h[1]) +
                 c2q * a[2][2] / (G.h[2] * G.h[2]);
      s += 2.0 * fabs(A01) / (G.h[0] * G.h[1]) + 2.0 * fabs(A02) / (G.h[0] * G.h[2]) +
           2.0 * fabs(A12) / (G.h[1] * G.h[2]);
      local = fmax(local, s);
    }
  }
  if (local > 0.0) atomic_max_pos(smax, local);
}

// Per-point stencil weights with dt^2 folded in (the centre carries the "2" of the
// leapfrog): centre 2 - 2 dt^2 sum_k a_kk/h_k^2; face -+k: dt^2 (a_kk/h_k^2 -+ b_k/(2 h_k));
// edge (k,l): +-dt^2 a_kl / (2 h_k h_l) (from 2 a_kl D0_k D0_l).  Cartesian grids with c(x)
// use a_kk = c^2, b = 0.
template <typename T>
__global__ void weight3_kernel(const Grid3Dev *grids, int gidx, const int8_t *mask,
                               const double *coef, const double *c2, T *Wt, double dt2) {
  const Grid3Dev G = grids[gidx];
  const int64_t npts = (int64_t)G.n0 * G.n1 * G.n2;
  const int64_t E = G.ext;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % G.n0), j = (int)((t / G.n0) % G.n1), k = (int)(t / ((int64_t)G.n0 * G.n1));
    const int64_t q = at3(G, i, j, k), ql = q - G.base;
    if (mask[q] != kDisc) continue;
    double A[3], B[3], Mx[3] = {0.0, 0.0, 0.0};
    if (G.kind == WH_CARTESIAN) {
      A[0] = A[1] = A[2] = c2[q];
      B[0] = B[1] = B[2] = 0.0;
    } else {
      const double *C = coef + G.kbase;
      A[0] = C[kA00 * E + ql];
      A[1] = C[kA11 * E + ql];
      A[2] = C[kA22 * E + ql];
      B[0] = C[kB0 * E + ql];
      B[1] = C[kB1 * E + ql];
      B[2] = C[kB2 * E + ql];
      Mx[0] = C[kA01 * E + ql];
      Mx[1] = C[kA02 * E + ql];
      Mx[2] = C[kA12 * E + ql];
    }
    T *W = Wt + G.wbase + ql;
    double xs[3], ys[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xs[a] = dt2 * A[a] / (G.h[a] * G.h[a]);
      ys[a] = dt2 * B[a] / (2.0 * G.h[a]);
    }
    W[0] = (T)(2.0 - 2.0 * (xs[0] + xs[1] + xs[2]));
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      W[(1 + 2 * a) * E] = (T)(xs[a] - ys[a]);
      W[(2 + 2 * a) * E] = (T)(xs[a] + ys[a]);
    }
    if (G.stencil == kPoint19) {
      const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const double z = dt2 * Mx[p] / (2.0 * G.h[pa[p]] * G.h[pb[p]]);
        W[(7 + 4 * p) * E] = (T)z;       // (-,-)
        W[(8 + 4 * p) * E] = (T)(-z);    // (+,-)
        W[(9 + 4 * p) * E] = (T)(-z);    // (-,+)
        W[(10 + 4 * p) * E] = (T)z;      // (+,+)
      }
    }
  }
}

// ---------------------------------------------------------------- iteration kernels

// W^0 = v at discretization and interpolation points, 0 elsewhere (ghosts included);
// V = w_0 W^0 at discretization points, 0 elsewhere (receivers add theirs after the
// level-0 interpolation).  blockIdx.y = grid.
template <typename T>
__global__ void init3_kernel(const Grid3Dev *grids, const int8_t *mask, const double *vin,
                             T *W0, double *V, const double *wf) {
  const Grid3Dev G = grids[blockIdx.y];
  const double w0 = wf[0];
  const int64_t pl = (int64_t)G.e0 * G.e1;
  for (int64_t ql = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ql < G.ext;
       ql += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(ql % G.e0) - G.g0, j = (int)((ql / G.e0) % G.e1) - G.g1,
              k = (int)(ql / pl) - G.g2;
    const int64_t q = G.base + ql;
    const int8_t m = mask[q];
    double v = 0.0;
    if ((m == kDisc || m == kInterpPt) && i >= 0 && i < G.n0 && j >= 0 && j < G.n1 && k >= 0 &&
        k < G.n2)
      v = vin[G.cbase + ((int64_t)k * G.n1 + j) * G.n0 + i];
    const T w = (T)v;
    W0[q] = w;
    V[q] = m == kDisc ? w0 * (double)w : 0.0;
  }
}

template <typename T>
__device__ __forceinline__ T fsel(double d, float f);
template <>
__device__ __forceinline__ double fsel<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float fsel<float>(double, float f) { return f; }

// One FP32 update of a constant-weight 7-point point (Eq. WaveSchemeexplicit, weights with
// dt^2 folded, centre including the "2"): W^{n+1} = c0 W + c1 (W_x- + W_x+) + c2 (W_y- + W_y+)
// + c3 (W_z- + W_z+) - W^{n-1} - fc_n F, every rounding fixed by the intrinsics so that the
// single-step march and the temporally blocked one give the same bits.
__device__ __forceinline__ float step7f(float c0, float c1, float c2, float c3, float wc,
                                        float sx, float sy, float sz, float wo, float fcs,
                                        float fq) {
  float S = __fmul_rn(c0, wc);
  S = __fmaf_rn(c1, sx, S);
  S = __fmaf_rn(c2, sy, S);
  S = __fmaf_rn(c3, sz, S);
  return __fmaf_rn(-fcs, fq, __fsub_rn(S, wo));
}

// One time step n -> n + 1 of every grid (Eq. WaveSchemeexplicit) with the fused filter
// term of level n + 1.  Block = one Tile3; each thread marches kTZ points along axis 2.
// W^{n-1} comes from Wprev, which is Wout itself in the two-level in-place layout (so
// neither carries __restrict__).
// Register caps for occupancy: FP32 48 (5 blocks per SM), FP64 64 (4), neither spills.
template <typename T>
__global__ void __launch_bounds__(kTX *kTY, sizeof(T) == 4 ? 5 : 4) march3_kernel(
    const Grid3Dev *__restrict__ grids, const Tile3 *__restrict__ tiles,
    const int8_t *__restrict__ mask, const T *__restrict__ Wn, const T *Wprev, T *Wout,
    const T *__restrict__ F, const T *__restrict__ Wt, double *__restrict__ V, Tab3 tab, int n,
    double fs) {
  const Tile3 tl = tiles[blockIdx.x];
  const Grid3Dev &Gg = grids[tl.grid];
  const int n0 = Gg.n0, n1 = Gg.n1, n2 = Gg.n2;
  const int i = tl.i0 + threadIdx.x, j = tl.j0 + threadIdx.y;
  if (i >= n0 || j >= n1) return;
  const bool first = n == 0;
  const double wfn = tab.wf[n + 1];
  const T fcn = first ? fsel<T>(tab.dt2h, tab.dt2hf) : fsel<T>(tab.fc[n], tab.fcf[n]);
  const T fsT = (T)fs;
  const int kend = min(tl.k0 + kTZ, n2);
  const int stencil = Gg.stencil, per = Gg.per;
  const int64_t e0 = Gg.e0, pl = (int64_t)Gg.e0 * Gg.e1;
  if (stencil == kConst7 && per == 0) {
    // constant weights, no wrap: a register queue of W^n along axis 2, and the next plane's
    // loads issued before this plane's arithmetic (more bytes in flight per warp)
    const T c0 = fsel<T>(Gg.cw[0], Gg.cwf[0]), c1 = fsel<T>(Gg.cw[1], Gg.cwf[1]),
            c2 = fsel<T>(Gg.cw[2], Gg.cwf[2]), c3 = fsel<T>(Gg.cw[3], Gg.cwf[3]);
    if constexpr (sizeof(T) == 4) {
      // FP32 (latency-bound): the next plane's x/y neighbours are prefetched too
      int64_t q = at3(Gg, i, j, tl.k0);
      T wm = Wn[q - pl], wc = Wn[q], wp = Wn[q + pl];
      T sx = __fadd_rn(Wn[q - 1], Wn[q + 1]), sy = __fadd_rn(Wn[q - e0], Wn[q + e0]);
      int8_t mk = mask[q];
      T fq = F[q], wo = first ? (T)0 : Wprev[q];
      double vq = V[q];
      const float fcs = fcn * fsT;
      for (int k = tl.k0; k < kend; ++k, q += pl) {
        T wp2 = (T)0, fq2 = (T)0, wo2 = (T)0, xm2 = (T)0, xp2 = (T)0, ym2 = (T)0, yp2 = (T)0;
        int8_t mk2 = 0;
        double vq2 = 0.0;
        if (k + 1 < kend) {  // plane k + 2 is at most the ghost plane n2
          const int64_t q1 = q + pl;
          wp2 = Wn[q1 + pl];
          xm2 = Wn[q1 - 1];
          xp2 = Wn[q1 + 1];
          ym2 = Wn[q1 - e0];
          yp2 = Wn[q1 + e0];
          mk2 = mask[q1];
          fq2 = F[q1];
          if (!first) wo2 = Wprev[q1];
          vq2 = V[q1];
        }
        if (mk == kDisc) {
          float out;
          if (first) {
            const T S = c0 * wc + c1 * sx + c2 * sy + c3 * (wm + wp);
            out = (T)0.5 * S - fcs * fq;
          } else {
            out = step7f(c0, c1, c2, c3, wc, sx, sy, __fadd_rn(wm, wp), wo, fcs, fq);
          }
          Wout[q] = out;
          V[q] = fma(wfn, wh::to_f64(out), vq);
        }
        wm = wc;
        wc = wp;
        wp = wp2;
        sx = __fadd_rn(xm2, xp2);
        sy = __fadd_rn(ym2, yp2);
        mk = mk2;
        fq = fq2;
        wo = wo2;
        vq = vq2;
      }
    } else {
      // FP64 (FP64-pipe bound): neighbours loaded in place (the extra registers of
      // their prefetch measured 1.6% slower here, 10% faster in FP32)
      int64_t q = at3(Gg, i, j, tl.k0);
      T wm = Wn[q - pl], wc = Wn[q], wp = Wn[q + pl];
      int8_t mk = mask[q];
      T fq = F[q], wo = first ? (T)0 : Wprev[q];
      double vq = V[q];
      for (int k = tl.k0; k < kend; ++k, q += pl) {
        T wp2 = (T)0, fq2 = (T)0, wo2 = (T)0;
        int8_t mk2 = 0;
        double vq2 = 0.0;
        if (k + 1 < kend) {  // plane k + 2 is at most the ghost plane n2
          wp2 = Wn[q + 2 * pl];
          mk2 = mask[q + pl];
          fq2 = F[q + pl];
          if (!first) wo2 = Wprev[q + pl];
          vq2 = V[q + pl];
        }
        if (mk == kDisc) {
          const T S = c0 * wc + c1 * (Wn[q - 1] + Wn[q + 1]) + c2 * (Wn[q - e0] + Wn[q + e0]) +
                      c3 * (wm + wp);
          const T out = first ? (T)0.5 * S - fcn * fsT * fq : S - wo - fcn * fsT * fq;
          Wout[q] = out;
          V[q] = vq + wfn * (double)out;
        }
        wm = wc;
        wc = wp;
        wp = wp2;
        mk = mk2;
        fq = fq2;
        wo = wo2;
        vq = vq2;
      }
    }
    return;
  }
  const Grid3Dev G = Gg;
  const int64_t E = G.ext;
  // neighbour offsets of this column: wraps on periodic axes 0 and 1 are fixed per column,
  // on a periodic axis 2 they depend on the plane (at3 is linear in each index, so the
  // offset of a diagonal neighbour is the sum of its axis offsets)
  const int64_t oxm = (per & 1) && i == 0 ? (int64_t)(n0 - 1) : -1;
  const int64_t oxp = (per & 1) && i == n0 - 1 ? -(int64_t)(n0 - 1) : 1;
  const int64_t oym = (per & 2) && j == 0 ? (int64_t)(n1 - 1) * e0 : -e0;
  const int64_t oyp = (per & 2) && j == n1 - 1 ? -(int64_t)(n1 - 1) * e0 : e0;
  const int64_t q0 = at3(G, i, j, tl.k0);
  for (int k = tl.k0; k < kend; ++k) {
    const int64_t q = q0 + (int64_t)(k - tl.k0) * pl;
    if (mask[q] != kDisc) continue;
    const int64_t ozm = (per & 4) && k == 0 ? (int64_t)(n2 - 1) * pl : -pl;
    const int64_t ozp = (per & 4) && k == n2 - 1 ? -(int64_t)(n2 - 1) * pl : pl;
    const int64_t xm = q + oxm, xp = q + oxp, ym = q + oym, yp = q + oyp, zm = q + ozm,
                  zp = q + ozp;
    T S;
    if (stencil == kConst7) {
      S = fsel<T>(G.cw[0], G.cwf[0]) * Wn[q] + fsel<T>(G.cw[1], G.cwf[1]) * (Wn[xm] + Wn[xp]) +
          fsel<T>(G.cw[2], G.cwf[2]) * (Wn[ym] + Wn[yp]) +
          fsel<T>(G.cw[3], G.cwf[3]) * (Wn[zm] + Wn[zp]);
    } else {
      const T *w = Wt + G.wbase + (q - G.base);
      S = w[0] * Wn[q] + w[E] * Wn[xm] + w[2 * E] * Wn[xp] + w[3 * E] * Wn[ym] +
          w[4 * E] * Wn[yp] + w[5 * E] * Wn[zm] + w[6 * E] * Wn[zp];
      if (stencil == kPoint19) {
        // edges of pairs (x,y), (x,z), (y,z): (-,-) (+,-) (-,+) (+,+)
        S += w[7 * E] * Wn[q + oxm + oym] + w[8 * E] * Wn[q + oxp + oym] +
             w[9 * E] * Wn[q + oxm + oyp] + w[10 * E] * Wn[q + oxp + oyp];
        S += w[11 * E] * Wn[q + oxm + ozm] + w[12 * E] * Wn[q + oxp + ozm] +
             w[13 * E] * Wn[q + oxm + ozp] + w[14 * E] * Wn[q + oxp + ozp];
        S += w[15 * E] * Wn[q + oym + ozm] + w[16 * E] * Wn[q + oyp + ozm] +
             w[17 * E] * Wn[q + oym + ozp] + w[18 * E] * Wn[q + oyp + ozp];
      }
    }
    const T out = first ? (T)0.5 * S - fcn * fsT * F[q] : S - Wprev[q] - fcn * fsT * F[q];
    Wout[q] = out;
    V[q] += wfn * (double)out;
  }
}

// cp.async (the asynchronous global -> shared copy): `bytes` (4 or 8) from src to the shared
// address dst, or zeros when src_bytes is 0 (src is then not read); groups committed per
// pipeline stage and awaited with wait_group.
__device__ __forceinline__ void cp_async(void *dst, const void *src, int bytes, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (bytes == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src),
                 "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Temporally blocked FP32 march: K steps n -> n + K over one Unit3 per block, from the
// levels n - 1 and n in the ring (2.5D overlapped tiling).  Thread (tx, ty) owns the column
// (x, y) = (i0 - K + tx, j0 - K + ty) of the unit's box widened by a K-point halo and
// streams it along axis 2: in iteration it it takes level n at plane p_0 = k0 - K + it and
// computes level s at plane p_s = p_0 - s (s = 1..K), where level s exists on the box
// shrunk by K - s points in every direction (columns further out carry the level below,
// which no computed point reads).
//   Inputs arrive through a ring of kStages shared-memory planes filled by cp.async
// kAhead iterations early: level n and FM at p_0, level n - 1 and (own columns) V at p_1.
// FM is the FP32 forcing at discretization points and NaN elsewhere, so one array gives
// both the forcing and the point class.  Level 0's axis-0/1 neighbours are read from the
// previous stage's plane; levels 1..K-1 keep a double-buffered shared plane each, written
// in one iteration and read in the next, so one __syncthreads per plane suffices.  Per
// level a register queue holds the planes p - 1, p, p + 1 (the axis-2 neighbours).
//   Points that are not discretization points are constant in time here (Dirichlet
// values, unused points); the unit's dilated box holds no receiver and no rewritten ghost
// (checked on the host).  Own points accumulate their K filter terms in registers (V read
// and written once) and write levels n + K - 1 and n + K (every level with the export
// flag).  The update is step7f, as in march3_kernel, so the results are the same bits.
constexpr int kAhead = 2, kStages = kAhead + 2;
template <int K>
struct BlockSmem {
  static constexpr int BX = kTX + 2 * K, BY = kUY + 2 * K, P = BX * BY;
  float wn[kStages][P];   // level n at p_0 of the stage
  float fm[kStages][P];   // FM at p_0
  float wm[kStages][P];   // level n - 1 at p_1
  double v[kStages][P];   // V at p_1 (own columns)
  float lev[2][K > 1 ? K - 1 : 1][P];  // levels 1..K-1, double-buffered
  float fc[K + 1];
  double wf[K + 1];
  int roff[K + 1];        // ring offset of level n + s (the ring has < 2^31 elements)
};

template <int K>
size_t block_smem_bytes() { return sizeof(BlockSmem<K>); }

template <int K>
__global__ void __launch_bounds__((kTX + 2 * K) * (kUY + 2 * K), 1) march3_block_kernel(
    const Grid3Dev *__restrict__ grids, const Unit3 *__restrict__ units, float *ring,
    int64_t stride, int L, const float *__restrict__ FM, double *__restrict__ V, Tab3 tab,
    int n, float fs) {
  using SM = BlockSmem<K>;
  constexpr int BX = SM::BX;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &S = *reinterpret_cast<SM *>(smem_raw);
  const Unit3 u = units[blockIdx.x];
  const Grid3Dev &G = grids[u.grid];
  const int tx = threadIdx.x, ty = threadIdx.y, to = ty * BX + tx;
  if (ty == 0 && tx >= 1 && tx <= K) {
    S.fc[tx] = tab.fcf[n + tx - 1] * fs;  // forcing factor of the step to level n + tx
    S.wf[tx] = tab.wf[n + tx];            // filter weight of level n + tx
    S.roff[tx] = (int)(((n + tx) % L) * stride);
  }
  const int x = u.i0 - K + tx, y = u.j0 - K + ty;
  const int dxy = max(max(max(u.i0 - x, x - (u.i0 + kTX - 1)),
                          max(u.j0 - y, y - (u.j0 + kUY - 1))), 0);
  const bool col_ok = x >= -G.g0 && x < G.n0 + G.g0 && y >= -G.g1 && y < G.n1 + G.g1;
  const bool own = dxy == 0 && x < G.n0 && y < G.n1;
  const bool exp_all = (u.flags & 1) != 0;
  // bit s: level s exists in this column (the box shrunk by K - s points)
  unsigned actb = 0u;
#pragma unroll
  for (int s = 1; s <= K; ++s) actb |= (dxy <= K - s ? 1u : 0u) << s;
  // 32-bit element indices: the host enables blocking only when the whole ring has fewer
  // than 2^31 elements
  const int pl = G.e0 * G.e1;
  // element (x, y, z) of the grid's extended array is at col + z * pl
  const int col = (int)G.base + (G.g2 * G.e1 + (y + G.g1)) * G.e0 + (x + G.g0);
  const int gbase = (int)G.base;
  const float c0 = G.cwf[0], c1 = G.cwf[1], c2 = G.cwf[2], c3 = G.cwf[3];
  const float *Wn = ring + (int64_t)(n % L) * stride;
  const float *Wm = ring + (int64_t)((n - 1) % L) * stride;
  const int zlo = -G.g2, zhi = G.n2 + G.g2;  // extended planes
  const int nz = u.nz, iters = nz + 2 * K;
  // stage `it`: level n and FM at p_0, level n - 1 and V at p_1 (zeros outside the array)
  int isl = 0;                                   // stage slot of the next issue
  int iq0 = col + (u.k0 - K) * pl;  // element at the next issue's p_0
  int ip0 = u.k0 - K;
  auto issue = [&]() {
    const int p0 = ip0, p1 = p0 - 1;
    const bool z0 = col_ok && p0 >= zlo && p0 < zhi;
    const bool z1 = col_ok && dxy < K && p1 >= zlo && p1 < zhi;
    const int q0 = z0 ? iq0 : gbase, q1 = z1 ? iq0 - pl : gbase;
    cp_async(&S.wn[isl][to], Wn + q0, 4, z0 ? 4 : 0);
    cp_async(&S.fm[isl][to], FM + q0, 4, z0 ? 4 : 0);
    cp_async(&S.wm[isl][to], Wm + q1, 4, z1 ? 4 : 0);
    const bool v1 = own && p1 >= u.k0 && p1 < u.k0 + nz;
    cp_async(&S.v[isl][to], V + (v1 ? q1 : gbase), 8, v1 ? 8 : 0);
    isl = isl + 1 == kStages ? 0 : isl + 1;
    iq0 += pl;
    ++ip0;
  };
#pragma unroll
  for (int a = 0; a < kAhead; ++a) {
    if (a < iters) issue();
    cp_async_commit();
  }
  float q[K][3];
  float fq[K + 1];
  double acc[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    q[j][0] = q[j][1] = q[j][2] = 0.0f;
    acc[j] = 0.0;
  }
#pragma unroll
  for (int j = 0; j <= K; ++j) fq[j] = 0.0f;
  unsigned mbits = 0u;
  int sl = 0, sp = kStages - 1;  // stage slots of this iteration and the previous one
  int cur = 0;                   // level buffer written this iteration
  int qz = col + (u.k0 - K) * pl;  // element at p_0
  int p0 = u.k0 - K;
  for (int it = 0; it < iters; ++it) {
    cp_async_wait<kAhead - 1>();  // this thread's copies of stage it have landed
    __syncthreads();              // everyone's; and last iteration's shared reads are done
    if (it + kAhead < iters) issue();
    cp_async_commit();
    const bool z0 = col_ok && p0 >= zlo && p0 < zhi;
    const float w0 = S.wn[sl][to], fm = S.fm[sl][to];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      q[j][0] = q[j][1];
      q[j][1] = q[j][2];
    }
#pragma unroll
    for (int j = K; j >= 1; --j) fq[j] = fq[j - 1];
#pragma unroll
    for (int j = K - 1; j >= 1; --j) acc[j] = acc[j - 1];
    fq[0] = fm;
    mbits = (mbits << 1) | ((z0 && !isnan(fm)) ? 1u : 0u);
    // own planes: level s is at plane p_0 - s, own when it - K - s is in [0, nz)
    acc[0] = (own && (mbits & 2u) && (unsigned)(it - K - 1) < (unsigned)nz) ? S.v[sl][to] : 0.0;
    q[0][2] = w0;
    const unsigned lv = mbits & actb;
    const float *lprv = &S.lev[cur ^ 1][0][0];
    float *lcur = &S.lev[cur][0][0];
#pragma unroll
    for (int s = 1; s <= K; ++s) {
      float out = q[s - 1][1];
      if ((lv >> s) & 1u) {
        // neighbours along axes 0 and 1 of level s - 1 at plane p_s: level 0 from the
        // previous stage's plane, higher levels from last iteration's level buffer
        const float *pl_prev = s == 1 ? &S.wn[sp][0] : lprv + (s >= 2 ? s - 2 : 0) * SM::P;
        const float xm = pl_prev[to - 1], xp = pl_prev[to + 1];
        const float ym = pl_prev[to - BX], yp = pl_prev[to + BX];
        const float wo = s == 1 ? S.wm[sl][to] : q[s >= 2 ? s - 2 : 0][0];
        out = step7f(c0, c1, c2, c3, q[s - 1][1], __fadd_rn(xm, xp), __fadd_rn(ym, yp),
                     __fadd_rn(q[s - 1][0], q[s - 1][2]), wo, S.fc[s], fq[s]);
        if (own && (unsigned)(it - K - s) < (unsigned)nz) {
          const int qs = qz - s * pl;
          acc[s - 1] = fma(S.wf[s], wh::to_f64(out), acc[s - 1]);
          if (exp_all || s >= K - 1) ring[S.roff[s] + qs] = out;
          if (s == K) V[qs] = acc[K - 1];
        }
      }
      if (s < K) {
        q[s < K ? s : 0][2] = out;
        lcur[(s >= 1 && s < K ? s - 1 : 0) * SM::P + to] = out;
      }
    }
    sp = sl;
    sl = sl + 1 == kStages ? 0 : sl + 1;
    cur ^= 1;
    qz += pl;
    ++p0;
  }
  cp_async_wait<0>();
}

// Ghost rules and interpolation of one time level, one thread per receiver: the 27 donors
// (i0 + a, j0 + b, k0 + c) at gbase + ox[a] + oy[b] + oz[c] (per-axis offsets, periodic wrap
// resolved at set-up) are all loaded first, then the tensor product is evaluated as rows
// sum_a wx[a] u, columns sum_b wy[b] row_b, and sum_c wz[c] col_c: 39 FP64 operations per
// receiver.  Metadata are planes of nrecv entries (goff[t * nrecv + r], gw[t * nrecv + r],
// t = 0..8: x, y, z), read coalesced.  The receiver's filter term is added as it is written.
// Every thread then copies Neumann ghosts (gdst <- gsrc).  Donors and ghost sources are
// discretization or Dirichlet points, so the two parts read nothing the other writes.
template <typename T>
__global__ void __launch_bounds__(256) gather3_kernel(
    int64_t nrecv, int64_t nghost, const int64_t *__restrict__ ridx,
    const int32_t *__restrict__ gbase, const int32_t *__restrict__ goff,
    const double *__restrict__ gw, const int32_t *__restrict__ gdst,
    const int32_t *__restrict__ gsrc, T *W, double *V, const double *__restrict__ wf,
    int level) {
  const double wl = wf[level];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrecv; r += stride) {
    int32_t o[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) o[t] = goff[t * nrecv + r];
    const int64_t b0 = gbase[r];
    T u[27];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a) u[9 * c + 3 * b + a] = W[b0 + o[a] + o[3 + b] + o[6 + c]];
    double w[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) w[t] = gw[t * nrecv + r];
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double col = 0.0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T *x = u + 9 * c + 3 * b;
        const double row = w[0] * wh::to_f64(x[0]) + w[1] * wh::to_f64(x[1]) + w[2] * wh::to_f64(x[2]);
        col = fma(w[3 + b], row, col);
      }
      s = fma(w[6 + c], col, s);
    }
    const T v = (T)s;
    const int64_t q = ridx[r];
    W[q] = v;
    V[q] += wl * wh::to_f64(v);
  }
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < nghost; g += stride)
    W[gdst[g]] = W[gsrc[g]];
}

// Dirichlet points with boundary data at one level: W = gfac g (gfac = the forcing switch
// times cos(omega_e t^level)) and the level's filter term.  Runs before the level's ghost
// rules and interpolation, which may read these points as donors.
template <typename T>
__global__ void dirichlet3_kernel(int64_t n, const int64_t *__restrict__ idx,
                                  const double *__restrict__ g, T *W, double *V, double gfac,
                                  const double *__restrict__ wf, int level) {
  const double wl = wf[level];
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = idx[t];
    const T w = (T)(gfac * g[t]);
    W[q] = w;
    V[q] = fma(wl, wh::to_f64(w), V[q]);
  }
}

// v_out (compact) = V at every point of every grid (with `mask`: at discretization points,
// zero elsewhere); blockIdx.y = grid.
__global__ void finish3_kernel(const Grid3Dev *grids, const int8_t *mask, const double *V,
                               double *vout) {
  const Grid3Dev G = grids[blockIdx.y];
  const int64_t npts = (int64_t)G.n0 * G.n1 * G.n2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % G.n0), j = (int)((t / G.n0) % G.n1), k = (int)(t / ((int64_t)G.n0 * G.n1));
    const int64_t q = at3(G, i, j, k);
    vout[G.cbase + t] = (!mask || mask[q] == kDisc) ? V[q] : 0.0;
  }
}

template <typename T>
__global__ void convert_kernel(const double *src, T *dst, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = (T)src[t];
}

// ------------------------------------------------------- fourth order (Cartesian grids)

// Per-point weights of a kPoint13 grid with dt^2 c(x)^2 folded in: the second difference
// D+D-(1 - h^2/12 D+D-) = (-W_-2 + 16 W_-1 - 30 W + 16 W_+1 - W_+2) / (12 h^2) per axis
// (Eq. SecondDerivOrderp, mu < 2), so with x_a = dt^2 c^2 / h_a^2 the centre (with the "2"
// of the leapfrog) is 2 - (30/12) sum_a x_a, the +-1 neighbours (16/12) x_a and the +-2
// neighbours -(1/12) x_a.
template <typename T>
__global__ void weight3o4_kernel(const Grid3Dev *grids, int gidx, const int8_t *mask,
                                 const double *c2, T *Wt, double dt2) {
  const Grid3Dev G = grids[gidx];
  const int64_t npts = (int64_t)G.n0 * G.n1 * G.n2;
  const int64_t E = G.ext;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npts;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t % G.n0), j = (int)((t / G.n0) % G.n1), k = (int)(t / ((int64_t)G.n0 * G.n1));
    const int64_t q = at3(G, i, j, k), ql = q - G.base;
    if (mask[q] != kDisc) continue;
    T *W = Wt + G.wbase + ql;
    double centre = 2.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double x = dt2 * c2[q] / (G.h[a] * G.h[a]);
      centre -= 2.5 * x;
      W[(1 + 4 * a) * E] = W[(2 + 4 * a) * E] = (T)(x * (16.0 / 12.0));
      W[(3 + 4 * a) * E] = W[(4 + 4 * a) * E] = (T)(-x / 12.0);
    }
    W[0] = (T)centre;
  }
}

// One step n -> n + 1 of the fourth-order march (Eq. WaveSchemeexplicit with the 13-point
// Laplacian above) with the fused filter term of level n + 1.  Block = one Tile3; each
// thread marches kTZ points along axis 2.  The +-1 and +-2 neighbours wrap on periodic axes
// and reach the two ghost layers on the others.  W^{n+1} overwrites W^{n-1} in place.
template <typename T>
__global__ void __launch_bounds__(kTX *kTY) march3o4_kernel(
    const Grid3Dev *__restrict__ grids, const Tile3 *__restrict__ tiles,
    const int8_t *__restrict__ mask, const T *__restrict__ Wn, const T *Wprev, T *Wout,
    const T *__restrict__ F, const T *__restrict__ Wt, double *__restrict__ V, Tab3 tab, int n,
    double fs) {
  const Tile3 tl = tiles[blockIdx.x];
  const Grid3Dev &G = grids[tl.grid];
  const int i = tl.i0 + threadIdx.x, j = tl.j0 + threadIdx.y;
  if (i >= G.n0 || j >= G.n1) return;
  const bool first = n == 0;
  const double wfn = tab.wf[n + 1];
  const T fcn = first ? fsel<T>(tab.dt2h, tab.dt2hf) : fsel<T>(tab.fc[n], tab.fcf[n]);
  const T fsT = (T)fs;
  const int kend = min(tl.k0 + kTZ, G.n2);
  const int64_t e0 = G.e0, pl = (int64_t)G.e0 * G.e1, E = G.ext;
  const int dd[4] = {-1, 1, -2, 2};
  int64_t ox[4], oy[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    ox[t] = (int64_t)(wrap(i + dd[t], G.n0, G.per & 1) - i);
    oy[t] = (int64_t)(wrap(j + dd[t], G.n1, G.per & 2) - j) * e0;
  }
  const bool cst = G.stencil == kConst13;
  if constexpr (sizeof(T) == 4) {
    if (cst && G.per == 0) {
      // FP32, constant weights, no periodic axis (two ghost layers everywhere): a register
      // queue of W^n at planes k - 2 .. k + 2, and the next plane's loads issued before
      // this plane's arithmetic.  Every load stays in the extended array: planes -2 .. n2 + 1
      // (the prefetched plane k + 3 only while k + 1 < kend <= n2), columns i - 2 .. i + 2.
      const float c0 = G.cwf[0], c1x = G.cwf[1], c2x = G.cwf[2], c1y = G.cwf[3],
                  c2y = G.cwf[4], c1z = G.cwf[5], c2z = G.cwf[6];
      const float fcs = fcn * fsT;
      int64_t q = at3(G, i, j, tl.k0);
      float wm2 = Wn[q - 2 * pl], wm = Wn[q - pl], wc = Wn[q], wp = Wn[q + pl],
            wp2 = Wn[q + 2 * pl];
      float sx1 = Wn[q - 1] + Wn[q + 1], sx2 = Wn[q - 2] + Wn[q + 2];
      float sy1 = Wn[q - e0] + Wn[q + e0], sy2 = Wn[q - 2 * e0] + Wn[q + 2 * e0];
      int8_t mk = mask[q];
      float fq = F[q], wo = first ? 0.0f : Wprev[q];
      double vq = V[q];
      for (int k = tl.k0; k < kend; ++k, q += pl) {
        float wp3 = 0.0f, nx1 = 0.0f, nx2 = 0.0f, ny1 = 0.0f, ny2 = 0.0f, fq2 = 0.0f,
              wo2 = 0.0f;
        int8_t mk2 = 0;
        double vq2 = 0.0;
        if (k + 1 < kend) {
          const int64_t q1 = q + pl;
          wp3 = Wn[q1 + 2 * pl];
          nx1 = Wn[q1 - 1] + Wn[q1 + 1];
          nx2 = Wn[q1 - 2] + Wn[q1 + 2];
          ny1 = Wn[q1 - e0] + Wn[q1 + e0];
          ny2 = Wn[q1 - 2 * e0] + Wn[q1 + 2 * e0];
          mk2 = mask[q1];
          fq2 = F[q1];
          if (!first) wo2 = Wprev[q1];
          vq2 = V[q1];
        }
        if (mk == kDisc) {
          const float S = c0 * wc + c1x * sx1 + c2x * sx2 + c1y * sy1 + c2y * sy2 +
                          c1z * (wm + wp) + c2z * (wm2 + wp2);
          const float out = first ? 0.5f * S - fcs * fq : S - wo - fcs * fq;
          Wout[q] = out;
          V[q] = fma(wfn, wh::to_f64(out), vq);
        }
        wm2 = wm;
        wm = wc;
        wc = wp;
        wp = wp2;
        wp2 = wp3;
        sx1 = nx1;
        sx2 = nx2;
        sy1 = ny1;
        sy2 = ny2;
        mk = mk2;
        fq = fq2;
        wo = wo2;
        vq = vq2;
      }
      return;
    }
  }
  T cw[7];
#pragma unroll
  for (int t = 0; t < 7; ++t) cw[t] = fsel<T>(G.cw[t], G.cwf[t]);
  for (int k = tl.k0; k < kend; ++k) {
    const int64_t q = at3(G, i, j, k);
    if (mask[q] != kDisc) continue;
    int64_t oz[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) oz[t] = (int64_t)(wrap(k + dd[t], G.n2, G.per & 4) - k) * pl;
    T S;
    if (cst) {
      S = cw[0] * Wn[q] + cw[1] * (Wn[q + ox[0]] + Wn[q + ox[1]]) +
          cw[2] * (Wn[q + ox[2]] + Wn[q + ox[3]]) + cw[3] * (Wn[q + oy[0]] + Wn[q + oy[1]]) +
          cw[4] * (Wn[q + oy[2]] + Wn[q + oy[3]]) + cw[5] * (Wn[q + oz[0]] + Wn[q + oz[1]]) +
          cw[6] * (Wn[q + oz[2]] + Wn[q + oz[3]]);
    } else {
      const T *w = Wt + G.wbase + (q - G.base);
      S = w[0] * Wn[q];
#pragma unroll
      for (int t = 0; t < 4; ++t)
        S += w[(1 + t) * E] * Wn[q + ox[t]] + w[(5 + t) * E] * Wn[q + oy[t]] +
             w[(9 + t) * E] * Wn[q + oz[t]];
    }
    const T out = first ? (T)0.5 * S - fcn * fsT * F[q] : S - Wprev[q] - fcn * fsT * F[q];
    Wout[q] = out;
    V[q] += wfn * wh::to_f64(out);
  }
}

// The ghost rules and the interpolation of one level at fourth order (Algorithm 2: after
// every grid has advanced).  Receivers: the width-5 tensor product evaluated axis by axis,
// one thread per receiver, with the receiver's filter term.  Ghost items: per boundary point
// of a Dirichlet or Neumann face the two ghosts from a 2 x 2 solve of
//   row 1, Dirichlet: c^2 (-G2 + 16 G1 - 30 U0 + 16 U1 - U2) / (12 h^2) = fcl f_b
//          (the scheme at the boundary point, where W stays 0);
//          Neumann: the centred fourth-order normal derivative 8 (U1 - G1) - (U2 - G2) = 0;
//   row 2: the extrapolation D+^5 G2 = G2 - 5 G1 + 10 U0 - 10 U1 + 5 U2 - U3 = 0,
// in FP64 from the level's values.  Donors and the points the rules read are discretization
// or Dirichlet points (the host checks both), so neither part reads what the other writes.
template <typename T>
__global__ void __launch_bounds__(256) gather3o4_kernel(
    int64_t nrecv, int64_t nitems, const int64_t *__restrict__ ridx,
    const int32_t *__restrict__ gbase, const int32_t *__restrict__ goff,
    const double *__restrict__ gw, const Ghost4 *__restrict__ items,
    const double *__restrict__ F, double fcl, T *W, double *V, const double *__restrict__ wf,
    int level) {
  const double wl = wf[level];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrecv; r += stride) {
    int32_t o[15];
    double w[15];
#pragma unroll
    for (int t = 0; t < 15; ++t) {
      o[t] = goff[t * nrecv + r];
      w[t] = gw[t * nrecv + r];
    }
    const int64_t b0 = gbase[r];
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      double col = 0.0;
#pragma unroll
      for (int b = 0; b < 5; ++b) {
        const T *x = W + b0 + o[5 + b] + o[10 + c];
        double row = 0.0;
#pragma unroll
        for (int a = 0; a < 5; ++a) row = fma(w[a], wh::to_f64(x[o[a]]), row);
        col = fma(w[5 + b], row, col);
      }
      s = fma(w[10 + c], col, s);
    }
    const T v = (T)s;
    const int64_t q = ridx[r];
    W[q] = v;
    V[q] += wl * wh::to_f64(v);
  }
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nitems; t += stride) {
    const Ghost4 it = items[t];
    double U[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) U[k] = wh::to_f64(W[it.q0 + k * it.s]);
    const double a10 = -5.0, a11 = 1.0;
    const double r1 = -(10.0 * U[0] - 10.0 * U[1] + 5.0 * U[2] - U[3]);
    double a00, a01, r0;
    if (it.a2 == 0.0) {
      a00 = -8.0;
      a01 = 1.0;
      r0 = -(8.0 * U[1] - U[2]);
    } else {
      a00 = 16.0 * it.a2;
      a01 = -it.a2;
      r0 = fcl * F[it.q0] - it.a2 * (-30.0 * U[0] + 16.0 * U[1] - U[2]);
    }
    const double det = a00 * a11 - a01 * a10;
    W[it.q0 - it.s] = (T)((r0 * a11 - a01 * r1) / det);
    W[it.q0 - 2 * it.s] = (T)((a00 * r1 - r0 * a10) / det);
  }
}

unsigned blocks_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

void launch_dirichlet3(bool fp32, cudaStream_t s, int64_t n, const int64_t *idx,
                       const double *g, void *W, double *V, double gfac, const double *wf,
                       int level) {
  const unsigned nb = blocks_for(n < 1 ? 1 : n, 256);
  if (fp32)
    dirichlet3_kernel<float><<<nb, 256, 0, s>>>(n, idx, g, (float *)W, V, gfac, wf, level);
  else
    dirichlet3_kernel<double><<<nb, 256, 0, s>>>(n, idx, g, (double *)W, V, gfac, wf, level);
}


void launch_coef3(cudaStream_t s, const Grid3Dev *grids, int gidx, const Grid3Dev &G,
                  const int8_t *mask, const double *rx, const double *c2, double *coef,
                  unsigned long long *smax) {
  const int64_t n = (int64_t)G.n0 * G.n1 * G.n2;
  coef3_kernel<<<blocks_for(n, 256), 256, 0, s>>>(grids, gidx, mask, rx, c2, coef, smax);
}

void launch_weight3(bool fp32, cudaStream_t s, const Grid3Dev *grids, int gidx,
                    const Grid3Dev &G, const int8_t *mask, const double *coef, const double *c2,
                    void *Wt, double dt2) {
  const int64_t n = (int64_t)G.n0 * G.n1 * G.n2;
  if (fp32)
    weight3_kernel<float><<<blocks_for(n, 256), 256, 0, s>>>(grids, gidx, mask, coef, c2,
                                                             (float *)Wt, dt2);
  else
    weight3_kernel<double><<<blocks_for(n, 256), 256, 0, s>>>(grids, gidx, mask, coef, c2,
                                                              (double *)Wt, dt2);
}

void launch_init3(bool fp32, cudaStream_t s, const Grid3Dev *grids, int ngrids,
                  int64_t max_ext, const int8_t *mask, const double *v, void *W0, double *V,
                  const double *wf) {
  dim3 gb(blocks_for(max_ext, 256), ngrids);
  if (fp32)
    init3_kernel<float><<<gb, 256, 0, s>>>(grids, mask, v, (float *)W0, V, wf);
  else
    init3_kernel<double><<<gb, 256, 0, s>>>(grids, mask, v, (double *)W0, V, wf);
}

void launch_march3(bool fp32, cudaStream_t s, int ntiles, const Grid3Dev *grids,
                   const Tile3 *tiles, const int8_t *mask, const void *Wn, const void *Wprev,
                   void *Wout, const void *F, const void *Wt, double *V, Tab3 tab, int n,
                   double fs) {
  if (ntiles < 1) return;
  dim3 tb(kTX, kTY);
  if (fp32)
    march3_kernel<float><<<ntiles, tb, 0, s>>>(grids, tiles, mask, (const float *)Wn,
                                               (const float *)Wprev, (float *)Wout,
                                               (const float *)F, (const float *)Wt, V, tab, n,
                                               fs);
  else
    march3_kernel<double><<<ntiles, tb, 0, s>>>(grids, tiles, mask, (const double *)Wn,
                                                (const double *)Wprev, (double *)Wout,
                                                (const double *)F, (const double *)Wt, V, tab,
                                                n, fs);
}

size_t march3_block_threads(int K) { return (size_t)(kTX + 2 * K) * (kUY + 2 * K); }

template <int K>
void launch_block_k(cudaStream_t s, int nunits, const Grid3Dev *grids, const Unit3 *units,
                    float *ring, int64_t stride, int L, const float *FM, double *V, Tab3 tab,
                    int n, float fs) {
  static bool attr = false;  // opt in to more than 48 KiB of dynamic shared memory once
  const size_t bytes = block_smem_bytes<K>();
  if (!attr) {
    cudaFuncSetAttribute(march3_block_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)bytes);
    attr = true;
  }
  march3_block_kernel<K><<<nunits, dim3(kTX + 2 * K, kUY + 2 * K), bytes, s>>>(
      grids, units, ring, stride, L, FM, V, tab, n, fs);
}

void launch_march3_block(int K, cudaStream_t s, int nunits, const Grid3Dev *grids,
                         const Unit3 *units, const float *FM, float *ring, int64_t stride,
                         int L, double *V, Tab3 tab, int n, double fs) {
  if (nunits < 1) return;
  const float f = (float)fs;
  switch (K) {
    case 2: launch_block_k<2>(s, nunits, grids, units, ring, stride, L, FM, V, tab, n, f); break;
    case 3: launch_block_k<3>(s, nunits, grids, units, ring, stride, L, FM, V, tab, n, f); break;
    default: launch_block_k<4>(s, nunits, grids, units, ring, stride, L, FM, V, tab, n, f); break;
  }
}

// FM = the FP32 forcing at discretization points, NaN elsewhere (the blocked march's input).
__global__ void forcing_mask_kernel(const float *__restrict__ F, const int8_t *__restrict__ mask,
                                    float *__restrict__ FM, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    FM[t] = mask[t] == kDisc ? F[t] : __int_as_float(0x7fc00000);
}

void launch_forcing_mask(cudaStream_t s, const float *F, const int8_t *mask, float *FM,
                         int64_t n) {
  forcing_mask_kernel<<<blocks_for(n, 256), 256, 0, s>>>(F, mask, FM, n);
}

void launch_gather3(bool fp32, cudaStream_t s, int64_t nrecv, int64_t nghost,
                    const int64_t *ridx, const int32_t *gbase, const int32_t *goff,
                    const double *gw, const int32_t *gdst, const int32_t *gsrc, void *W,
                    double *V, const double *wf, int level) {
  const int threads = 256;
  int64_t need = nrecv > nghost ? nrecv : nghost;
  if (need < 1) need = 1;
  const unsigned nb = blocks_for(need, threads);
  if (fp32)
    gather3_kernel<float><<<nb, threads, 0, s>>>(nrecv, nghost, ridx, gbase, goff, gw, gdst,
                                                 gsrc, (float *)W, V, wf, level);
  else
    gather3_kernel<double><<<nb, threads, 0, s>>>(nrecv, nghost, ridx, gbase, goff, gw, gdst,
                                                  gsrc, (double *)W, V, wf, level);
}

void launch_weight3o4(bool fp32, cudaStream_t s, const Grid3Dev *grids, int gidx,
                      const Grid3Dev &G, const int8_t *mask, const double *c2, void *Wt,
                      double dt2) {
  const int64_t n = (int64_t)G.n0 * G.n1 * G.n2;
  if (fp32)
    weight3o4_kernel<float><<<blocks_for(n, 256), 256, 0, s>>>(grids, gidx, mask, c2,
                                                               (float *)Wt, dt2);
  else
    weight3o4_kernel<double><<<blocks_for(n, 256), 256, 0, s>>>(grids, gidx, mask, c2,
                                                                (double *)Wt, dt2);
}

void launch_march3o4(bool fp32, cudaStream_t s, int ntiles, const Grid3Dev *grids,
                     const Tile3 *tiles, const int8_t *mask, const void *Wn, const void *Wprev,
                     void *Wout, const void *F, const void *Wt, double *V, Tab3 tab, int n,
                     double fs) {
  if (ntiles < 1) return;
  dim3 tb(kTX, kTY);
  if (fp32)
    march3o4_kernel<float><<<ntiles, tb, 0, s>>>(grids, tiles, mask, (const float *)Wn,
                                                 (const float *)Wprev, (float *)Wout,
                                                 (const float *)F, (const float *)Wt, V, tab,
                                                 n, fs);
  else
    march3o4_kernel<double><<<ntiles, tb, 0, s>>>(grids, tiles, mask, (const double *)Wn,
                                                  (const double *)Wprev, (double *)Wout,
                                                  (const double *)F, (const double *)Wt, V,
                                                  tab, n, fs);
}

void launch_gather3o4(bool fp32, cudaStream_t s, int64_t nrecv, int64_t nitems,
                      const int64_t *ridx, const int32_t *gbase, const int32_t *goff,
                      const double *gw, const Ghost4 *items, const double *F, double fcl,
                      void *W, double *V, const double *wf, int level) {
  const int threads = 256;
  int64_t need = nrecv > nitems ? nrecv : nitems;
  if (need < 1) need = 1;
  const unsigned nb = blocks_for(need, threads);
  if (fp32)
    gather3o4_kernel<float><<<nb, threads, 0, s>>>(nrecv, nitems, ridx, gbase, goff, gw, items,
                                                   F, fcl, (float *)W, V, wf, level);
  else
    gather3o4_kernel<double><<<nb, threads, 0, s>>>(nrecv, nitems, ridx, gbase, goff, gw, items,
                                                    F, fcl, (double *)W, V, wf, level);
}

void launch_finish3(cudaStream_t s, const Grid3Dev *grids, int ngrids, int64_t max_compact,
                    const double *V, double *vout) {
  dim3 gb(blocks_for(max_compact, 256), ngrids);
  finish3_kernel<<<gb, 256, 0, s>>>(grids, nullptr, V, vout);
}

void launch_disc3(cudaStream_t s, const Grid3Dev *grids, int ngrids, int64_t max_compact,
                  const int8_t *mask, const double *W, double *vout) {
  dim3 gb(blocks_for(max_compact, 256), ngrids);
  finish3_kernel<<<gb, 256, 0, s>>>(grids, mask, W, vout);
}

void launch_to_precision(bool fp32, cudaStream_t s, const double *src, void *dst, int64_t n) {
  if (fp32)
    convert_kernel<float><<<blocks_for(n, 256), 256, 0, s>>>(src, (float *)dst, n);
  else
    convert_kernel<double><<<blocks_for(n, 256), 256, 0, s>>>(src, (double *)dst, n);
}

}  // namespace wh3
