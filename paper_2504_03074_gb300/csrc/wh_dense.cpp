// wh_dense.cpp -- small dense eigenproblems on the host for the Krylov eigensolver
// (wh_eigs): the projected matrices there are at most a few hundred wide, so plain O(m^3)
// host code is enough.
//
// Method (the standard one of numerical linear algebra, written here from its definition):
//   1. Householder reduction of the real matrix to upper Hessenberg form, A = Q H Q^T;
//   2. the QR algorithm on H in complex arithmetic, one implicit shift per sweep (the
//      Wilkinson shift: the eigenvalue of the trailing 2 x 2 block nearer its last diagonal
//      entry, with an exceptional shift every tenth sweep without progress), deflating
//      wherever a subdiagonal entry drops below the working precision; this gives the
//      complex Schur form H = Z T Z^* with T upper triangular;
//   3. the eigenvectors of T by back substitution, mapped back through Q Z.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "wh_internal.h"

namespace wh {
namespace {

using cd = std::complex<double>;
constexpr double kEps = 2.220446049250313e-16;

// A (m x m, row-major) <- Q^T A Q upper Hessenberg; Q (m x m, row-major) accumulated.
void hessenberg(int m, std::vector<double> &A, std::vector<double> &Q) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<double> v(m);
  for (int k = 0; k + 2 < m; ++k) {
    // reflector I - 2 v v^T / (v^T v) zeroing A[k+2.., k]
    double alpha = 0.0;
    for (int i = k + 1; i < m; ++i) alpha += A[(size_t)i * m + k] * A[(size_t)i * m + k];
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = A[(size_t)(k + 1) * m + k];
    if (x0 > 0) alpha = -alpha;
    double vv = 0.0;
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    v[k + 1] = x0 - alpha;
    for (int i = k + 2; i < m; ++i) v[i] = A[(size_t)i * m + k];
    for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // A <- P A (rows k+1..m-1)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int i = k + 1; i < m; ++i) s += v[i] * A[(size_t)i * m + j];
      s *= beta;
      for (int i = k + 1; i < m; ++i) A[(size_t)i * m + j] -= s * v[i];
    }
    // A <- A P (columns k+1..m-1), Q <- Q P
    for (int i = 0; i < m; ++i) {
      double s = 0.0, t = 0.0;
      for (int j = k + 1; j < m; ++j) {
        s += A[(size_t)i * m + j] * v[j];
        t += Q[(size_t)i * m + j] * v[j];
      }
      s *= beta;
      t *= beta;
      for (int j = k + 1; j < m; ++j) {
        A[(size_t)i * m + j] -= s * v[j];
        Q[(size_t)i * m + j] -= t * v[j];
      }
    }
    for (int i = k + 2; i < m; ++i) A[(size_t)i * m + k] = 0.0;
  }
}

// Rotation G = [[c, s], [-conj(s), c]] (c real) with G [a; b] = [r; 0].
void givens(cd a, cd b, double &c, cd &s) {
  const double aa = std::abs(a), bb = std::abs(b);
  if (bb == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  if (aa == 0.0) {
    c = 0.0;
    s = 1.0;
    return;
  }
  const double r = std::hypot(aa, bb);
  c = aa / r;
  s = (a / aa) * std::conj(b) / r;
}

// Complex Schur form of the upper Hessenberg H (m x m, row-major): H <- T = Z^* H Z upper
// triangular, Z <- Z Z_qr (Z enters as the accumulated transform).  False if a sweep limit
// is hit.
bool schur(int m, std::vector<cd> &H, std::vector<cd> &Z) {
  auto h = [&](int i, int j) -> cd & { return H[(size_t)i * m + j]; };
  double anorm = 0.0;
  for (const cd &x : H) anorm = std::max(anorm, std::abs(x));
  if (anorm == 0.0) return true;
  int hi = m - 1, stall = 0;
  long sweeps = 0;
  const long max_sweeps = 60L * m + 100;
  while (hi > 0) {
    // deflation: the lowest l with a negligible subdiagonal entry above the active block
    int l = hi;
    while (l > 0) {
      const double sc = std::abs(h(l, l)) + std::abs(h(l - 1, l - 1));
      if (std::abs(h(l, l - 1)) <= kEps * (sc > 0 ? sc : anorm)) {
        h(l, l - 1) = 0.0;
        break;
      }
      --l;
    }
    if (l == hi) {  // 1 x 1 block converged
      --hi;
      stall = 0;
      continue;
    }
    if (++sweeps > max_sweeps) return false;
    // shift: Wilkinson, or an exceptional one after ten sweeps without deflation
    cd mu;
    if (++stall % 10 == 0) {
      mu = h(hi, hi) + 0.75 * std::abs(h(hi, hi - 1));
    } else {
      const cd a = h(hi - 1, hi - 1), b = h(hi - 1, hi), c = h(hi, hi - 1), d = h(hi, hi);
      const cd tr = 0.5 * (a + d), det = a * d - b * c;
      const cd disc = std::sqrt(tr * tr - det);
      const cd e1 = tr + disc, e2 = tr - disc;
      mu = std::abs(e1 - d) < std::abs(e2 - d) ? e1 : e2;
    }
    // implicit single-shift QR sweep on rows/columns l..hi, bulge chased down
    cd x = h(l, l) - mu, y = h(l + 1, l);
    for (int k = l; k < hi; ++k) {
      double c;
      cd s;
      givens(x, y, c, s);
      // rows k, k+1 (left multiplication by G)
      for (int j = std::max(l, k - 1); j < m; ++j) {
        const cd t1 = h(k, j), t2 = h(k + 1, j);
        h(k, j) = c * t1 + s * t2;
        h(k + 1, j) = -std::conj(s) * t1 + c * t2;
      }
      // columns k, k+1 (right multiplication by G^*), and Z
      const int rmax = std::min(k + 2, hi);
      for (int i = 0; i <= rmax; ++i) {
        const cd t1 = h(i, k), t2 = h(i, k + 1);
        h(i, k) = c * t1 + std::conj(s) * t2;
        h(i, k + 1) = -s * t1 + c * t2;
      }
      for (int i = 0; i < m; ++i) {
        const cd t1 = Z[(size_t)i * m + k], t2 = Z[(size_t)i * m + k + 1];
        Z[(size_t)i * m + k] = c * t1 + std::conj(s) * t2;
        Z[(size_t)i * m + k + 1] = -s * t1 + c * t2;
      }
      if (k + 1 < hi) {
        x = h(k + 1, k);
        y = h(k + 2, k);
      }
    }
  }
  // clean the strictly lower part
  for (int i = 1; i < m; ++i)
    for (int j = 0; j < i; ++j) h(i, j) = 0.0;
  return true;
}

}  // namespace

bool dense_eig(int m, const double *A, std::vector<std::complex<double>> &w,
               std::vector<std::complex<double>> &V) {
  w.assign(m, 0.0);
  V.assign((size_t)m * m, 0.0);
  if (m <= 0) return true;
  std::vector<double> H(A, A + (size_t)m * m), Q;
  hessenberg(m, H, Q);
  std::vector<cd> T(H.begin(), H.end()), Z(Q.begin(), Q.end());
  if (!schur(m, T, Z)) return false;
  double tnorm = 0.0;
  for (const cd &x : T) tnorm = std::max(tnorm, std::abs(x));
  const double small = kEps * (tnorm > 0 ? tnorm : 1.0);
  std::vector<cd> x(m);
  for (int i = 0; i < m; ++i) {
    const cd ti = T[(size_t)i * m + i];
    w[i] = ti;
    // T x = t_ii x with x_i = 1, x_j = 0 for j > i (back substitution upwards)
    for (int j = 0; j < m; ++j) x[j] = 0.0;
    x[i] = 1.0;
    for (int j = i - 1; j >= 0; --j) {
      cd s = 0.0;
      for (int l = j + 1; l <= i; ++l) s += T[(size_t)j * m + l] * x[l];
      cd d = T[(size_t)j * m + j] - ti;
      if (std::abs(d) < small) d = small;  // a repeated eigenvalue: perturb the pivot
      x[j] = -s / d;
    }
    // eigenvector of the original matrix: (Q Z) x, unit 2-norm
    double nrm = 0.0;
    for (int r = 0; r < m; ++r) {
      cd s = 0.0;
      for (int l = 0; l <= i; ++l) s += Z[(size_t)r * m + l] * x[l];
      V[(size_t)r * m + i] = s;
      nrm += std::norm(s);
    }
    nrm = std::sqrt(nrm);
    for (int r = 0; r < m; ++r) V[(size_t)r * m + i] /= nrm;
  }
  return true;
}

}  // namespace wh
