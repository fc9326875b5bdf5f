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

// Swap the adjacent diagonal entries i, i+1 of the upper triangular T (complex Schur form)
// by a unitary rotation, updating Z: the rotation's first column is the eigenvector of the
// 2 x 2 block for its second eigenvalue.
void schur_swap(int m, std::vector<cd> &T, std::vector<cd> &Z, int i) {
  auto t = [&](int r, int c) -> cd & { return T[(size_t)r * m + c]; };
  const cd a = t(i, i), b = t(i + 1, i + 1), c = t(i, i + 1);
  cd x1 = c, x2 = b - a;
  const double nx = std::sqrt(std::norm(x1) + std::norm(x2));
  if (nx == 0.0) return;  // equal eigenvalues, nothing to swap
  x1 /= nx;
  x2 /= nx;
  // T <- U^* T U with U = [[x1, -conj(x2)], [x2, conj(x1)]]
  for (int j = i; j < m; ++j) {
    const cd p = t(i, j), q = t(i + 1, j);
    t(i, j) = std::conj(x1) * p + std::conj(x2) * q;
    t(i + 1, j) = -x2 * p + x1 * q;
  }
  for (int r = 0; r <= i + 1; ++r) {
    const cd p = t(r, i), q = t(r, i + 1);
    t(r, i) = x1 * p + x2 * q;
    t(r, i + 1) = -std::conj(x2) * p + std::conj(x1) * q;
  }
  for (int r = 0; r < m; ++r) {
    const cd p = Z[(size_t)r * m + i], q = Z[(size_t)r * m + i + 1];
    Z[(size_t)r * m + i] = x1 * p + x2 * q;
    Z[(size_t)r * m + i + 1] = -std::conj(x2) * p + std::conj(x1) * q;
  }
  t(i + 1, i) = 0.0;
}

}  // namespace

int invariant_basis(int m, const double *A, int want, std::vector<double> &Q,
                    std::vector<std::complex<double>> &w) {
  // the real basis may need one column per selected eigenvalue and, for members of split
  // conjugate pairs, one more (see below); callers check the returned size
  Q.clear();
  w.clear();
  if (m <= 0 || want <= 0) return 0;
  want = std::min(want, m);
  std::vector<double> H(A, A + (size_t)m * m), Qh;
  hessenberg(m, H, Qh);
  std::vector<cd> T(H.begin(), H.end()), Z(Qh.begin(), Qh.end());
  if (!schur(m, T, Z)) return -1;
  // the wanted eigenvalues: largest modulus, a complex pair kept whole
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::vector<cd> d(m);
  for (int i = 0; i < m; ++i) d[i] = T[(size_t)i * m + i];
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return std::abs(d[a]) > std::abs(d[b]); });
  std::vector<char> sel(m, 0);
  int p = 0;
  for (int t = 0; t < m && p < want; ++t) {
    const int i = idx[t];
    if (sel[i]) continue;
    sel[i] = 1;
    ++p;
    if (std::fabs(d[i].imag()) > 1e-8 * std::abs(d[i])) {  // its conjugate too
      int best = -1;
      for (int j = 0; j < m; ++j)
        if (!sel[j] && (best < 0 || std::abs(d[j] - std::conj(d[i])) < std::abs(d[best] - std::conj(d[i]))))
          best = j;
      if (best >= 0) {
        sel[best] = 1;
        ++p;
      }
    }
  }
  // bubble the selected eigenvalues to the leading positions
  int slot = 0;
  for (int i = 0; i < m; ++i) {
    if (!sel[i]) continue;
    for (int j = i; j > slot; --j) {
      schur_swap(m, T, Z, j - 1);
      std::swap(sel[j], sel[j - 1]);
    }
    ++slot;
  }
  for (int i = 0; i < p; ++i) w.push_back(T[(size_t)i * m + i]);
  // A real orthonormal basis of span(Re Z_p, Im Z_p) — the real span of the selected complex
  // subspace and of its conjugate, itself invariant since A is real — by Gram-Schmidt with
  // column pivoting (the column with the largest remaining norm first, each orthogonalised
  // twice), stopped when what remains is below 1e-6 of the largest column: rounding leaves
  // ~1e-14 for a real eigenvalue's Schur vector, and a nearly real conjugate pair split by
  // the selection keeps the extra dimension that its invariance needs.  (An eigensolve of
  // the Gram matrix would not do: its nonzero eigenvalues are all near 1.)
  const int q = 2 * p;
  std::vector<double> B((size_t)m * q);
  for (int c = 0; c < p; ++c)
    for (int r = 0; r < m; ++r) {
      B[(size_t)(2 * c) * m + r] = Z[(size_t)r * m + c].real();
      B[(size_t)(2 * c + 1) * m + r] = Z[(size_t)r * m + c].imag();
    }
  auto norm = [&](int c) {
    double t = 0.0;
    for (int r = 0; r < m; ++r) t += B[(size_t)c * m + r] * B[(size_t)c * m + r];
    return std::sqrt(t);
  };
  double n0 = 0.0;
  for (int c = 0; c < q; ++c) n0 = std::max(n0, norm(c));
  std::vector<char> used(q, 0);
  Q.clear();
  int rank = 0;
  while (rank < std::min(q, m)) {
    int best = -1;
    double bn = 0.0;
    for (int c = 0; c < q; ++c)
      if (!used[c]) {
        const double t = norm(c);
        if (t > bn) {
          bn = t;
          best = c;
        }
      }
    if (best < 0 || !(bn > 1e-6 * n0)) break;
    used[best] = 1;
    std::vector<double> v(B.begin() + (size_t)best * m, B.begin() + (size_t)(best + 1) * m);
    for (int pass = 0; pass < 2; ++pass)
      for (int d = 0; d < rank; ++d) {
        const double *y = &Q[(size_t)d * m];
        double h = 0.0;
        for (int r = 0; r < m; ++r) h += y[r] * v[r];
        for (int r = 0; r < m; ++r) v[r] -= h * y[r];
      }
    double nv = 0.0;
    for (int r = 0; r < m; ++r) nv += v[r] * v[r];
    nv = std::sqrt(nv);
    for (int r = 0; r < m; ++r) v[r] /= nv;
    Q.insert(Q.end(), v.begin(), v.end());
    ++rank;
    // remove the new direction from the columns still waiting
    for (int c = 0; c < q; ++c)
      if (!used[c]) {
        double *b = &B[(size_t)c * m];
        double h = 0.0;
        for (int r = 0; r < m; ++r) h += v[r] * b[r];
        for (int r = 0; r < m; ++r) b[r] -= h * v[r];
      }
  }
  return rank;
}

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
