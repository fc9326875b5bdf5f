"""WaveHoltz with deflation (Algorithm 3, Sec. 4.4) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module.  It runs on top of an oracle object (``Oracle`` or
``Oracle3``: anything with ``iterate(v, forcing)``) and a deflation set of discrete
eigenpairs (phi_m, lambda_m^2) supplied by the caller:

* each WaveHoltz iteration is followed by the deflation step
  v <- v - sum_m (v, phi_m) phi_m   (the components along the deflated modes removed);
* after the iteration has converged the missing components of the Helmholtz solution are
  added back ("inflate"): v <- v + sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m.

Inner products are the plain sum over the compact vector (unused points hold 0); the
eigenvectors must be orthonormal in that inner product.  In (f, phi_m) the forcing counts
at discretization points only: Sec. 4.4 writes the discrete eigenproblem as A x = lambda B x
with B = 1 on the rows where the PDE is discretized and 0 on the boundary and interpolation
rows, which is also where the forcing enters the discrete Helmholtz system.  With g = 0
only, as in the paper.
The deflated fixed-point iteration converges at the rate max over non-deflated modes of
|beta_d(lambda~_m)| (Theorem "WaveHoltz FPI convergence with deflation").
"""
from __future__ import annotations

import numpy as np


def deflate(v, Phi):
    """v - sum_m (v, phi_m) phi_m, Phi of shape (K, n) with orthonormal rows."""
    if Phi is None or len(Phi) == 0:
        return v
    return v - Phi.T @ (Phi @ v)


def disc_mask(problem):
    """1.0 at discretization points, 0.0 elsewhere, as a compact vector."""
    return np.concatenate([(np.asarray(g.mask) == 1).ravel() for g in problem.grids]
                          ).astype(np.float64)


def inflate(v, Phi, lam2, f, omega, disc=None):
    """v + sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m (the Helmholtz solution's
    components along the deflated modes, g = 0); with `disc` (1 at discretization points)
    the pairing (f, phi_m) takes f on those points only."""
    if Phi is None or len(Phi) == 0:
        return v
    fd = f if disc is None else f * disc
    coef = (Phi @ fd) / (omega ** 2 - np.asarray(lam2, np.float64))
    return v + Phi.T @ coef


def deflated_fpi(orc, Phi, lam2, f, omega, iters, v0=None):
    """Algorithm 3 for a fixed number of iterations from v0 (default 0).

    Returns (u, history, residuals): u is the inflated approximation after `iters`
    iterations, history the deflated iterates v^(k), residuals ||v^(k+1) - v^(k)||_2."""
    v = orc.zeros() if v0 is None else np.array(v0, np.float64)
    hist, res = [v.copy()], []
    for _ in range(iters):
        vn = deflate(orc.iterate(v, True), Phi)
        res.append(float(np.linalg.norm(vn - v)))
        v = vn
        hist.append(v.copy())
    return inflate(v, Phi, lam2, f, omega, disc_mask(orc.problem)), hist, res


class _Deflated:
    """The deflated WaveHoltz map v -> P W_h(v, f), P = I - Phi^T Phi, with the oracle's
    interface (``iterate``, ``zeros``), so that the oracle's GMRES solves its fixed point."""

    def __init__(self, orc, Phi):
        self.orc, self.Phi, self.problem = orc, Phi, orc.problem

    def iterate(self, v, forcing=True):
        return deflate(self.orc.iterate(v, forcing), self.Phi)

    def zeros(self):
        return self.orc.zeros()


def deflated_gmres(orc, Phi, lam2, f, omega, tol=1e-12, restart=60, max_it=2000):
    """GMRES (Sec. 4.3) on the deflated fixed-point iteration of Algorithm 3: solves
    (I - P S) v = P b, then inflates.  Returns (u, products, history)."""
    from .oracle import gmres
    v, its, hist = gmres(_Deflated(orc, Phi), tol=tol, restart=restart, max_it=max_it)
    return inflate(v, Phi, lam2, f, omega, disc_mask(orc.problem)), its, hist


def rayleigh_matrix(orc, Q):
    """T = Q S Q^T (T[i, j] = (q_i, S q_j)) for the rows q_i of Q, by one zero-forcing
    WaveHoltz iteration per row."""
    SQ = np.array([orc.iterate(q, False) for q in Q])
    return Q @ SQ.T


def schur_inflate(orc, v, Q, T):
    """The Helmholtz solution from the deflated fixed point v, exactly, when the rows of Q
    are an orthonormal basis of an S-invariant subspace with S Q^T = Q^T T: writing
    U = v + Q^T c and U = S U + b (Sec. 4.3) and projecting on the rows of Q gives
    (I - T) c = Q W_h(v, f).  On a self-adjoint discretization, with Q eigenvectors, this
    equals Algorithm 3's inflation; on overset grids it does not need left eigenvectors."""
    w = orc.iterate(v, True)
    c = np.linalg.solve(np.eye(len(Q)) - T, Q @ w)
    return v + Q.T @ c


def deflated_gmres_schur(orc, Q, T, tol=1e-12, restart=60, max_it=3000):
    """GMRES on the deflated fixed-point iteration (projector I - Q^T Q), then the exact
    inflation of schur_inflate.  Returns (u, products, history)."""
    from .oracle import gmres
    v, its, hist = gmres(_Deflated(orc, Q), tol=tol, restart=restart, max_it=max_it)
    return schur_inflate(orc, v, Q, T), its, hist


def wave_eigenpairs(orc, k, tol=1e-12, seed=0, passes=2):
    """The k eigenpairs of the zero-forcing WaveHoltz map S = W_h(., 0) of largest |beta|
    (the modes the fixed-point iteration reduces most slowly), by ARPACK (implicitly
    restarted Arnoldi, scipy) on S as a linear operator, each with its eigenvalue lambda^2
    of the constrained spatial operator from the Rayleigh quotient -(phi, c^2 L_h phi) /
    (phi, phi) over the discretization points (ghosts filled by the boundary rules first).

    A single-vector Krylov method finds repeated eigenvalues (symmetric geometries) only
    through rounding, so each further pass runs ARPACK again on (I - Q Q^T) S (I - Q Q^T),
    Q an orthonormal basis of the eigenvectors found so far, and the k pairs of largest
    |beta| of the union are kept.  An eigenvector of S is an eigenvector of the discrete
    spatial operator with its boundary and interpolation constraints (S is a polynomial of
    the one-step map), so the quotient is exact up to the eigensolver's accuracy.  Returns
    (Phi, lam2, beta): Phi (k, n) with orthonormal rows (a QR of the eigenvectors: exact
    eigenvectors for a self-adjoint discretization, a basis of their span otherwise), lam2
    (k,), beta (k,)."""
    import scipy.sparse.linalg as spla
    n = orc.problem.n_total
    act = orc.active()
    rng = np.random.default_rng(seed)
    vals_all, vecs_all = [], []
    Q = np.zeros((n, 0))
    for _ in range(max(1, passes)):
        def matvec(x, Q=Q):
            x = np.real(x)
            if Q.shape[1]:
                x = x - Q @ (Q.T @ x)
            y = orc.iterate(x, False)
            if Q.shape[1]:
                y = y - Q @ (Q.T @ y)
            return y
        op = spla.LinearOperator((n, n), matvec=matvec, dtype=np.float64)
        v0 = rng.standard_normal(n) * act
        if Q.shape[1]:
            v0 = v0 - Q @ (Q.T @ v0)
        vals, vecs = spla.eigs(op, k=k, which="LM", v0=v0, tol=tol)
        vals_all.append(np.real(vals))
        vecs_all.append(np.real(vecs))
        Q, _ = np.linalg.qr(np.concatenate(vecs_all, axis=1))
    vals = np.concatenate(vals_all)
    vecs = np.concatenate(vecs_all, axis=1)
    order = np.argsort(-np.abs(vals))[:k]
    vals, vecs = vals[order], vecs[:, order]
    Q, _ = np.linalg.qr(vecs)
    Phi = Q.T.copy()
    lam2 = np.array([_rayleigh_lam2(orc, vecs[:, m]) for m in range(k)])
    return Phi, lam2, vals


def _rayleigh_lam2(orc, phi):
    """-(phi, c^2 L_h phi) / (phi, phi) over discretization points, phi a compact vector."""
    prob = orc.problem
    num = den = 0.0
    parts = prob.split(phi)
    for gi, g in enumerate(prob.grids):
        shape = orc.ext_shape(gi)
        u = np.zeros(shape)
        gh = [(shape[a] - p) // 2 for a, p in enumerate(parts[gi].shape)]
        sl = tuple(slice(gh[a], gh[a] + parts[gi].shape[a]) for a in range(len(shape)))
        u[sl] = parts[gi]
        u = orc.apply_bc(gi, u, 0.0) if getattr(prob, "dim", 2) == 2 else orc.apply_bc(gi, u)
        lu = orc.apply_lap(gi, u)[sl]
        disc = g.mask == 1
        num += float(np.sum(parts[gi][disc] * lu[disc]))
        den += float(np.sum(parts[gi][disc] ** 2))
    return -num / den
