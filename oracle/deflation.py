"""WaveHoltz with deflation (Algorithm 3, Sec. 4.4) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module.  It runs on top of an oracle object (``Oracle`` or
``Oracle3``: anything with ``iterate(v, forcing)``) and a deflation set of discrete
eigenpairs (phi_m, lambda_m^2) supplied by the caller:

* each WaveHoltz iteration is followed by the deflation step
  v <- v - sum_m (v, phi_m) phi_m   (the components along the deflated modes removed);
* after the iteration has converged the missing components of the Helmholtz solution are
  added back ("inflate"): v <- v + sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m.

Inner products are the plain sum over the compact vector (unused points hold 0); the
eigenvectors must be orthonormal in that inner product.  With g = 0 only, as in the paper.
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


def inflate(v, Phi, lam2, f, omega):
    """v + sum_m (f, phi_m) / (omega^2 - lambda_m^2) phi_m (the Helmholtz solution's
    components along the deflated modes, g = 0)."""
    if Phi is None or len(Phi) == 0:
        return v
    coef = (Phi @ f) / (omega ** 2 - np.asarray(lam2, np.float64))
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
    return inflate(v, Phi, lam2, f, omega), hist, res
