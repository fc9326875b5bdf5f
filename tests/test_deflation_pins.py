"""Pins for WaveHoltz with deflation (Algorithm 3) on the oracle (CPU only): on the unit
square the discrete eigenmodes are DST-I modes with known eigenvalues, so every deflated
iterate has a closed form."""
import math

import numpy as np
import pytest
import scipy.fft as sfft

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _square_modes(prob, ts):
    """DST-I data of the 64^2 unit square: f_hat, lambda_h^2 and beta_d(lambda~) per mode
    (Eqs. betad, discreteExplicitLambdaTilde; eigenvalues of D+D- with Dirichlet data)."""
    from oracle.oracle import beta_d_sum, lambda_tilde
    n = prob.grids[0].n[0]
    h = prob.grids[0].h[0]
    fh = sfft.dstn(prob.f[0][1:-1, 1:-1], type=1, norm="ortho")
    m = np.arange(1, n - 1)
    sx = np.sin(m * np.pi * h / 2) ** 2
    lam2 = (4 / h ** 2) * (sx[None, :] + sx[:, None])
    lt = lambda_tilde(np.sqrt(lam2).ravel(), ts.dt)
    bd = beta_d_sum(lt, ts.omega_e, ts.dt, ts.Nt, ts.alpha).reshape(lam2.shape)
    return fh, lam2, bd


def _mode_vector(n, my, mx):
    """Orthonormal (Euclidean, compact n x n vector) DST-I mode (my, mx), zero on the
    boundary."""
    phi = np.zeros((n, n))
    z = np.zeros((n - 2, n - 2))
    z[my - 1, mx - 1] = 1.0
    phi[1:-1, 1:-1] = sfft.idstn(z, type=1, norm="ortho")
    return phi.ravel()


@pytest.mark.parametrize("K", [1, 8])
def test_deflated_iterates_match_closed_form(oracle_mod, K):
    """Deflating the K modes with |beta_d| closest to 1: the k-th deflated iterate from
    v = 0 is sum over kept modes (1 - beta_m^k) U_m Phi_m (the deflated components stay 0),
    the inflated iterate adds U_m Phi_m for the deflated modes, with
    U_m = f_m / (omega^2 - lambda_m^2) (Algorithm 3; c2 reading: omega-hat = omega)."""
    from oracle import deflation as D
    prob = G.unit_square_problem(64, 2, 10.0, seed=0)
    orc = oracle_mod.Oracle(prob)
    ts = orc.time
    fh, lam2, bd = _square_modes(prob, ts)
    order = np.argsort(-np.abs(bd).ravel())[:K]
    dmask = np.zeros(bd.size, bool)
    dmask[order] = True
    dmask = dmask.reshape(bd.shape)
    n = 64
    Phi = np.array([_mode_vector(n, i + 1, j + 1) for i, j in zip(*np.nonzero(dmask))])
    lam2_d = lam2[dmask]
    f = prob.f[0].ravel()
    U = fh / (prob.omega ** 2 - lam2)
    iters = 12
    u, hist, res = D.deflated_fpi(orc, Phi, lam2_d, f, prob.omega, iters)
    for k in (1, 5, iters):
        kept = np.where(dmask, 0.0, (1 - bd ** k) * U)
        ref = np.zeros((n, n))
        ref[1:-1, 1:-1] = sfft.idstn(kept, type=1, norm="ortho")
        got = hist[k].reshape(n, n)
        assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref)), k
    # inflation adds the deflated modes' Helmholtz components exactly
    full = np.where(dmask, U, (1 - bd ** iters) * U)
    ref = np.zeros((n, n))
    ref[1:-1, 1:-1] = sfft.idstn(full, type=1, norm="ortho")
    assert np.max(np.abs(u.reshape(n, n) - ref)) < 1e-12 * np.max(np.abs(ref))


def test_deflated_rate_is_largest_kept_beta(oracle_mod):
    """Theorem (WaveHoltz FPI convergence with deflation): the deflated zero-forcing map
    P S (P the projector off the deflated modes) sends a kept mode to beta_d times itself
    and a deflated mode to 0, so its spectral radius is the largest |beta_d| kept; deflating
    the 8 modes nearest omega lowers it from 0.99965 here."""
    from oracle import deflation as D
    prob = G.unit_square_problem(64, 2, 10.0, seed=0)
    orc = oracle_mod.Oracle(prob)
    fh, lam2, bd = _square_modes(prob, orc.time)
    order = np.argsort(-np.abs(bd).ravel())
    K = 8
    idx = [np.unravel_index(q, bd.shape) for q in order]
    Phi = np.array([_mode_vector(64, i + 1, j + 1) for i, j in idx[:K]])
    for i, j in idx[:K + 3]:
        phi = _mode_vector(64, i + 1, j + 1)
        out = D.deflate(orc.iterate(phi, False), Phi)
        expect = 0.0 if (i, j) in idx[:K] else bd[i, j]
        assert np.max(np.abs(out - expect * phi)) < 1e-13
    mu = np.abs(bd.ravel()[order[K]])
    assert np.abs(bd).max() == pytest.approx(0.99965, abs=1e-5)
    assert mu < np.abs(bd).max()
    # the rate: error after k deflated iterations decays like mu^k along the slowest kept mode
    iters = 30
    u, hist, res = D.deflated_fpi(orc, Phi, lam2[tuple(np.array(idx[:K]).T)],
                                  prob.f[0].ravel(), prob.omega, iters)
    ratios = [res[k + 1] / res[k] for k in range(iters - 6, iters - 1)]
    assert max(ratios) <= mu + 1e-9


def test_wave_eigenpairs_match_closed_form(oracle_mod):
    """The oracle's eigenpairs of S on the 32^2 unit square: the six of largest |beta| carry
    beta_d(lambda~) and lambda_h^2 of the DST-I modes nearest omega, in closed form."""
    from oracle import deflation as D
    prob = G.unit_square_problem(32, 2, 10.0, seed=0)
    orc = oracle_mod.Oracle(prob)
    fh, lam2, bd = _square_modes(prob, orc.time)
    order = np.argsort(-np.abs(bd).ravel())[:6]
    Phi, l2, beta = D.wave_eigenpairs(orc, 6)
    assert np.allclose(np.sort(beta), np.sort(bd.ravel()[order]), rtol=0, atol=1e-10)
    assert np.allclose(np.sort(l2), np.sort(lam2.ravel()[order]), rtol=1e-10)
    assert np.allclose(Phi @ Phi.T, np.eye(6), atol=1e-12)


def test_wave_eigenpairs_match_discrete_pencil_on_overset_grid(oracle_mod):
    """On an overset disk-in-square (order 2) the eigenvalues lambda^2 of the six slowest
    modes of S are eigenvalues of the discrete pencil A(omega) x = (omega^2 - lambda^2) B x,
    assembled independently from textbook stencils (tests/dhs.py; B = 1 on discretization
    rows, 0 on the boundary and interpolation rows: the constrained eigenproblem of the
    deflation set, Sec. 4.4)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import dhs
    from oracle import deflation as D
    dp = G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=8.0, width=0.8, r_cut=0.75)
    orc = oracle_mod.Oracle(dp)
    Phi, l2, beta = D.wave_eigenpairs(orc, 6)
    A, rhs, lay = dhs.assemble(dp, dp.omega)
    Bd = np.zeros(lay.N)
    for gi, g in enumerate(dp.grids):
        for j, i in zip(*np.nonzero(g.mask == G.DISC)):
            Bd[lay.idx(gi, int(i), int(j))] = 1.0
    mu, _ = spla.eigs(A.tocsc(), k=12, M=sp.diags(Bd).tocsc(), sigma=0.0)
    lam_pencil = np.real(dp.omega ** 2 - mu)
    for x in l2:
        assert np.min(np.abs(lam_pencil - x)) < 1e-7 * x, (x, np.sort(lam_pencil))
    assert np.all(np.abs(beta) > 0.99)  # the modes nearest omega: |beta| close to 1


def test_wave_eigenpairs_3d_cube_closed_form():
    """3D: on the 11^3 Dirichlet cube the six modes of S with largest |beta| are two
    triply degenerate groups of sine modes; beta_d(lambda~) and lambda_h^2 in closed form,
    each eigenspace complete (the second ARPACK pass on the projected map finds the copies
    a single Krylov sequence misses)."""
    from oracle import deflation as D
    from oracle import oracle3 as O3
    from oracle.oracle import beta_d_sum, lambda_tilde
    from paper_2504_03074_gb300 import grids3 as G3
    n = 11
    prob = G3.unit_cube_problem(n, omega=9.0)
    orc = O3.Oracle3(prob)
    ts = orc.time
    h = 1.0 / (n - 1)
    s2 = (4 / h ** 2) * np.sin(np.arange(1, n - 1) * np.pi * h / 2) ** 2
    L2 = (s2[:, None, None] + s2[None, :, None] + s2[None, None, :]).ravel()
    bd = beta_d_sum(lambda_tilde(np.sqrt(L2), ts.dt), ts.omega_e, ts.dt, ts.Nt, ts.alpha)
    top = np.argsort(-np.abs(bd))[:6]
    Phi, l2, beta = D.wave_eigenpairs(orc, 6)
    assert np.allclose(np.sort(beta), np.sort(bd[top]), rtol=0, atol=1e-10)
    assert np.allclose(np.sort(l2), np.sort(L2[top]), rtol=1e-10)
    assert np.allclose(Phi @ Phi.T, np.eye(6), atol=1e-10)


def test_wave_eigenpairs_3d_overset_match_pencil_with_multiplicity():
    """3D overset (box-in-box, cubic symmetry): the six slowest modes of S are two triply
    degenerate eigenvalues of the discrete pencil A(omega) x = (omega^2 - lambda^2) B x,
    assembled independently (tests/dhs3.py), with the full multiplicity."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import dhs3
    from oracle import deflation as D
    from oracle import oracle3 as O3
    from paper_2504_03074_gb300 import grids3 as G3
    bp = G3.box_in_box_problem(omega=6.0)
    Phi, l2, beta = D.wave_eigenpairs(O3.Oracle3(bp), 6)
    A, rhs, lay = dhs3.assemble(bp)
    Bd = np.zeros(lay.N)
    for gi, g in enumerate(bp.grids):
        for k, j, i in zip(*np.nonzero(g.mask == G.DISC)):
            Bd[lay.idx(gi, int(i), int(j), int(k))] = 1.0
    mu, _ = spla.eigs(A.tocsc(), k=12, M=sp.diags(Bd).tocsc(), sigma=0.0)
    lp = np.real(bp.omega ** 2 - mu)
    for x in l2:
        close = lambda arr: int(np.sum(np.abs(arr - x) < 1e-9 * x))
        assert close(lp) >= 1 and close(l2) == close(lp), (x, np.sort(lp), np.sort(l2))


def test_deflated_gmres_reaches_closed_form_solution(oracle_mod):
    """GMRES (Sec. 4.3) on the deflated fixed-point iteration of Algorithm 3, then the
    inflation: on the unit square, where the DST-I modes are exact orthonormal eigenvectors
    of the self-adjoint discrete operator, the result is the discrete Helmholtz solution
    sum_m f_m / (omega^2 - lambda_m^2) Phi_m in closed form, whatever modes are deflated."""
    from oracle import deflation as D
    prob = G.unit_square_problem(32, 2, 10.0, seed=3)
    orc = oracle_mod.Oracle(prob)
    fh, lam2, bd = _square_modes(prob, orc.time)
    n = 32
    order = np.argsort(-np.abs(bd).ravel())[:6]
    idx = [np.unravel_index(q, bd.shape) for q in order]
    Phi = np.array([_mode_vector(n, i + 1, j + 1) for i, j in idx])
    l2 = np.array([lam2[i, j] for i, j in idx])
    u, its, hist = D.deflated_gmres(orc, Phi, l2, prob.f[0].ravel(), prob.omega, tol=1e-13)
    ref = np.zeros((n, n))
    ref[1:-1, 1:-1] = sfft.idstn(fh / (prob.omega ** 2 - lam2), type=1, norm="ortho")
    assert np.max(np.abs(u.reshape(n, n) - ref)) < 1e-10 * np.max(np.abs(ref))
    # the deflated components of the deflated iterate are zero before the inflation
    v = u - Phi.T @ ((Phi @ prob.f[0].ravel()) / (prob.omega ** 2 - l2))
    assert np.max(np.abs(Phi @ v)) < 1e-12 * np.max(np.abs(ref))


def test_schur_inflation_reaches_direct_solve_on_overset_grid(oracle_mod):
    """On an overset disk-in-square (order 2, interpolation makes the discrete operator
    non-symmetric) with the six slowest modes of S (a complete degenerate pair included, so
    their span is S-invariant): GMRES on the deflated fixed-point iteration followed by the
    exact inflation (I - T) c = Q W_h(v, f), T = Q S Q^T, reaches the independently
    assembled direct solution of the discrete Helmholtz system to 1e-9 (8e-11 measured);
    Algorithm 3's printed inflation, exact only for self-adjoint discretizations, is off by
    tens of percent on this nearly resonant problem (beta up to 0.99998)."""
    import dhs
    from oracle import deflation as D
    dp = G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=8.0, width=0.8, r_cut=0.75)
    orc = oracle_mod.Oracle(dp)
    U = dhs.solve(dp)
    Phi, l2, beta = D.wave_eigenpairs(orc, 6, passes=1)
    T = D.rayleigh_matrix(orc, Phi)
    SP = np.array([orc.iterate(p, False) for p in Phi])
    assert np.linalg.norm(SP.T - Phi.T @ T) < 1e-9  # invariant subspace
    u, its, _ = D.deflated_gmres_schur(orc, Phi, T, tol=1e-13)
    nu = np.max(np.abs(U))
    assert np.max(np.abs(u - U)) < 1e-9 * nu
    f = np.concatenate([np.asarray(x).ravel() for x in dp.f])
    v = u - Phi.T @ (Phi @ u)
    up = D.inflate(v, Phi, l2, f, dp.omega, D.disc_mask(dp))
    assert np.max(np.abs(up - U)) > 1e-3 * nu
