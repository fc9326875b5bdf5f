"""The GPU eigensolver and the deflated solves on three-dimensional contexts: closed-form
eigenpairs of an anisotropic Dirichlet box, Algorithm 3's fixed-point iteration with the
GPU's eigenpairs against the oracle's, and on the overset box-in-box the agreement of each
beta with the filter at its Rayleigh lambda^2 and deflated GMRES with the exact inflation
against the direct solution of the discrete Helmholtz system."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids3 as G3

pytestmark = pytest.mark.gpu

_NS = (13, 16, 19)  # distinct spacings per axis: no repeated eigenvalues


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    assert torch.cuda.is_available()
    return torch, W


def _box(omega):
    g = G3.cartesian_grid3("box", _NS, (0.0,) * 3, (1.0,) * 3, [G3.BC_DIRICHLET] * 6)
    f = [G3.gaussian3(g, np.array([0.45, 0.55, 0.5]), 1.0, 200.0)]
    return G3.Problem3([g], G3.Interp3.empty(), omega, f, name="box-13x16x19")


def _box_closed_form(ts, k):
    """The k modes of largest |beta_d(lambda~)| of the 7-point Laplacian on the box with
    Dirichlet walls: lambda^2 = sum over axes of (4 / h_a^2) sin^2(m_a pi h_a / 2)."""
    from oracle.oracle import beta_d_sum, lambda_tilde
    comps = []
    for n in _NS:
        h = 1.0 / (n - 1)
        m = np.arange(1, n - 1)
        comps.append((4 / h ** 2) * np.sin(m * np.pi * h / 2) ** 2)
    lam2 = (comps[2][:, None, None] + comps[1][None, :, None] + comps[0][None, None, :]).ravel()
    bd = beta_d_sum(lambda_tilde(np.sqrt(lam2), ts.dt), ts.omega_e, ts.dt, ts.Nt, ts.alpha)
    top = np.argsort(-np.abs(bd))
    return bd[top[:k]], lam2[top[:k]], abs(bd[top[k]])


def test_eigs3_box_closed_form_and_deflated_fpi(env):
    """Seven modes of the 13 x 16 x 19 box (omega 10; a gap of 0.1 in |beta| after the
    seventh): beta and lambda^2 in closed form, an orthonormal basis with T = Q S Q^T by
    the oracle's map; then 20 iterations of Algorithm 3 with these eigenpairs on the GPU
    equal the oracle's (inflation with the forcing at discretization points)."""
    torch, W = env
    import oracle.oracle3 as O3
    from oracle import deflation as D
    prob = _box(10.0)
    orc = O3.Oracle3(prob)
    k = 7
    bref, lref, nxt = _box_closed_form(orc.time, k)
    assert nxt < np.min(np.abs(bref)) - 0.05
    s = W.Solver(prob)
    s.prepare()
    Q, T, beta, lam2, st = s.eigs(k, tol=1e-12, max_products=3000)
    assert st.converged == 1, (st.status, st.residual, st.iterations)
    assert np.allclose(np.sort(beta), np.sort(bref), rtol=0, atol=1e-10)
    assert np.allclose(np.sort(lam2), np.sort(lref), rtol=1e-10)
    Qh = Q.cpu().numpy()
    assert np.allclose(Qh @ Qh.T, np.eye(k), atol=1e-12)
    assert np.allclose(T, D.rayleigh_matrix(orc, Qh), atol=1e-11)
    # self-adjoint with distinct eigenvalues: T is diagonal and the rows of Q are the
    # eigenvectors; pair each row with its lambda^2 through its beta
    assert np.max(np.abs(T - np.diag(np.diag(T)))) < 1e-10
    l2 = np.array([lam2[int(np.argmin(np.abs(beta - T[i, i])))] for i in range(k)])
    f = np.concatenate([x.ravel() for x in prob.f])
    ref, _, _ = D.deflated_fpi(orc, Qh, l2, f, prob.omega, 20)
    phi = torch.from_numpy(Qh).cuda().contiguous()
    s.set_deflation(phi, l2)
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    s.solve(u, W.FPI, tol=1e-300, max_it=20)
    got = u.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_eigs3_overset_consistency_and_deflated_gmres(env):
    """Box-in-box overset grid (omega 6): each beta from the Krylov-Schur run equals the
    filter's transfer function at the eigenvector's Rayleigh lambda^2 (two independent
    computations: one from S, one from one step of the spatial operator), and GMRES on the
    deflated iteration with the exact inflation reaches the direct solution, in the FP64
    and the FP32-then-FP64 forms."""
    import dhs3
    from oracle.oracle import beta_d_sum, lambda_tilde
    torch, W = env
    prob = G3.box_in_box_problem()
    s = W.Solver(prob)
    ti = s.prepare()
    k = 4
    Q, T, beta, lam2, st = s.eigs(k, tol=1e-12, max_products=4000)
    assert st.converged == 1, (st.status, st.residual, st.iterations)
    bd = beta_d_sum(lambda_tilde(np.sqrt(lam2), ti.dt), ti.omega_e, ti.dt, ti.Nt, ti.alpha)
    assert np.allclose(np.sort(bd), np.sort(beta), rtol=0, atol=1e-8), (bd, beta)
    U = dhs3.solve(prob)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    for prec in (W.FP64, W.FP32):
        sp = W.Solver(prob, precision=prec)
        sp.prepare()
        sp.set_deflation_basis(Q, T)
        u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
        std = sp.solve(u, W.GMRES, tol=1e-12, max_it=1000, restart=200)
        assert std.converged == 1
        got = u.cpu().numpy()
        assert np.max(np.abs(got - U)[act]) <= 1e-8 * np.max(np.abs(U)), prec
        sp.close()
