"""The GPU eigensolver for the deflation set (wh_eigs) against closed forms, the oracle's
eigenpairs and an independently assembled discrete pencil, and deflated GMRES with its
basis against the direct solution of the discrete Helmholtz system."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    assert torch.cuda.is_available()
    return torch, W


def _square_closed_form(prob, ts, k):
    from oracle.oracle import beta_d_sum, lambda_tilde
    n, h = prob.grids[0].n[0], prob.grids[0].h[0]
    m = np.arange(1, n - 1)
    sx = np.sin(m * np.pi * h / 2) ** 2
    lam2 = ((4 / h ** 2) * (sx[None, :] + sx[:, None])).ravel()
    bd = beta_d_sum(lambda_tilde(np.sqrt(lam2), ts.dt), ts.omega_e, ts.dt, ts.Nt, ts.alpha)
    top = np.argsort(-np.abs(bd))
    return bd[top[:k]], lam2[top[:k]], abs(bd[top[k]])


def _subspace_gap(A, B):
    """Largest sine of the principal angles between the row spaces of A and B (orthonormal
    rows, same count): the spectral norm of A's rows minus their projection on B's span
    (computed directly; sqrt(1 - cos^2) would lose half the digits)."""
    R = A - (A @ B.T) @ B
    return float(np.linalg.norm(R, 2))


def test_eigs_unit_square_closed_form_and_oracle(env, oracle_mod):
    """32^2 unit square: the five modes of S with largest |beta| (two degenerate pairs
    complete; the sixth would split a pair) carry beta_d(lambda~) and lambda_h^2 in closed form (1e-10), their span equals the
    oracle's ARPACK span, and the basis is orthonormal with T = Q S Q^T."""
    torch, W = env
    from oracle import deflation as D
    prob = G.unit_square_problem(32, 2, 10.0, seed=0)
    s = W.Solver(prob)
    ti = s.prepare()
    orc = oracle_mod.Oracle(prob)
    bref, lref, nxt = _square_closed_form(prob, orc.time, 5)
    assert nxt < np.min(np.abs(bref)) - 1e-6  # a gap after the sixth
    Q, T, beta, lam2, st = s.eigs(5, tol=1e-11, max_products=3000)
    assert st.converged == 1, (st.status, st.residual, st.iterations)
    assert np.allclose(np.sort(beta), np.sort(bref), rtol=0, atol=1e-10)
    assert np.allclose(np.sort(lam2), np.sort(lref), rtol=1e-10)
    Qh = Q.cpu().numpy()
    assert np.allclose(Qh @ Qh.T, np.eye(5), atol=1e-12)
    Phi, l2, b2 = D.wave_eigenpairs(orc, 5)
    assert _subspace_gap(Qh, Phi) < 1e-8
    # T is the Rayleigh matrix: T = Q S Q^T, checked with the oracle's map
    assert np.allclose(T, D.rayleigh_matrix(orc, Qh), atol=1e-11)


def test_eigs_overset_disk_match_pencil_and_deflated_solve(env, oracle_mod):
    """Overset disk-in-square (order 2, non-self-adjoint): the GPU eigenpairs are those of
    the independently assembled pencil A(omega) x = (omega^2 - lambda^2) B x (B = 1 on
    discretization rows, the constrained eigenproblem of Sec. 4.4): the six pencil
    eigenvalues of largest |beta_d(lambda~)| (the filter's transfer function, Eq. betad)
    give the GPU's beta (to 5e-8, see below) and its lambda^2 (1e-7 relative); GMRES on the deflated
    iteration with the exact inflation reaches the direct solution with fewer wave solves
    than plain GMRES."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    import dhs
    from oracle.oracle import beta_d_sum, lambda_tilde
    torch, W = env
    dp = G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=8.0, width=0.8, r_cut=0.75)
    s = W.Solver(dp)
    ti = s.prepare()
    Q, T, beta, lam2, st = s.eigs(6, tol=1e-11, max_products=4000)
    assert st.converged == 1, (st.status, st.residual, st.iterations)
    A, rhs, lay = dhs.assemble(dp, dp.omega)
    Bd = np.zeros(lay.N)
    for gi, g in enumerate(dp.grids):
        for j, i in zip(*np.nonzero(g.mask == G.DISC)):
            Bd[lay.idx(gi, int(i), int(j))] = 1.0
    mu, _ = spla.eigs(A.tocsc(), k=16, M=sp.diags(Bd).tocsc(), sigma=0.0)
    lp = np.real(dp.omega ** 2 - mu)
    orc = oracle_mod.Oracle(dp)
    ts = orc.time
    bp = beta_d_sum(lambda_tilde(np.sqrt(lp), ts.dt), ts.omega_e, ts.dt, ts.Nt, ts.alpha)
    top = np.argsort(-np.abs(bp))[:6]
    # 5e-8: the third and fourth modes are a nearly defective pair (the pencil returns them
    # as a complex pair with imaginary part 1.2e-8), whose eigenvalues move by about the
    # square root of a perturbation; the others agree to rounding
    assert np.allclose(np.sort(beta), np.sort(bp[top]), rtol=0, atol=5e-8)
    assert np.allclose(np.sort(lam2), np.sort(lp[top]), rtol=1e-7)
    U = dhs.solve(dp)
    s.set_deflation_basis(Q, T)
    u = torch.zeros(dp.n_total, dtype=torch.float64, device="cuda")
    std = s.solve(u, W.GMRES, tol=1e-12, max_it=4000, restart=100)
    assert std.converged
    got = u.cpu().numpy()
    assert np.max(np.abs(got - U)) <= 1e-8 * np.max(np.abs(U))
    s.set_deflation(None)
    u0 = torch.zeros_like(u)
    st0 = s.solve(u0, W.GMRES, tol=1e-12, max_it=4000, restart=100)
    assert st0.converged and std.iterations < st0.iterations


def test_eigs_arguments_and_state(env):
    torch, W = env
    from paper_2504_03074_gb300 import grids3 as G3
    prob = G.unit_square_problem(16, 2, 3.0)
    s = W.Solver(prob)
    with pytest.raises(W.WHError) as e:
        s.eigs(2)
    assert e.value.status == -3  # before wh_prepare
    s.prepare()
    with pytest.raises(W.WHError) as e:
        s.eigs(4, m=5)
    assert e.value.status == -1  # basis smaller than k + 2
    c = W.Solver(G3.unit_cube_problem(9, omega=4.0))
    with pytest.raises(W.WHError) as e:
        c.eigs(2)
    assert e.value.status == -3  # a 3D context, before wh_prepare


def test_eigs_large_basis_invariant(env):
    """A basis of 40 vectors (overset disk, order 4, four periods, where S has many modes
    of |beta| near 1 in conjugate pairs and clusters): Q has orthonormal rows and spans an
    S-invariant subspace, S Q^T = Q^T T, checked by applying the map to each row; T is
    Q S Q^T.  Both coefficient sets of the final products are uploaded while the first
    product may still run, so this also guards their ordering."""
    torch, W = env
    dp = G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=12.0)
    s = W.Solver(dp, periods=4)
    s.prepare()
    k = 40
    Q, T, beta, lam2, st = s.eigs(k, tol=1e-12, max_products=4000)
    assert st.converged == 1, (st.status, st.residual, st.iterations)
    SQ = torch.empty_like(Q)
    for i in range(k):
        s.iterate(Q[i].contiguous(), SQ[i], False)
    torch.cuda.synchronize()
    Tt = torch.from_numpy(np.ascontiguousarray(T)).to(Q.device)
    eye = torch.eye(k, dtype=Q.dtype, device=Q.device)
    assert float((Q @ Q.T - eye).abs().max()) < 1e-12
    assert float((SQ.T - Q.T @ Tt).abs().max()) < 1e-10
    assert float((Q @ SQ.T - Tt).abs().max()) < 1e-12
    # the reported beta are the eigenvalues of T (real parts, pairs repeated), descending
    ev = np.linalg.eigvals(T)
    assert np.allclose(np.sort(beta), np.sort(ev.real), atol=1e-10)
    assert np.all(np.abs(beta) <= 1.0 + 1e-9) and np.all(np.isfinite(lam2))
