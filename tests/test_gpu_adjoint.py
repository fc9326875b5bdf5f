"""Differentiation form: the transposed WaveHoltz map and gradients of a receiver misfit.

* transposition: <S v, w> = <v, S^T w> to 1e-12 relative, S the zero-forcing iteration map;
* gradients of J = 0.5 |P u - d|^2 (P: bilinear sampling at 64 receivers on a circle of
  radius 1.5, d: data from a perturbed c) w.r.t. c(x)^2 and f against central finite
  differences in ten random directions (1e-6 relative) and against an independent adjoint of
  the direct discrete Helmholtz system (tests/dhs.py)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    return T


@pytest.fixture(scope="module")
def W():
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz
    return waveholtz


CASES = [
    ("square-o2", lambda: G.unit_square_problem(24, 2, 10.0)),
    ("square-o4", lambda: G.unit_square_problem(24, 4, 10.0)),
    ("channel-neumann-o4", lambda: G.channel_problem(24, 4, 5.0, bc=G.BC_NEUMANN)),
    ("torus-o4-box", lambda: G.sheared_torus_problem(24, 20, 4)),
    ("disk-o2", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=4.0, width=0.8,
                                       r_cut=0.75)),
    ("disk-o4", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8,
                                       r_cut=0.75)),
    ("disk-o4-cx", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, c_bumps=8,
                                          width=0.8, r_cut=0.75)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_transposition(torch, W, name, make):
    prob = make()
    s = W.Solver(prob)
    s.prepare()
    rng = np.random.default_rng(1)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    v = rng.standard_normal(prob.n_total) * act
    w = rng.standard_normal(prob.n_total) * act
    vt = torch.from_numpy(v).cuda()
    wt = torch.from_numpy(w).cuda()
    sv = torch.empty_like(vt)
    stw = torch.empty_like(wt)
    s.iterate(vt, sv, False)
    s.apply_adjoint(wt, stw)
    torch.cuda.synchronize()
    lhs = float(sv.cpu().numpy() @ w)
    rhs = float(v @ stw.cpu().numpy())
    scale = np.linalg.norm(sv.cpu().numpy()) * np.linalg.norm(w)
    assert abs(lhs - rhs) <= 1e-12 * scale, (lhs, rhs)


@pytest.fixture(scope="module")
def misfit_problem():
    """The sound-speed inversion workload (c = 1 + 0.2 sum of 8 Gaussian bumps, 64 receivers
    on the circle of radius 1.5, data from a locally faster medium) at a size where the
    forward and adjoint solves reach 1e-13."""
    prob = G.misfit_problem(nb=64, omega=4.0, seed=5, width=0.8, r_cut=0.75)
    P = G.receiver_matrix(prob, n=64, radius=1.5)
    import copy
    pert = copy.deepcopy(prob)
    pert.c2 = G.perturbed_c2(prob)
    import dhs
    d = P @ dhs.solve(pert)
    return prob, P, d


def solve_u(torch, W, prob, c2=None, f=None):
    s = W.Solver(prob)
    if c2 is not None:
        for gi, c in enumerate(prob.split(c2)):
            s.set_coefficient(gi, c)
    if f is not None:
        for gi, ff in enumerate(prob.split(f)):
            s.set_forcing(gi, ff)
    ti = s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-13, max_it=800, restart=400)
    assert st.converged == 1, (st.status, st.residual)
    return s, u, ti


def test_gradient_vs_finite_differences_and_direct_adjoint(torch, W, misfit_problem):
    import dhs
    prob, P, d = misfit_problem
    s, u, ti = solve_u(torch, W, prob)
    un = u.cpu().numpy()
    r = P @ un - d
    g = torch.from_numpy(P.T @ r).cuda()
    lam, gc2, gf, st = s.adjoint(u, g, tol=1e-13, max_it=800, restart=400)
    assert st.converged == 1
    gc2 = gc2.cpu().numpy()
    gf = gf.cpu().numpy()
    # independent adjoint of the direct discrete system
    U, J0, gc2_d, gf_d = dhs.adjoint_gradients(prob, P, d)
    assert np.max(np.abs(un - U)) <= 1e-9 * np.max(np.abs(U))
    assert np.linalg.norm(gc2 - gc2_d) <= 1e-6 * np.linalg.norm(gc2_d)
    assert np.linalg.norm(gf - gf_d) <= 1e-6 * np.linalg.norm(gf_d)
    # central finite differences in random directions
    c2 = np.concatenate([c.ravel() for c in prob.c2])
    f = np.concatenate([x.ravel() for x in prob.f])
    rng = np.random.default_rng(2)

    def J_of(c2v, fv):
        s2, u2, ti2 = solve_u(torch, W, prob, c2=c2v, f=fv)
        assert ti2.M == ti.M
        rr = P @ u2.cpu().numpy() - d
        return 0.5 * float(rr @ rr)

    for kind in ("c2",) * 6 + ("f",) * 4:  # ten random directions
        dirn = rng.standard_normal(prob.n_total)
        if kind == "c2":
            eps = 1e-5
            jp, jm = J_of(c2 + eps * dirn * c2, f), J_of(c2 - eps * dirn * c2, f)
            pred = float(gc2 @ (dirn * c2))
        else:
            eps = 1e-5 * np.max(np.abs(f))
            jp, jm = J_of(c2, f + eps * dirn), J_of(c2, f - eps * dirn)
            pred = float(gf @ dirn)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - pred) <= 1e-6 * max(abs(fd), abs(pred)) + 1e-14, (kind, fd, pred)


def test_autograd_function(torch, W, misfit_problem):
    """torch.autograd through DifferentiableSolve equals the explicit adjoint call and the
    direct-system adjoint."""
    import dhs
    prob, P, d = misfit_problem
    ds = W.DifferentiableSolve(prob, tol=1e-13, max_it=800, restart=400)
    c2 = torch.from_numpy(np.concatenate([c.ravel() for c in prob.c2])).cuda().requires_grad_()
    f = torch.from_numpy(np.concatenate([x.ravel() for x in prob.f])).cuda().requires_grad_()
    Pt = torch.from_numpy(P.toarray()).cuda()
    dt = torch.from_numpy(d).cuda()
    u = ds(c2, f)
    J = 0.5 * ((Pt @ u - dt) ** 2).sum()
    J.backward()
    U, J0, gc2_d, gf_d = dhs.adjoint_gradients(prob, P, d)
    assert abs(J.item() - J0) <= 1e-9 * J0
    g1 = c2.grad.cpu().numpy()
    g2 = f.grad.cpu().numpy()
    assert np.linalg.norm(g1 - gc2_d) <= 1e-6 * np.linalg.norm(gc2_d)
    assert np.linalg.norm(g2 - gf_d) <= 1e-6 * np.linalg.norm(gf_d)
    assert ds.forward_stats.converged == 1 and ds.adjoint_stats.converged == 1
    ds.close()


@pytest.mark.parametrize("name,make", [CASES[1], CASES[2], CASES[6]], ids=[CASES[1][0], CASES[2][0], CASES[6][0]])
def test_checkpointed_sweep_matches_whole_trajectory(torch, W, name, make):
    """Forward states recomputed from checkpoints (trajectory_bytes=1) give the gradients of
    the whole stored trajectory."""
    prob = make()
    out = []
    for tb in (0, 1):
        s = W.Solver(prob, trajectory_bytes=tb)
        ti = s.prepare()
        rng = np.random.default_rng(3)
        act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
        u = torch.from_numpy(rng.standard_normal(prob.n_total) * act).cuda()
        g = torch.from_numpy(rng.standard_normal(prob.n_total) * act).cuda()
        lam, gc2, gf, st = s.adjoint(u, g, 1e-10, 40, 40)
        out.append((lam.cpu().numpy(), gc2.cpu().numpy(), gf.cpu().numpy()))
        s.close()
    for a, b in zip(out[0], out[1]):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(a)), name


def test_gradient_vs_finite_differences_inversion_geometry_512(torch, W):
    """The sound-speed inversion workload at full size: disk-in-square 512^2 + 1024x32,
    order 4, omega 20, c = 1 + 0.2 sum of 8 Gaussian bumps, 64 receivers on the circle of
    radius 1.5, data from a medium 5% faster in a Gaussian patch; N_p = 4 periods per
    iteration (forward and adjoint GMRES reach 1e-12 in about 330 wave solves; at N_p = 1
    they need thousands) and the reverse march from checkpoints every 16 steps
    (trajectory_bytes = 1).  Gradients w.r.t. c^2 and f against central finite differences
    in ten random directions (six c^2, four f), 1e-6 relative."""
    prob = G.misfit_problem(nb=512, omega=20.0, seed=0)
    P = G.receiver_matrix(prob, n=64, radius=1.5)
    n = prob.n_total

    def solve(c2=None, f=None, tol=1e-12):
        s = W.Solver(prob, periods=4, trajectory_bytes=1)
        if c2 is not None:
            for gi, c in enumerate(prob.split(c2)):
                s.set_coefficient(gi, c)
        if f is not None:
            for gi, ff in enumerate(prob.split(f)):
                s.set_forcing(gi, ff)
        s.prepare()
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = s.solve(u, W.GMRES, tol=tol, max_it=3000, restart=400)
        assert st.converged == 1, (st.status, st.residual, st.iterations)
        return s, u

    c2 = np.concatenate([c.ravel() for c in prob.c2])
    f = np.concatenate([x.ravel() for x in prob.f])
    _, up = solve(c2=np.concatenate([c.ravel() for c in G.perturbed_c2(prob)]), tol=1e-10)
    d = P @ up.cpu().numpy()
    s, u = solve()
    r = P @ u.cpu().numpy() - d
    g = torch.from_numpy(P.T @ r).cuda()
    lam, gc2, gf, st = s.adjoint(u, g, tol=1e-12, max_it=3000, restart=400)
    assert st.converged == 1
    gc2 = gc2.cpu().numpy()
    gf = gf.cpu().numpy()
    rng = np.random.default_rng(2)

    def J_of(c2v, fv):
        _, u2 = solve(c2=c2v, f=fv)
        rr = P @ u2.cpu().numpy() - d
        return 0.5 * float(rr @ rr)

    for kind in ("c2",) * 6 + ("f",) * 4:
        dirn = rng.standard_normal(n)
        if kind == "c2":
            eps = 1e-5
            jp, jm = J_of(c2 + eps * dirn * c2, f), J_of(c2 - eps * dirn * c2, f)
            pred = float(gc2 @ (dirn * c2))
        else:
            eps = 1e-5 * np.max(np.abs(f))
            jp, jm = J_of(c2, f + eps * dirn), J_of(c2, f - eps * dirn)
            pred = float(gf @ dirn)
        fd = (jp - jm) / (2 * eps)
        assert abs(fd - pred) <= 1e-6 * max(abs(fd), abs(pred)), (kind, fd, pred)
