"""Inhomogeneous Dirichlet data on the GPU (wh_set_boundary_data): iterations equal the
oracle's in every launch layout and both precisions, GMRES reaches the direct solution of
the discrete Helmholtz system with U = g, batches carry each instance's data, the exact
deflated inflation stays exact, and the calls that do not take g refuse it."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu
TOL = 1e-12


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


def _g(x, y):
    return 0.4 * np.cos(1.3 * x + 0.7 * y) + 0.2 * y


def rel_err(a, b, act):
    return np.max(np.abs(a - b)[act]) / np.max(np.abs(b)[act])


def gpu_iterate(torch, s, v, forcing):
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    s.iterate(vi, vo, forcing)
    torch.cuda.synchronize()
    return vo.cpu().numpy()


CASES = [
    ("square64-o2", lambda: G.with_boundary_data(G.unit_square_problem(64, 2, 10.0), _g)),
    ("square37-o4", lambda: G.with_boundary_data(G.unit_square_problem(37, 4, 10.0, seed=2), _g)),
    ("channel40-o4", lambda: G.with_boundary_data(
        G.channel_problem(40, 4, 5.0, bc=G.BC_DIRICHLET),
        lambda x, y: np.sin(2 * np.pi * x) * (1 + y))),
    ("disk-o4", lambda: G.with_boundary_data(
        G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0), _g)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_iteration_with_boundary_data(torch, W, oracle_mod, name, make):
    """FP64 at 1e-12 in every launch layout (persistent; graph with the gather folded or
    separate, tiles by ticket or stride); FP32 (TMA-staged and plain) within 1e-4."""
    prob = make()
    orc = oracle_mod.Oracle(prob)
    act = orc.active()
    v = G.random_state(prob, 7)
    refs = {f: orc.iterate(v, f) for f in (True, False)}
    for prec, tol in ((W.FP64, TOL), (W.FP32, 1e-4)):
        s = W.Solver(prob, precision=prec)
        s.prepare()
        layouts = [(W.PERSISTENT, -1, -1, -1, -1), (W.GRAPH, 1, -1, 0, 1), (W.GRAPH, 0, 1, 0, 1),
                   (W.GRAPH, 0, 0, 0, 0)]
        if prec == W.FP32:
            layouts += [(W.GRAPH, 1, -1, 1, 1), (W.GRAPH, 0, -1, 1, 1)]
        for lay in layouts:
            s.set_tuning(*lay)
            for f in (True, False):
                got = gpu_iterate(torch, s, v, f)
                assert rel_err(got, refs[f], act) <= tol, (name, prec, lay, f)
                assert np.all(got[~act] == 0.0)
        s.close()


@pytest.mark.parametrize("name", ["square-o4", "disk-o4"])
def test_gmres_with_boundary_data_reaches_direct_solution(torch, W, name):
    import dhs
    prob = G.with_boundary_data(
        G.unit_square_problem(24, 4, 10.0) if name == "square-o4" else
        G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75), _g)
    U = dhs.solve(prob)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    for prec in (W.FP64, W.FP32):
        s = W.Solver(prob, precision=prec)
        s.prepare()
        u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
        st = s.solve(u, W.GMRES, tol=1e-12, max_it=600, restart=200)
        assert st.converged == 1, (st.status, st.residual)
        assert rel_err(u.cpu().numpy(), U, act) < 1e-9
        # the Dirichlet points carry the data
        dmask = np.concatenate([(g.mask == G.DIRICHLET).ravel() for g in prob.grids])
        gvec = np.concatenate([x.ravel() for x in prob.g])
        assert np.max(np.abs(u.cpu().numpy()[dmask] - gvec[dmask])) < 1e-9
        s.close()


def test_batch_with_boundary_data(torch, W, oracle_mod):
    probs = [G.with_boundary_data(G.unit_square_problem(n, 4, om, seed=k),
                                  lambda x, y, a=a: a * np.cos(2 * x + y))
             for k, (n, om, a) in enumerate(((24, 6.0, 0.5), (32, 9.0, -1.0), (28, 7.0, 2.0)))]
    bp = G.batch_problems(probs)
    s = W.Solver(bp)
    s.prepare()
    vs = [G.random_state(p, 20 + k) for k, p in enumerate(probs)]
    got = gpu_iterate(torch, s, np.concatenate(vs), True)
    off = 0
    for k, p in enumerate(probs):
        orc = oracle_mod.Oracle(p)
        ref = orc.iterate(vs[k], True)
        assert rel_err(got[off:off + p.n_total], ref, orc.active()) <= TOL, k
        off += p.n_total


def test_exact_deflated_inflation_with_boundary_data(torch, W):
    """The exact inflation U = v + Q (I - T)^{-1} Q^T W_h(v, f, g) holds for any affine map,
    so a deflated GMRES with boundary data reaches the direct solution."""
    import dhs
    prob = G.with_boundary_data(
        G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75), _g)
    U = dhs.solve(prob)
    s = W.Solver(prob)
    s.prepare()
    Q, T, beta, lam2, st = s.eigs(4, tol=1e-11, max_products=3000)
    assert st.converged == 1
    s.set_deflation_basis(Q, T)
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    std = s.solve(u, W.GMRES, tol=1e-12, max_it=600, restart=200)
    assert std.converged == 1
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    assert rel_err(u.cpu().numpy(), U, act) < 1e-8


def test_calls_that_take_no_boundary_data_refuse_it(torch, W):
    prob = G.with_boundary_data(G.unit_square_problem(24, 4, 10.0), _g)
    s = W.Solver(prob)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WHError) as e:
        s.adjoint(u, u, tol=1e-8, max_it=10, restart=10)
    assert e.value.status == -3
    phi = torch.zeros((1, prob.n_total), dtype=torch.float64, device="cuda")
    phi[0, prob.n_total // 2] = 1.0
    s.set_deflation(phi, np.array([3.0]))
    with pytest.raises(W.WHError) as e:
        s.solve(u, W.FPI, tol=1e-8, max_it=5)
    assert e.value.status == -3
    s.set_deflation(None)
    # removing the data restores the plain problem
    s.set_boundary_data(0, None)
    s.prepare()
    s.solve(u, W.FPI, tol=1e-30, max_it=2)
    # curvilinear Dirichlet sides at order 4 do not take data
    A = G.annulus_grid("annulus", 96, 10, 0.5, 0.8, 1.5, 4, inner_bc=G.BC_DIRICHLET)
    p2 = G.Problem([A], G.Interp.empty(4), 4, 4.0, [np.zeros(A.mask.shape)])
    s2 = W.Solver(p2)
    with pytest.raises(W.WHError) as e:
        s2.set_boundary_data(0, np.ones(A.mask.shape))
    assert e.value.status == -7



# ------------------------------------------------------------------ three dimensions

def _g3(x, y, z):
    return 0.5 * np.cos(1.1 * x + 0.6 * y - 0.4 * z) + 0.1 * z


@pytest.mark.parametrize("make", ["cube", "box_in_box"])
def test_iteration_with_boundary_data_3d(torch, W, make):
    """3D contexts: FP64 at 1e-12 and the FP32 march within 1e-4 of the 3D oracle, forcing
    on and off; on the cube also the temporally blocked FP32 march (the units near the
    Dirichlet walls with data take single steps) within the same bound."""
    from paper_2504_03074_gb300 import grids3 as G3
    from oracle import oracle3 as O3
    base = G3.unit_cube_problem(70, omega=6.0) if make == "cube" else G3.box_in_box_problem()
    prob = G3.with_boundary_data3(base, _g3)
    orc = O3.Oracle3(prob)
    act = orc.active()
    v = G3.random_state3(prob, 5)
    refs = {f: orc.iterate(v, f) for f in (True, False)}
    for prec, tol in ((W.FP64, TOL), (W.FP32, 1e-4)):
        s = W.Solver(prob, precision=prec)
        s.prepare()
        depths = (1, 3) if (prec == W.FP32 and make == "cube") else (-1,)
        for K in depths:
            if K != -1:
                s.set_tuning(temporal_depth=K, unit_depth=8)
                assert (s.get_tuning()["blocked_points"] > 0) == (K > 1)
            for f in (True, False):
                got = gpu_iterate(torch, s, v, f)
                assert rel_err(got, refs[f], act) <= tol, (make, prec, K, f)
        s.close()


def test_gmres_with_boundary_data_3d(torch, W):
    import dhs3
    from paper_2504_03074_gb300 import grids3 as G3
    prob = G3.with_boundary_data3(G3.box_in_box_problem(), _g3)
    U = dhs3.solve(prob)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    for prec in (W.FP64, W.FP32):
        s = W.Solver(prob, precision=prec)
        s.prepare()
        u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
        st = s.solve(u, W.GMRES, tol=1e-11, max_it=800, restart=200)
        assert st.converged == 1, (st.status, st.residual)
        assert rel_err(u.cpu().numpy(), U, act) < 1e-8
        s.close()
