"""Parity of the three-dimensional fourth-order CUDA path (Cartesian grids, through the C
ABI) with the fourth-order 3D CPU oracle: one iteration in FP64 and in the FP32 march on
grids that span several tiles with ragged tails (distinct spacings per axis, Dirichlet,
Neumann and periodic faces, c(x), the overset box-in-box), and GMRES against the
independently assembled fourth-order discrete Helmholtz solve."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

pytestmark = pytest.mark.gpu
P, N, D = G.BC_PERIODIC, G.BC_NEUMANN, G.BC_DIRICHLET


@pytest.fixture(scope="module")
def env():
    import torch
    from oracle import oracle3 as O3
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    assert torch.cuda.is_available()
    return torch, O3, W


def _forced(g, omega, c2=None):
    return G3.Problem3([g], G3.Interp3.empty(), omega,
                       [G3.gaussian3(g, np.array([0.41, 0.37, 0.33]), 1.0, 40.0)], c2=c2,
                       order=4)


def _box():
    # 45 x 37 x 29 points (tiles of 32 x 8 x 8: ragged on every axis), three spacings
    return _forced(G3.cartesian_grid3("box", (45, 37, 29), (0.0,) * 3, (1.0, 0.8, 0.7),
                                      [D] * 6), 8.0)


def _box_c2():
    g = G3.cartesian_grid3("box", (37, 33, 29), (0.0,) * 3, (1.0, 0.9, 0.8), [D] * 6)
    X = g.coords()
    c = 1.0 + 0.3 * np.exp(-((X[0] - 0.4) ** 2 + (X[1] - 0.6) ** 2 + (X[2] - 0.5) ** 2) / 0.05)
    return _forced(g, 7.0, c2=[c * c])


def _slab(n, bc, omega):
    g = G3.cartesian_grid3("slab", n, (0.0,) * 3, ((n[0] - 1) / n[0], 0.8, 0.9), bc)
    return _forced(g, omega)


CASES = [
    ("dirichlet-box-45x37x29", _box),
    ("neumann-dirichlet-slab", lambda: _slab((40, 20, 36), [P, P, P, P, N, D], 6.0)),
    ("dirichlet-neumann-slab", lambda: _slab((33, 17, 40), [P, P, P, P, D, N], 6.0)),
    ("neumann-slab-axis1", lambda: G3.Problem3(
        [G3.cartesian_grid3("s", (33, 24, 17), (0.0,) * 3, (32 / 33, 1.0, 16 / 17),
                            [P, P, N, N, P, P])], G3.Interp3.empty(), 5.0,
        [np.zeros((17, 24, 33))], order=4)),
    ("periodic-torus", lambda: _forced(
        G3.cartesian_grid3("t", (24, 20, 18), (0.0,) * 3, (23 / 24, 19 / 20, 17 / 18), [P] * 6),
        5.0)),
    ("box-c(x)", _box_c2),
    ("box-in-box-17-15", lambda: G3.box_in_box_problem(nb=17, ni=15, omega=6.0, order=4,
                                                       hole=0.1)),
    ("box-in-box-33-29", lambda: G3.box_in_box_problem(nb=33, ni=29, omega=6.0, order=4,
                                                       hole=0.1)),
]


def _err(got, ref, v, act):
    """Max-norm difference over the active points, relative to the larger of the input's
    and the result's scale (the filter leaves little of a white-noise input)."""
    scale = max(np.max(np.abs(ref)[act]), np.max(np.abs(v)[act]))
    return np.max(np.abs(got - ref)[act]) / scale


def _fp64_bound(M):
    # two evaluation orders of the same sums: 1e-12, or 1e-14 per step beyond 100 steps
    return max(1e-12, 1e-14 * M)


def _fp32_bound(M):
    # the FP32 state is rounded every step: 1e-4 up to 165 steps, growing as M^2 beyond
    return 1e-4 * max(1.0, (M / 165.0) ** 2)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fourth_order_iteration_matches_oracle_3d(env, name, make):
    """One WaveHoltz iteration, forcing on and off, from a random state: FP64 and the FP32
    march against the fourth-order oracle; the time setup (C = sqrt(3)/2) equals the
    oracle's; exactly 2M + 3 launches; inactive points stay 0."""
    torch, O3, W = env
    prob = make()
    orc = O3.Oracle3(prob)
    act = orc.active()
    v = G3.random_state3(prob, 11)
    refs = {f: orc.iterate(v, f) for f in (True, False)}
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    for prec, bound in ((W.FP64, _fp64_bound), (W.FP32, _fp32_bound)):
        s = W.Solver(prob, precision=prec)
        ti = s.prepare()
        assert ti.Nt == orc.time.Nt and ti.M == orc.time.M
        assert ti.dt_max == pytest.approx(orc.time.dt_max, rel=1e-12)
        for forcing in (True, False):
            s.iterate(vi, vo, forcing)
            torch.cuda.synchronize()
            assert s.L.wh_last_launch_count(s.h) == 2 * ti.M + 3
            got = vo.cpu().numpy()
            e = _err(got, refs[forcing], v, act)
            assert e <= bound(ti.M), (name, prec, forcing, e)
            assert np.all(got[~act] == 0.0)
        s.close()


def test_fourth_order_fp32_ignores_temporal_blocking(env):
    """Temporal blocking is a second-order FP32 path: asked for on a fourth-order context it
    blocks no point and the iteration is unchanged."""
    torch, O3, W = env
    prob = _box()
    s = W.Solver(prob, precision=W.FP32)
    s.prepare()
    v = G3.random_state3(prob, 2)
    vi = torch.from_numpy(v).cuda()
    a, b = torch.empty_like(vi), torch.empty_like(vi)
    s.iterate(vi, a, True)
    s.set_tuning(temporal_depth=3, unit_depth=8)
    assert s.get_tuning()["blocked_points"] == 0
    s.iterate(vi, b, True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    s.close()


@pytest.mark.parametrize("name", ["box-in-box", "neumann-dirichlet-slab"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_fourth_order_gmres_matches_direct_solve_3d(env, name, precision):
    """GMRES on the GPU (the FP32 form: FP32 wave solves, then FP64 ones) reaches the
    direct solution of the fourth-order discrete Helmholtz system (13-point stencil, two
    ghost rows per boundary point, width-5 interpolation), assembled on the CPU."""
    import dhs3
    torch, O3, W = env
    prob = (G3.box_in_box_problem(nb=17, ni=15, omega=6.0, order=4, hole=0.1)
            if name == "box-in-box" else _slab((20, 12, 18), [P, P, P, P, N, D], 6.0))
    U = dhs3.solve(prob)
    s = W.Solver(prob, precision=W.FP32 if precision == "fp32" else W.FP64)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-11, max_it=800, restart=200)
    assert st.converged == 1, st.status
    if precision == "fp32":
        assert st.products_fp32 > 0
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    got = u.cpu().numpy()
    assert np.max(np.abs(got - U)[act]) <= 1e-8 * np.max(np.abs(U))
    s.close()


def test_fourth_order_refusals_3d(env):
    """Curvilinear grids and boundary data are refused at fourth order (WH_ERR_ARG)."""
    torch, O3, W = env
    patch = G3.pole_patch_grid("north", 9, 5, 0.5, 0.5, 0.3, 1.0)
    prob = G3.Problem3([patch], G3.Interp3.empty(), 5.0, [np.zeros(patch.mask.shape)], order=4)
    with pytest.raises(W.WHError) as e:
        W.Solver(prob)
    assert e.value.status == -1
    p = G3.with_boundary_data3(G3.unit_cube_problem(9, order=4), lambda x, y, z: 1.0 + x)
    with pytest.raises(W.WHError) as e:
        W.Solver(p)
    assert e.value.status == -1
