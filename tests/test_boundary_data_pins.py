"""Inhomogeneous Dirichlet data (boundary value g on Dirichlet sides, the first item of the
paper's note that g != 0 needs further work, Sec. 4.4): the oracle against what the
mathematics fixes -- a manufactured solution that is non-zero on the boundary converges
at the order of the scheme, the WaveHoltz fixed point equals the direct solution of the
discrete Helmholtz system with U = g on Dirichlet points, and the zero-forcing map does
not see g."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G


def _manufactured(kind):
    if kind == "square":
        fn = lambda x, y: np.sin(np.pi * x + 0.3) * np.sin(2 * np.pi * y + 0.2)
        k2 = 5 * np.pi ** 2
    else:  # channel: periodic in x on [0, 1), Dirichlet walls
        fn = lambda x, y: np.cos(2 * np.pi * x + 0.1) * np.sin(np.pi * y + 0.4)
        k2 = 5 * np.pi ** 2
    return fn, k2


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("kind", ["square", "channel"])
def test_manufactured_solution_with_boundary_data(oracle_mod, order, kind):
    """u non-zero on the Dirichlet sides, f = (omega^2 - k^2) u: the oracle's WaveHoltz
    solution converges to u at order p."""
    om = 3.0
    fn, k2 = _manufactured(kind)
    errs = []
    for n in (17, 33):
        prob = G.unit_square_problem(n, order, om) if kind == "square" else \
            G.channel_problem(n, order, om, bc=G.BC_DIRICHLET)
        X, Y = prob.grids[0].xy
        prob.f = [(om ** 2 - k2) * fn(X, Y)]
        prob = G.with_boundary_data(prob, fn)
        orc = oracle_mod.Oracle(prob)
        v, its, hist = oracle_mod.gmres(orc, tol=1e-12, restart=100, max_it=300)
        errs.append(np.max(np.abs(v.reshape(n, n) - fn(X, Y))))
    assert errs[1] < 1e-2
    assert math.log2(errs[0] / errs[1]) > order - 0.3, errs


def _disk_with_g(order):
    p = G.disk_problem(nb=48, nth=96, nr=10, order=order, omega=4.0, width=0.8, r_cut=0.75)
    return G.with_boundary_data(p, lambda x, y: 0.3 * np.cos(1.3 * x + 0.4 * y) + 0.1 * y)


CASES = [
    ("square-o2", lambda: G.with_boundary_data(G.unit_square_problem(16, 2, 10.0),
                                               lambda x, y: np.cos(3 * x + 2 * y))),
    ("square-o4", lambda: G.with_boundary_data(G.unit_square_problem(20, 4, 10.0),
                                               lambda x, y: np.cos(3 * x + 2 * y))),
    ("channel-o4", lambda: G.with_boundary_data(
        G.channel_problem(20, 4, 5.0, bc=G.BC_DIRICHLET),
        lambda x, y: np.sin(2 * np.pi * x) * (1 + y))),
    ("disk-o2", lambda: _disk_with_g(2)),
    ("disk-o4", lambda: _disk_with_g(4)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_fixed_point_equals_direct_solve_with_boundary_data(oracle_mod, name, make):
    import dhs
    prob = make()
    orc = oracle_mod.Oracle(prob)
    U = dhs.solve(prob)
    assert np.max(np.abs(U)) > 0.1  # the data reach the solution
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)) < 1e-11 * np.max(np.abs(U))
    v, its, hist = oracle_mod.gmres(orc, tol=1e-13, restart=200, max_it=400)
    act = orc.active()
    assert np.max(np.abs(v - U)[act]) < 1e-9 * np.max(np.abs(U))


def test_zero_forcing_map_ignores_boundary_data(oracle_mod):
    base = G.unit_square_problem(20, 4, 10.0)
    withg = G.with_boundary_data(base, lambda x, y: np.cos(3 * x + 2 * y))
    v = G.random_state(base, 3)
    a = oracle_mod.Oracle(base).iterate(v, False)
    b = oracle_mod.Oracle(withg).iterate(v, False)
    assert np.array_equal(a, b)
    # the forced map is affine in g: W_h(v, f, g) - W_h(v, f, 0) is linear in g
    c = oracle_mod.Oracle(withg).iterate(v, True) - oracle_mod.Oracle(base).iterate(v, True)
    twice = G.with_boundary_data(base, lambda x, y: 2 * np.cos(3 * x + 2 * y))
    d = oracle_mod.Oracle(twice).iterate(v, True) - oracle_mod.Oracle(base).iterate(v, True)
    assert np.max(np.abs(d - 2 * c)) < 1e-12 * np.max(np.abs(d))


def test_curvilinear_dirichlet_data_at_order_4_is_refused(oracle_mod):
    p = G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75)
    p = G.with_boundary_data(p, lambda x, y: 1.0 + 0 * x)
    p.grids = list(p.grids)
    A = G.annulus_grid("annulus", 96, 10, 0.5, 0.8, 1.5, 4, inner_bc=G.BC_DIRICHLET)
    p.grids[1] = A
    p.g = [p.g[0], np.where(A.mask == G.DIRICHLET, 1.0, 0.0)]
    with pytest.raises(ValueError):
        oracle_mod.Oracle(p)


# ------------------------------------------------------------------ three dimensions

def test_manufactured_solution_with_boundary_data_3d():
    """Unit cube, Dirichlet walls carrying u: u = sin(pi x + 0.3) sin(pi y + 0.5)
    sin(pi z + 0.2), f = (omega^2 - 3 pi^2) u; the 3D oracle's solution converges at
    second order."""
    import math
    from paper_2504_03074_gb300 import grids3 as G3
    from oracle import oracle3 as O3
    om = 3.0
    fn = lambda x, y, z: np.sin(np.pi * x + 0.3) * np.sin(np.pi * y + 0.5) * np.sin(np.pi * z + 0.2)
    errs = []
    for n in (9, 17):
        prob = G3.unit_cube_problem(n, omega=om)
        X = prob.grids[0].coords()
        prob.f = [(om ** 2 - 3 * np.pi ** 2) * fn(X[0], X[1], X[2])]
        prob = G3.with_boundary_data3(prob, fn)
        orc = O3.Oracle3(prob)
        from oracle.oracle import gmres
        v, its, hist = gmres(orc, tol=1e-12, restart=100, max_it=300)
        errs.append(np.max(np.abs(v - fn(X[0], X[1], X[2]).ravel())))
    assert math.log2(errs[0] / errs[1]) > 1.7, errs


@pytest.mark.parametrize("make", ["cube", "box_in_box"])
def test_fixed_point_equals_direct_solve_with_boundary_data_3d(make):
    import dhs3
    from paper_2504_03074_gb300 import grids3 as G3
    from oracle import oracle3 as O3
    fn = lambda x, y, z: 0.5 * np.cos(1.1 * x + 0.6 * y - 0.4 * z) + 0.1 * z
    base = G3.unit_cube_problem(10, omega=6.0) if make == "cube" else G3.box_in_box_problem()
    prob = G3.with_boundary_data3(base, fn)
    orc = O3.Oracle3(prob)
    U = dhs3.solve(prob)
    assert np.max(np.abs(U)) > 0.1
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)) < 1e-11 * np.max(np.abs(U))
    v = G3.random_state3(base, 1)
    a = O3.Oracle3(base).iterate(v, False)
    assert np.array_equal(a, orc.iterate(v, False))  # the zero-forcing map ignores g


# ------------------------------------------------------------------ Neumann data (2D)

def _u(x, y):
    return np.cos(2 * np.pi * x) * (np.cos(3 * y) + y * y)


def _grad_u(x, y):
    return (-2 * np.pi * np.sin(2 * np.pi * x) * (np.cos(3 * y) + y * y),
            np.cos(2 * np.pi * x) * (-3 * np.sin(3 * y) + 2 * y))


def _lap_u(x, y):
    return -4 * np.pi ** 2 * _u(x, y) + np.cos(2 * np.pi * x) * (-9 * np.cos(3 * y) + 2)


@pytest.mark.parametrize("order", [2, 4])
def test_manufactured_solution_with_neumann_data(oracle_mod, order):
    """dU/dn = gn on the walls of a periodic channel (outward normal), with a solution
    whose normal derivative does not vanish there: the WaveHoltz solution converges at
    order p."""
    om, errs = 3.0, []
    for n in (24, 48):
        p = G.channel_problem(n, order, om, bc=G.BC_NEUMANN)
        x, y = p.grids[0].xy
        p.f = [_lap_u(x, y) + om ** 2 * _u(x, y)]
        p = G.with_neumann_data(p, _grad_u)
        v, its, hist = oracle_mod.gmres(oracle_mod.Oracle(p), tol=1e-12, restart=200,
                                        max_it=600)
        errs.append(np.max(np.abs(v.reshape(x.shape) - _u(x, y))))
    rate = math.log2(errs[0] / errs[1])
    assert order - 0.3 < rate < order + 0.4, errs


def _disk_c2():
    p = G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75)
    p.c2 = [G.bumps_c2(g.xy, [(0.6, 0.4), (-0.5, -0.6)]) for g in p.grids]
    return p


NEUMANN_CASES = [
    ("disk-o4-c(x)", _disk_c2),
    ("channel-o2", lambda: G.channel_problem(30, 2, 5.0, bc=G.BC_NEUMANN)),
    ("channel-o4", lambda: G.channel_problem(30, 4, 5.0, bc=G.BC_NEUMANN)),
    ("sheared-channel-o2", lambda: G.sheared_channel_problem(shear=0.4)),
]


@pytest.mark.parametrize("name,make", NEUMANN_CASES, ids=[c[0] for c in NEUMANN_CASES])
def test_fixed_point_equals_direct_solve_with_neumann_data(oracle_mod, name, make):
    """The fixed point with Neumann data equals the direct solve whose Neumann rows carry
    gn on their right sides (tests/dhs.py); the zero-forcing map ignores gn."""
    import dhs
    base = make()
    p = G.with_neumann_data(base, _grad_u)
    assert max(np.max(np.abs(x)) for x in p.gn) > 0.3
    orc = oracle_mod.Oracle(p)
    U = dhs.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    v = G.random_state(base, 2)
    assert np.array_equal(orc.iterate(v, False), oracle_mod.Oracle(base).iterate(v, False))


def test_overset_disk_with_dirichlet_and_neumann_data_fourth_order(oracle_mod):
    """Disk-in-square at order 4 with Dirichlet data on the box and Neumann data on the
    disk (the annulus's curvilinear side, outward normal pointing into the disk): fixed
    point equal to the direct solve, and a manufactured solution converging at fourth
    order through the overset interpolation (finer level on the all-cores build)."""
    import dhs

    def u(x, y):
        return np.cos(1.5 * x + 0.5 * y) + 0.3 * np.sin(0.7 * x - 1.1 * y)

    def grad(x, y):
        return (-1.5 * np.sin(1.5 * x + 0.5 * y) + 0.21 * np.cos(0.7 * x - 1.1 * y),
                -0.5 * np.sin(1.5 * x + 0.5 * y) - 0.33 * np.cos(0.7 * x - 1.1 * y))

    def lap(x, y):
        return -2.5 * np.cos(1.5 * x + 0.5 * y) - 0.3 * 1.7 * np.sin(0.7 * x - 1.1 * y)

    om, errs = 4.0, []
    for s in (1, 2):
        p = G.disk_problem(nb=48 * s, nth=96 * s, nr=10 * s, order=4, omega=om, width=0.8,
                           r_cut=0.75)
        p.f = [lap(*g.xy) + om ** 2 * u(*g.xy) for g in p.grids]
        p = G.with_neumann_data(G.with_boundary_data(p, u), grad)
        orc = oracle_mod.Oracle(p, openmp=s > 1)
        if s == 1:
            U = dhs.solve(p)
            assert np.max(np.abs(orc.iterate(U, True) - U)[orc.active()]) < \
                1e-12 * np.max(np.abs(U))
        v, its, hist = oracle_mod.gmres(orc, tol=1e-12, restart=300, max_it=900)
        ref = np.concatenate([u(*g.xy).ravel() for g in p.grids])
        errs.append(np.max(np.abs(v - ref)[orc.active()]))
    assert 3.5 < math.log2(errs[0] / errs[1]) < 4.5, errs


def test_library_refuses_neumann_data():
    """The GPU binding takes no Neumann data and says so (before any device work)."""
    from paper_2504_03074_gb300 import waveholtz as W
    p = G.with_neumann_data(G.channel_problem(16, 2, 5.0, bc=G.BC_NEUMANN), _grad_u)
    with pytest.raises(ValueError):
        W.Solver(p)
