"""The three-dimensional oracle on curvilinear grids against the independently assembled
discrete Helmholtz system of tests/dhs3.py (Sec. 6's comparison with the direct solve):
the fixed point on a closed curvilinear grid, and the mapped Laplacian's rows (metric
coefficients, b_k from the metrics, mixed terms) on the sphere-in-box's component grids
(CPU only)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

D, N = G.BC_DIRICHLET, G.BC_NEUMANN


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


@pytest.mark.parametrize("order,bc_in,bc_out", [(2, D, D), (2, N, N), (2, D, N), (4, N, N),
                                               (4, D, D), (4, D, N)])
def test_annular_cylinder_fixed_point_equals_direct_solve(o3, order, bc_in, bc_out):
    """An annular cylinder (periodic in th and z, metric terms b_th = 0, b_r = 1/r in the
    mapped Laplacian): the oracle's fixed point equals the direct solve to 1e-12, and its
    GMRES reaches it."""
    import dhs3
    from oracle.oracle import gmres
    p = G3.annular_cylinder_problem(order=order, bc_in=bc_in, bc_out=bc_out)
    orc = o3.Oracle3(p)
    U = dhs3.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    v, its, hist = gmres(orc, tol=1e-12, restart=200, max_it=400)
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U)), its


def _single(g, order):
    return G3.Problem3([g], G3.Interp3.empty(), 5.0, [np.zeros(g.mask.shape)], order=order)


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("kind", ["patch", "shell"])
def test_mapped_laplacian_rows_equal_direct_assembly(o3, kind, order):
    """On an orthographic pole patch (the mixed a-b term present) and a spherical shell,
    the direct assembly's discretization rows minus omega^2 applied to random data give the
    oracle's c^2 L_h, with c(x) varying."""
    import dhs3
    if kind == "patch":
        g = G3.pole_patch_grid("north", 14, 8, 0.5, 0.5, 0.3, 1.0, order=order)
    else:
        g = G3.shell_grid("shell", 24, 13, 8, 0.5, 0.3, 40.0, 140.0, order=order)
    p = _single(g, order)
    X = g.coords()
    p.c2 = [(1.0 + 0.2 * np.sin(2 * X[0]) * np.cos(X[2])) ** 2]
    orc = o3.Oracle3(p)
    A, rhs, L = dhs3.assemble(p)
    u = np.random.default_rng(order).standard_normal(L.N)
    Au = A @ u - p.omega ** 2 * u
    lap = orc.apply_lap(0, u.reshape(orc.ext_shape(0))).ravel()
    gh = g.ghosts(order)
    disc = np.zeros(orc.ext_shape(0), bool)
    disc[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]] = g.mask == G.DISC
    disc = disc.ravel()
    assert np.max(np.abs(Au[disc] - lap[disc])) < 1e-11 * np.max(np.abs(lap[disc]))


def test_annular_cylinder_dirichlet_solution_fourth_order(o3):
    """u = (r^2 - a^2)(b^2 - r^2) cos(2 th) cos(2 pi z) vanishes on both walls; with
    f = Lap u + omega^2 u the solution on the curvilinear annular cylinder (order-4
    Dirichlet compatibility rows with a_nn and b_n) converges at fourth order."""
    import math
    from oracle.oracle import gmres
    a, b, om = 0.3, 0.6, 4.0
    errs = []
    for s_ in (1, 2):
        p = G3.annular_cylinder_problem(nth=32 * s_, nr=8 * s_ + 1, nz=10 * s_, r_in=a, r_out=b,
                                        order=4, omega=om)
        x, y, z = p.grids[0].coords()
        r, th = np.hypot(x, y), np.arctan2(y, x)
        R = (r * r - a * a) * (b * b - r * r)
        R1 = -4 * r ** 3 + 2 * (a * a + b * b) * r
        R2 = -12 * r * r + 2 * (a * a + b * b)
        ang = np.cos(2 * th) * np.cos(2 * np.pi * z)
        u = R * ang
        lap = (R2 + R1 / r - 4 * R / (r * r) - (2 * np.pi) ** 2 * R) * ang
        p.f = [lap + om ** 2 * u]
        v, its, hist = gmres(o3.Oracle3(p), tol=1e-12, restart=200, max_it=600)
        errs.append(np.max(np.abs(v - u.ravel())))
    assert 3.6 < math.log2(errs[0] / errs[1]) < 4.5, errs
