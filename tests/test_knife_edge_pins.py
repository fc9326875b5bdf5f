"""The knife-edge geometry (Sec. 6's knife edge): the generator's outline and metrics are
checked against what they must satisfy, the oracle's fixed point on it against the
independent direct solve, the library's host-side validation takes it, and implicit
time-stepping (Sec. 4.5) reaches the same solution with far fewer time steps there
(CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

SMALL = dict(j=8, omega=20.0, width=0.04, height=0.3, b=300.0)


def test_outline_closes_with_continuous_curvature():
    """The outline leaves the right side upward, turns by pi over the tip and meets the
    left side at (-width/2, y_s) going down; the apex is at (0, height); it is
    parametrized by arclength (|d gamma / d sigma| = 1) with d phi / d sigma = kappa, and
    kappa vanishes where the tip meets the sides."""
    ko = G.KnifeOutline(0.02, 0.5)
    x, y, phi, k = ko.frame(np.array([ko.ys, ko.ys + ko.ell / 2, ko.ys + ko.ell]))
    assert (x[0], y[0], phi[0]) == pytest.approx((0.01, ko.ys, math.pi / 2), abs=1e-15)
    assert (x[1], y[1], phi[1]) == pytest.approx((0.0, 0.5, math.pi), abs=1e-14)
    assert (x[2], y[2], phi[2]) == pytest.approx((-0.01, ko.ys, 1.5 * math.pi), abs=1e-14)
    assert k[0] == pytest.approx(0.0, abs=1e-12) and k[2] == pytest.approx(0.0, abs=1e-12)
    assert k[1] == pytest.approx(ko.kmax, rel=1e-14)
    sig = np.linspace(ko.ys - 0.01, ko.ys + ko.ell + 0.01, 4001)
    ds = 1e-6
    xp, yp, php, _ = ko.frame(sig + ds)
    xm, ym, phm, _ = ko.frame(sig - ds)
    _, _, _, ks = ko.frame(sig)
    speed = np.hypot(xp - xm, yp - ym) / (2 * ds)
    assert np.max(np.abs(speed - 1.0)) < 1e-8
    assert np.max(np.abs((php - phm) / (2 * ds) - ks)) < 1e-5 * ko.kmax
    assert ko.S == pytest.approx(2 * ko.ys + ko.ell, rel=1e-15)


def test_knife_grid_metrics_invert_the_mapping():
    """The analytic inverse metrics of the knife grid equal the inverse of the mapping's
    Jacobian (central differences of x(t0, t1)) at interior and ghost points, and the grid
    is orthogonal."""
    grids, _, ko = G.knife_edge(j=8, width=0.04, height=0.3)
    K = grids[1]
    m = K.mapping["knife"]
    rng = np.random.default_rng(0)
    t0 = rng.uniform(-0.01, 1.01, 200)
    t1 = rng.uniform(-0.1, 1.0, 200)
    e = 1e-7
    x0p, y0p = m.xy(t0 + e, t1)
    x0m, y0m = m.xy(t0 - e, t1)
    x1p, y1p = m.xy(t0, t1 + e)
    x1m, y1m = m.xy(t0, t1 - e)
    J = np.stack([[(x0p - x0m) / (2 * e), (x1p - x1m) / (2 * e)],
                  [(y0p - y0m) / (2 * e), (y1p - y1m) / (2 * e)]])  # dx/dt
    rx = np.stack(m.rx(t0, t1))  # dt0/dx, dt0/dy, dt1/dx, dt1/dy
    for q in range(t0.size):
        inv = np.linalg.inv(J[:, :, q])
        assert np.allclose(rx[:, q], inv.ravel(), rtol=1e-6, atol=1e-6 * np.abs(inv).max())
    assert np.max(np.abs((J[:, 0] * J[:, 1]).sum(axis=0)) /
                  (np.linalg.norm(J[:, 0], axis=0) * np.linalg.norm(J[:, 1], axis=0))) < 1e-6


@pytest.mark.parametrize("order", [2, 4])
def test_knife_edge_generator_invariants(order):
    """Explicit interpolation (donors are discretization or Dirichlet points), each
    interpolation point listed once, weights summing to 1, no discretization point whose
    stencil reads an unused point, and every ghost rule (at order 4: each Dirichlet point
    of a Dirichlet side) reading discretization or Dirichlet points only."""
    p = G.knife_edge_problem(order=order, **SMALL)
    it = p.interp
    G.check_explicit_interp(p.grids, it, order)
    assert np.allclose(it.wx.sum(axis=1), 1.0) and np.allclose(it.wy.sum(axis=1), 1.0)
    keys = set(zip(it.recv_grid.tolist(), it.recv_i.tolist(), it.recv_j.tolist()))
    assert len(keys) == it.n == sum(int((g.mask == G.INTERP).sum()) for g in p.grids)
    r = order // 2
    for g in p.grids:
        n1, n0 = g.mask.shape
        pad = np.pad(g.mask, r, constant_values=-1)
        disc = g.mask == G.DISC
        for a in range(-r, r + 1):
            for b in range(-r, r + 1):
                nb = pad[r + a:r + a + n1, r + b:r + b + n0]
                assert not np.any(disc & (nb == G.UNUSED)), g.name
        if order == 4:
            for side in range(4):
                if g.bc[side] != G.BC_DIRICHLET:
                    continue
                ax, hi = side // 2, side % 2
                m = np.moveaxis(g.mask, 1 - ax, 0)  # axis `ax` first: (normal, tangential)
                m = m[::-1] if hi else m
                rows = m[0] == G.DIRICHLET
                inward = m[1:4][:, rows]
                assert np.all((inward == G.DISC) | (inward == G.DIRICHLET)), (g.name, side)


@pytest.mark.parametrize("order", [2, 4])
def test_knife_edge_fixed_point_equals_direct_solve(order):
    """Sec. 6: on the knife edge the oracle's WaveHoltz fixed point is the direct solution
    of the discrete Helmholtz system (tests/dhs.py), and GMRES reaches it."""
    import dhs
    from oracle.oracle import Oracle, gmres
    p = G.knife_edge_problem(order=order, **SMALL)
    orc = Oracle(p)
    U = dhs.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    v, its, hist = gmres(orc, tol=1e-12, restart=200, max_it=600)
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U)), its


def test_knife_edge_implicit_time_stepping():
    """Sec. 4.5 on the knife edge: the explicit step is bound by the smallest cells (at the
    tip), the implicit one is not; with N_ITS = 10 the implicit map has the same fixed
    point, and GMRES reaches it with several times fewer time steps."""
    import dhs
    from oracle.implicit import ImplicitOracle
    from oracle.oracle import Oracle, gmres
    p = G.knife_edge_problem(order=2, **SMALL)
    U = dhs.solve(p)
    imp = ImplicitOracle(p, n_its=10)
    act = imp.active()
    assert np.max(np.abs(imp.iterate(U, True) - U)[act]) < 1e-11 * np.max(np.abs(U))
    _, its_i, _ = gmres(imp, tol=1e-10, restart=200, max_it=600)
    orc = Oracle(p)
    _, its_e, _ = gmres(orc, tol=1e-10, restart=200, max_it=600)
    assert orc.time.M > 8 * imp.time["M"]
    assert its_e * orc.time.M > 4 * its_i * imp.time["M"], (its_e, orc.time.M, its_i)


def test_knife_edge_taken_by_the_library_host_checks():
    """The library's host-side validation (grid descriptions and interpolation data) takes
    the knife-edge grids at orders 2 and 4 (no device work)."""
    from host_checks import library_takes
    for order in (2, 4):
        library_takes(G.knife_edge_problem(order=order, **SMALL))


def test_knife_edge_refuses_grids_that_do_not_fit():
    """A knife grid whose ghost lines would fold at the tip, or whose outer lines would
    reach the top wall, is refused."""
    with pytest.raises(ValueError):
        G.knife_edge(j=8, width=0.01, height=0.3)
    with pytest.raises(ValueError):
        G.knife_edge(j=16)
