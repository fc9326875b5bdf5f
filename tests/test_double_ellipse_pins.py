"""Pins for the double ellipse, Penrose's unilluminable room (Sec. 6): the wall outlines
against the closed-form ellipse geometry, the overset grid's invariants, the oracle's fixed
point against the independent direct solve, and fourth-order convergence to a manufactured
solution that vanishes on every wall (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G


@pytest.fixture(scope="module")
def orc_mod():
    from oracle import oracle
    return oracle


@pytest.fixture(scope="module")
def rooms():
    return {order: G.double_ellipse_problem(j=2, order=order) for order in (2, 4)}


def test_room_outlines_match_the_ellipses():
    """The wall outlines lie on the room's ellipses and segments; their lengths equal the
    complete elliptic integral's half perimeters (scipy.special.ellipe, independent of the
    arclength table); the tangent is the derivative of the point along sigma and continuous
    at the joins; the curvature takes its closed-form values at the axis ends."""
    from scipy.special import ellipe
    room = G.DoubleEllipseRoom()
    f = room.f
    y0 = 5.7
    left, right, top, bottom = room.outlines(y0)
    for o in (left, right):
        assert abs(o.S - 2 * 6.0 * ellipe(1 - (3.0 / 6.0) ** 2)) < 1e-10
    for o in (top, bottom):
        assert abs(o.S - (2 * 2.0 * ellipe(1 - (1.0 / 2.0) ** 2) + 2 * (y0 - f))) < 1e-10
    sig = np.linspace(0.0, left.S, 20001)
    x, y, tx, ty, kap = left.frame(sig)
    assert np.max(np.abs(((x + 2) / 3) ** 2 + (y / 6) ** 2 - 1)) < 1e-12 and np.all(x <= -2 + 1e-12)
    assert np.max(np.abs(np.gradient(x, sig)[1:-1] - tx[1:-1])) < 1e-6
    assert np.max(np.abs(np.gradient(y, sig)[1:-1] - ty[1:-1])) < 1e-6
    # curvature b/a^2 at the ends of the major (vertical) axis, a/b^2 at x = -5
    assert abs(kap[0] + 6.0 / 9.0) < 1e-10 and abs(kap[-1] + 6.0 / 9.0) < 1e-10
    assert abs(left.frame(np.array([left.S / 2]))[4][0] + 3.0 / 36.0) < 1e-10
    sig = np.linspace(0.0, top.S, 20001)
    x, y, tx, ty, kap = top.frame(sig)
    seg = np.abs(np.abs(x) - 2.0) < 1e-12
    cap = ~seg
    assert np.all(y[seg] >= f - 1e-12) and np.all(y[seg] <= y0 + 1e-12)
    assert np.max(np.abs((x[cap] / 2) ** 2 + (y[cap] - f) ** 2 - 1)) < 1e-12
    assert np.all(y[cap] <= f + 1e-12)
    for s0 in top.starts[1:-1]:  # tangent continuous, curvature 0 -> a1/b1^2 = 2 at the foci
        e = np.array([s0 - 1e-9, s0 + 1e-9])
        _, _, tx2, ty2, k2 = top.frame(e)
        assert abs(tx2[0] - tx2[1]) < 1e-8 and abs(ty2[0] - ty2[1]) < 1e-8
        assert abs(k2).min() < 1e-12 and abs(abs(k2).max() - 2.0) < 1e-8
    # the bottom of the top cap: curvature b1/a1^2 = 1/4, turning counterclockwise
    assert abs(top.frame(np.array([top.S / 2]))[4][0] - 0.25) < 1e-10


@pytest.mark.parametrize("order", [2, 4])
def test_room_generator_invariants(rooms, order):
    """Five grids; every wall grid is orthogonal with its wall row on the room's walls and
    its outer order/2 rows interpolated; the large half-ellipse grids end on the alcove
    segments x = -+2 (Dirichlet end columns between the foci and y = +-6); background points
    in use lie inside the room, at least cut W from every wall; donor stencils of width
    order + 1 hold discretization or Dirichlet points only; weights sum to 1 per axis;
    every interpolation point is listed once."""
    p = rooms[order]
    room = G.DoubleEllipseRoom()
    assert [g.name for g in p.grids] == ["background", "left", "right", "top", "bottom"]
    G.check_explicit_interp(p.grids, p.interp, order)
    it = p.interp
    for w in (it.wx, it.wy):
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
    keys = set(zip(it.recv_grid.tolist(), it.recv_i.tolist(), it.recv_j.tolist()))
    assert len(keys) == it.n
    g1 = order // 2
    for g in p.grids[1:]:
        X, Y = g.xy
        r = g.rx
        assert np.max(np.abs(r[0] * r[2] + r[1] * r[3])) < 1e-12 * np.max(np.abs(r))
        assert np.all(g.mask[0] == G.DIRICHLET) and np.all(g.mask[-g1:] == G.INTERP)
        x0, y0 = X[0], Y[0]
        if g.name in ("left", "right"):
            s = -1.0 if g.name == "left" else 1.0
            assert np.max(np.abs(((x0 - 2 * s) / 3) ** 2 + (y0 / 6) ** 2 - 1)) < 1e-12
            for col in (0, -1):
                assert np.max(np.abs(X[:, col] - 2 * s)) < 1e-12
                assert np.all((np.abs(Y[:, col]) >= room.f) & (np.abs(Y[:, col]) <= 6 + 1e-12))
                assert np.all(g.mask[:-g1, col] == G.DIRICHLET)
        else:
            on_seg = np.abs(np.abs(x0) - 2) < 1e-12
            cy = room.f if g.name == "top" else -room.f
            assert np.max(np.abs((x0[~on_seg] / 2) ** 2 + (y0[~on_seg] - cy) ** 2 - 1)) < 1e-12
            assert np.all(g.mask[1:, :g1] == G.INTERP) and np.all(g.mask[1:, -g1:] == G.INTERP)
    B = p.grids[0]
    XB, YB = B.xy
    disc = B.mask == G.DISC
    assert np.all(room.inside(XB[disc], YB[disc]))
    W = p.grids[1].xy[1][-1, 0] - p.grids[1].xy[1][0, 0]
    for g in p.grids[1:]:
        X, Y = g.xy
        d2 = (XB[disc][:, None] - X[0][None, :]) ** 2 + (YB[disc][:, None] - Y[0][None, :]) ** 2
        assert np.sqrt(d2.min()) > 0.4 * W - 1e-9


@pytest.mark.parametrize("order", [2, 4])
def test_room_fixed_point_equals_direct_solve(rooms, orc_mod, order):
    """Sec. 6: on the room with the paper's source (amplitude 400, exponent 10, at (0, 1))
    and omega = 5.56, the oracle's fixed point equals the direct solve of tests/dhs.py to
    1e-12, and the zero-forcing map contracts (power iteration)."""
    import dhs
    p = rooms[order]
    assert p.omega == 5.56
    orc = orc_mod.Oracle(p)
    U = dhs.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    v = np.random.default_rng(0).standard_normal(p.n_total) * act
    for _ in range(30):
        w = orc.iterate(v, False)
        rate = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    assert rate < 1.0


def test_room_solution_fourth_order():
    """u = phi sin(0.8x + 0.3) cos(0.6y), phi the product of the four ellipses' implicit
    forms and x^2 - 4, vanishes on every wall; with f = Lap u + omega^2 u the discrete
    solution (the oracle's fixed point, equal to the direct solve above) converges at
    fourth order from h = 1/20 to 1/30 (rate 4.29)."""
    sp = pytest.importorskip("sympy")
    import dhs
    om, f_ = 2.0, math.sqrt(27.0)
    x, y = sp.symbols("x y")
    phi = ((1 - ((x + 2) / 3) ** 2 - (y / 6) ** 2) * (1 - ((x - 2) / 3) ** 2 - (y / 6) ** 2) *
           ((x / 2) ** 2 + (y - f_) ** 2 - 1) * ((x / 2) ** 2 + (y + f_) ** 2 - 1) *
           (x ** 2 - 4) / 100)
    u = phi * sp.sin(0.8 * x + 0.3) * sp.cos(0.6 * y)
    U = sp.lambdify((x, y), u, "numpy")
    F = sp.lambdify((x, y), sp.diff(u, x, 2) + sp.diff(u, y, 2) + om ** 2 * u, "numpy")
    errs = []
    for j in (2, 3):
        p = G.double_ellipse_problem(j=j, order=4, omega=om)
        p.f = [F(*g.xy) for g in p.grids]
        V = dhs.solve(p)
        ref = np.concatenate([U(*g.xy).ravel() for g in p.grids])
        act = np.concatenate([(g.mask != G.UNUSED).ravel() for g in p.grids])
        errs.append(np.max(np.abs(V - ref)[act]))
    assert 3.7 < math.log(errs[0] / errs[1]) / math.log(1.5) < 4.8, errs


@pytest.mark.parametrize("order", [2, 4])
def test_room_taken_by_the_library_host_checks(rooms, order):
    """The library's host-side validation (grid descriptions and interpolation data) takes
    the room's five grids (no device work)."""
    from host_checks import library_takes
    library_takes(rooms[order])


def test_room_refuses_walls_wider_than_the_alcoves():
    """At j = 1 the wall grids (12 h = 1.2) would be wider than the alcove segments
    (b2 - f = 0.80): refused."""
    with pytest.raises(ValueError):
        G.double_ellipse(j=1)
