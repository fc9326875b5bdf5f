"""Pins for the paper's three-dimensional pipe (Sec. 6): a Cartesian background over the
pipe's cross-section, periodic along the axis, cut outside r_cut, and a cylindrical shell
along the Dirichlet wall, at orders 2 and 4 (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

# small versions: a shorter period along the axis keeps the direct solve in seconds
SMALL = {2: dict(j=2, lz=0.25), 4: dict(j=2, lz=0.3)}


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


def _ext_coords(g, order):
    gh = g.ghosts(order)
    X = g.coords()
    return [np.pad(x, [(gh[2], gh[2]), (gh[1], gh[1]), (gh[0], gh[0])], mode="edge") for x in X]


def _receivers(orc, gi, g, order):
    gh = g.ghosts(order)
    rec = np.zeros(orc.ext_shape(gi), bool)
    rec[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]] = g.mask == G.INTERP
    return rec


@pytest.mark.parametrize("order", [2, 4])
def test_pipe_generator_invariants(order):
    """The shell spans [R - W, R], W = min(8 h, 0.3) at order 2 and min(12 h, 0.3) at
    order 4, with the wall at R Dirichlet and order/2 interpolation
    layers inside; z is periodic on both grids with the same planes; background points in
    use lie inside r_cut; donor stencils of width order + 1 hold discretization or Dirichlet
    points only; weights sum to 1 per axis; every interpolation point is listed once."""
    kw = SMALL[order]
    prob = G3.pipe_problem(order=order, **kw)
    B, S = prob.grids
    it = prob.interp
    assert it.wx.shape[1] == order + 1
    G3.check_explicit_interp3(prob.grids, it)
    for w in (it.wx, it.wy, it.wz):
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
    keys = set(zip(it.recv_grid.tolist(), it.recv_i.tolist(), it.recv_j.tolist(),
                   it.recv_k.tolist()))
    assert len(keys) == it.n
    assert B.bc[4] == B.bc[5] == G.BC_PERIODIC and S.bc[4] == S.bc[5] == G.BC_PERIODIC
    assert S.bc[3] == G.BC_DIRICHLET
    assert B.n[2] == S.n[2] and np.allclose(B.coords()[2][:, 0, 0], S.coords()[2][:, 0, 0])
    x, y, _ = S.coords()
    r = np.hypot(x, y)
    h = 1.0 / (10 * kw["j"])
    W = r.max() - r.min()
    assert abs(r.max() - 0.5) < 1e-12
    assert abs(W - min((8 if order == 2 else 12) * h, 0.3)) < 1e-12
    assert np.all(S.mask[:, -1] == G.DIRICHLET)
    assert np.all(S.mask[:, :order // 2] == G.INTERP)
    assert np.all(S.mask[:, order // 2:-1] == G.DISC)
    xb, yb, _ = B.coords()
    rb = np.hypot(xb, yb)
    r_in = 0.5 - W
    assert np.all(rb[B.mask == G.DISC] <= r_in + 0.5 * W + 1e-12)
    assert np.any(B.mask == G.UNUSED) and np.all(rb[B.mask == G.UNUSED] > r_in + 0.5 * W)


@pytest.mark.parametrize("order", [2, 4])
def test_pipe_interpolation_exact_on_donor_polynomials(o3, order):
    """rho^(order/2) (1 + cos(2 pi z / lz) / 2), rho = x^2 + y^2, is a polynomial of degree
    <= order per axis in the background's coordinates and in the shell's (r, theta, z)
    (theta-free, and the z planes coincide): width-(order+1) Lagrange interpolation
    reproduces it at every receiver."""
    kw = SMALL[order]
    prob = G3.pipe_problem(order=order, **kw)
    orc = o3.Oracle3(prob)
    us = []
    for g in prob.grids:
        X = _ext_coords(g, order)
        us.append((X[0] ** 2 + X[1] ** 2) ** (order // 2) *
                  (1 + 0.5 * np.cos(2 * np.pi * X[2] / kw["lz"])))
    got = orc.interpolate([u.copy() for u in us])
    for gi, g in enumerate(prob.grids):
        rec = _receivers(orc, gi, g, order)
        assert rec.any()
        assert np.max(np.abs(got[gi] - us[gi])[rec]) < 1e-12


def test_pipe_interpolation_third_order(o3):
    """Width-3 interpolation of a smooth non-polynomial function between the pipe's grids
    converges at third order under refinement."""
    errs = []
    for j in (2, 4):
        prob = G3.pipe_problem(j=j, order=2, lz=0.25)
        orc = o3.Oracle3(prob)
        us = []
        for g in prob.grids:
            X = _ext_coords(g, 2)
            us.append(np.sin(3 * X[0] + X[1]) * np.exp(X[0] * X[1]) + np.cos(8 * np.pi * X[2]))
        got = orc.interpolate([u.copy() for u in us])
        e = 0.0
        for gi, g in enumerate(prob.grids):
            rec = _receivers(orc, gi, g, 2)
            e = max(e, float(np.max(np.abs(got[gi] - us[gi])[rec])))
        errs.append(e)
    assert 2.6 < math.log2(errs[0] / errs[1]) < 3.6, errs


@pytest.mark.parametrize("order,kw,periods", [(2, SMALL[2], 1), (4, SMALL[4], 1),
                                              (4, dict(j=2), 4), (4, dict(j=3, lz=0.3), 1)],
                         ids=["o2", "o4", "o4-G2-Np4", "o4-centred"])
def test_pipe_fixed_point_equals_direct_solve(o3, order, kw, periods):
    """Sec. 6: on the pipe with the paper's source (amplitude 150, exponent 10, centred at
    (0.1, 0.1, 0.5)) and omega = 8.5, the oracle's fixed point equals the direct solve of
    tests/dhs3.py to 1e-12 -- among them the paper's order-4 run on its grid G^(2) over the
    full period lz = 1 with four periods in the time filter, whose donor stencils are partly
    off-centred, and a finer grid whose stencils are all centred."""
    import dhs3
    prob = G3.pipe_problem(order=order, **kw)
    assert prob.omega == 8.5
    orc = o3.Oracle3(prob, periods=periods)
    U = dhs3.solve(prob)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))


def test_pipe_off_centred_stencils(o3):
    """On G^(2) at order 4 some donor stencils are off-centred (the receiver lies more than
    half a cell from the stencil's middle point), the nearest valid placement; with
    centring enforced the generator refuses.  The off-centred width-5 weights still
    reproduce quartics along each axis."""
    prob = G3.pipe_problem(order=4, **SMALL[4])
    it = prob.interp
    from paper_2504_03074_gb300.grids import lagrange_weights
    fr = []
    for w in (it.wx, it.wy, it.wz):
        # recover each receiver's fractional position from its weights: sum_k k w_k
        fr.append(w @ np.arange(5.0))
    off = np.zeros(it.n, bool)
    for f in fr:
        off |= np.abs(f - 2.0) > 0.5 + 1e-12
    assert off.any() and np.all(np.abs(np.stack(fr) - 2.0) <= 1.5 + 1e-12)
    for f, w in zip(fr, (it.wx, it.wy, it.wz)):
        assert np.allclose(lagrange_weights(f, 5), w, atol=1e-12)
        for k in range(5):
            assert np.allclose(w @ np.arange(5.0) ** k, f ** k, atol=1e-10)
    with pytest.raises(ValueError):
        G3.pipe_problem(order=4, shift=0, **SMALL[4])


def test_pipe_solution_second_order(o3):
    """u = (R^2 - r^2) cos(3x + y) cos(2 pi z / lz) vanishes on the wall; with
    f = Lap u + omega^2 u the WaveHoltz solution on the pipe converges at second order."""
    from oracle.oracle import gmres
    R, om, lz = 0.5, 3.0, 0.25
    k = 2 * np.pi / lz
    errs = []
    for j in (2, 4):
        prob = G3.pipe_problem(j=j, order=2, lz=lz, omega=om)
        us, fs = [], []
        for g in prob.grids:
            x, y, z = g.coords()
            P = R * R - x * x - y * y
            Q, S, Z = np.cos(3 * x + y), np.sin(3 * x + y), np.cos(k * z)
            u = P * Q * Z
            lap = Z * (-4 * Q + 2 * (6 * x + 2 * y) * S - 10 * P * Q) - k * k * u
            us.append(u)
            fs.append(lap + om * om * u)
        prob.f = fs
        orc = o3.Oracle3(prob)
        v, its, hist = gmres(orc, tol=1e-12, restart=200, max_it=600)
        ref = np.concatenate([u.ravel() for u in us])
        errs.append(np.max(np.abs(v - ref)[orc.active()]))
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.4, errs


def test_pipe_library_host_checks():
    """The library's host checks take the pipe at order 2 (the kernels of the sphere-in-box:
    a curvilinear shell periodic in theta and z, a Cartesian background periodic in z);
    at order 4 they refuse the curvilinear shell with a message (the library's fourth-order
    3D path is Cartesian only)."""
    from host_checks import library_status3
    st, msg = library_status3(G3.pipe_problem(order=2, **SMALL[2]))
    assert st == 0, msg
    st, msg = library_status3(G3.pipe_problem(order=4, **SMALL[4]))
    assert st != 0 and msg
