"""Pins for physical sides on non-orthogonal grids in the 2D oracle (order 2): a sheared
channel whose grid lines cross the walls at an angle.  The Neumann rule is the normal
derivative with its tangential term, a_nn D0_n W + a_nt D0_t W = 0; a Dirichlet side reads
no ghost at this order (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G


@pytest.fixture(scope="module")
def orc_mod():
    from oracle import oracle
    return oracle


def test_neumann_rule_is_the_normal_derivative(orc_mod):
    """After the ghost rules, the centred normal derivative grad(eta) . grad(W) =
    a_11 D0_eta W + a_01 D0_xi W vanishes at every wall point (random data), and differs
    from the orthogonal rule W_{-1} = W_{+1} by the tangential term."""
    shear, L = 0.5, 0.6
    p = G.sheared_channel_problem(n0=24, n1=13, shear=shear, L=L)
    g = p.grids[0]
    orc = orc_mod.Oracle(p)
    rng = np.random.default_rng(1)
    w = orc.apply_bc(0, rng.standard_normal(orc.ext_shape(0)), 0.0)
    a11, a01 = 1.0 / L ** 2, -shear / L ** 2
    h0, h1 = g.h
    for jb, jg, jin, sg in ((1, 0, 2, 1.0), (g.n[1], g.n[1] + 1, g.n[1] - 1, -1.0)):
        row = w[jb]
        dn = sg * (w[jin] - w[jg]) / (2 * h1)  # along +eta
        dt = (np.roll(row, -1) - np.roll(row, 1)) / (2 * h0)
        assert np.max(np.abs(a11 * dn + a01 * dt)) < 1e-10 * np.max(np.abs(a11 * dn))
        assert np.max(np.abs(w[jg] - w[jin])) > 1e-3


def test_sheared_channel_map_is_a_contraction(orc_mod):
    """The zero-forcing map's largest |eigenvalue| (power iteration) stays below 1 on the
    sheared channel with Neumann walls crossed at up to 40 degrees, as on the unsheared
    channel: the fixed-point iteration converges there."""
    for shear in (0.0, 0.4, 0.5):
        p = G.sheared_channel_problem(shear=shear)
        orc = orc_mod.Oracle(p)
        v = np.random.default_rng(0).standard_normal(p.n_total)
        for _ in range(40):
            w = orc.iterate(v, False)
            rate = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        assert rate < 0.99, (shear, rate)


@pytest.mark.parametrize("bc", [G.BC_NEUMANN, G.BC_DIRICHLET])
@pytest.mark.parametrize("shear", [0.4, 0.5])
def test_sheared_channel_fixed_point_equals_direct_solve(orc_mod, bc, shear):
    """Sec. 6: the oracle's fixed point on the sheared channel (mixed terms at the walls)
    equals the direct discrete solve of tests/dhs.py, whose Neumann rows are written from
    the normal-derivative definition; GMRES reaches it."""
    import dhs
    p = G.sheared_channel_problem(shear=shear, bc=bc)
    orc = orc_mod.Oracle(p)
    U = dhs.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    v, its, hist = orc_mod.gmres(orc, tol=1e-12, restart=200, max_it=600)
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U)), its


def test_sheared_channel_neumann_solution_second_order(orc_mod):
    """u = cos(2 pi x) cos(pi y / L) has zero normal derivative on both walls; with
    f = (omega^2 - 4 pi^2 - pi^2 / L^2) u the WaveHoltz solution on the sheared grid
    converges to it at second order."""
    om, L = 3.0, 0.6
    errs = []
    for n in (32, 64):
        p = G.sheared_channel_problem(n0=n, n1=int(round(n * L)) + 1, shear=0.4, L=L, omega=om)
        x, y = p.grids[0].xy
        u = np.cos(2 * np.pi * x) * np.cos(np.pi * y / L)
        p.f = [(om ** 2 - 4 * np.pi ** 2 - np.pi ** 2 / L ** 2) * u]
        v, its, hist = orc_mod.gmres(orc_mod.Oracle(p), tol=1e-12, restart=200, max_it=600)
        errs.append(np.max(np.abs(v.reshape(u.shape) - u)))
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.3, errs


def test_nonorthogonal_physical_sides_refused_where_not_defined(orc_mod):
    """Order 4 on a non-orthogonal grid with a physical side, and a Neumann side whose
    tangential axis is not periodic, are refused."""
    with pytest.raises(ValueError):
        orc_mod.Oracle(G.sheared_channel_problem(order=4))
    p = G.sheared_channel_problem()
    g = p.grids[0]
    g.bc = [G.BC_NONE, G.BC_NONE, G.BC_NEUMANN, G.BC_NEUMANN]
    g.rx = np.pad(g.rx, ((0, 0), (0, 0), (1, 1)), mode="edge")
    g.mask[:, 0] = g.mask[:, -1] = G.INTERP
    with pytest.raises(ValueError):
        orc_mod.Oracle(p)
