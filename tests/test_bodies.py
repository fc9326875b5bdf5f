"""The multi-body overset generator (several disks and ellipses in a square, Sec. 3.1's
overset grids with more than one curvilinear component): the body mappings invert
exactly, their analytic inverse metrics equal finite differences of the inverse map, and
the generated overset grid satisfies the explicit-interpolation invariants; invalid
layouts are refused.  (Its fixed point equals the direct discrete solve:
test_oracle_pins.py.)"""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

BODIES = [G.Body((-0.9, 0.55), 0.5, 0.25, 0.3, 320, 24),
          G.Body((0.85, -0.6), 0.6, 0.35, 0.3, 384, 24),
          G.Body((0.6, 1.05), 0.3, 0.3, 0.3, 256, 24)]


@pytest.mark.parametrize("k", range(len(BODIES)))
def test_mapping_inverts_and_metrics_are_exact(k):
    b = BODIES[k]
    m = G._BodyMap(b)
    rng = np.random.default_rng(k)
    t, s = rng.uniform(0, 1, 200), rng.uniform(-0.05, 1.05, 200)
    x, y = m.xy(t, s)
    fi, fj, s2 = m.param(x, y)
    assert np.max(np.abs(np.mod(fi / b.nth - t + 0.5, 1.0) - 0.5)) < 1e-12
    assert np.max(np.abs(s2 - s)) < 1e-12
    assert np.allclose(fj, s * (b.nr - 1), atol=1e-10)
    # analytic dt/dx, dt/dy, ds/dx, ds/dy against central differences of the inverse map
    e = 1e-6
    r = m.rx(t, s)
    tp, _, sp = m.param(x + e, y)
    tm, _, sm = m.param(x - e, y)
    dtdx = (np.mod(tp - tm + b.nth / 2, b.nth) - b.nth / 2) / b.nth / (2 * e)
    dsdx = (sp - sm) / (2 * e)
    tp, _, sp = m.param(x, y + e)
    tm, _, sm = m.param(x, y - e)
    dtdy = (np.mod(tp - tm + b.nth / 2, b.nth) - b.nth / 2) / b.nth / (2 * e)
    dsdy = (sp - sm) / (2 * e)
    for a, fd in zip(r, (dtdx, dtdy, dsdx, dsdy)):
        assert np.max(np.abs(a - fd)) <= 1e-7 * np.max(np.abs(fd))
    # orthogonal grid lines: grad t . grad s = 0
    assert np.max(np.abs(r[0] * r[2] + r[1] * r[3])) < 1e-12 * np.max(np.abs(r[2]) * np.abs(r[0]))


def test_ellipse_boundary_is_the_ellipse():
    b = BODIES[1]
    m = G._BodyMap(b)
    t = np.linspace(0, 1, 97)
    x, y = m.xy(t, np.zeros_like(t))
    cx, cy = b.center
    assert np.allclose(((x - cx) / b.a) ** 2 + ((y - cy) / b.b) ** 2, 1.0, atol=1e-13)
    x, y = m.xy(t, np.ones_like(t))  # outer edge: semi-major axis a + width
    assert np.isclose(np.max(x - cx), b.a + b.width)


def test_overset_invariants():
    p = G.ellipses_problem(nb=256)
    grids, it = p.grids, p.interp
    G.check_explicit_interp(grids, it, 4)
    assert len(grids) == 4 and it.n > 0
    # every receiver is an interpolation point of its grid, weights sum to one
    for k in range(it.n):
        assert grids[it.recv_grid[k]].mask[it.recv_j[k], it.recv_i[k]] == G.INTERP
    assert np.allclose(it.wx.sum(1), 1) and np.allclose(it.wy.sum(1), 1)
    # background receivers take donors on a body grid, body receivers on the background
    assert np.all(it.donor_grid[it.recv_grid == 0] > 0)
    assert np.all(it.donor_grid[it.recv_grid > 0] == 0)
    # each body grid's interpolation points are its outer order/2 lines
    for g in grids[1:]:
        assert np.all(g.mask[-2:] == G.INTERP) and np.all(g.mask[:-2] == G.DISC)


def test_invalid_layouts_are_refused():
    a = G.Body((0.0, 0.0), 0.5, 0.3, 0.4, 128, 16)
    b = G.Body((0.3, 0.0), 0.4, 0.4, 0.4, 128, 16)  # cuts overlap
    with pytest.raises(ValueError):
        G.bodies_in_square(128, [a, b], 4)
    with pytest.raises(ValueError):
        G._BodyMap(G.Body((0.0, 0.0), 0.3, 0.5, 0.3, 64, 12))  # b > a
    with pytest.raises(ValueError):  # cut too thin for the background's interpolation layer
        G.bodies_in_square(48, [G.Body((0.0, 0.0), 0.4, 0.22, 0.6, 64, 12, cut=0.3)], 4)
