"""Pins for the dissipative march of the 3D oracle (the paper's upwind-dissipation variant,
read as in two dimensions): the dissipation acts on the march's deviation from the
iterate's periodic motion, so the discrete Helmholtz solution stays the fixed point; on the
grid-scale mode of a periodic cube the map equals the scheme's scalar recurrence, whose
characteristic equation gives the stability limit (CPU only)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


def _rate(orc, n, act, its=25):
    """Largest |eigenvalue| of the zero-forcing map by power iteration."""
    v = np.random.default_rng(0).standard_normal(n) * act
    for _ in range(its):
        w = orc.iterate(v, False)
        rate = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return rate


CASES = [
    ("cube-o2", lambda: G3.unit_cube_problem(11, omega=5.0, b=20.0), 0.02),
    ("cube-o4", lambda: G3.unit_cube_problem(11, omega=5.0, b=20.0, order=4), 0.01),
    ("box-in-box-o2", lambda: G3.box_in_box_problem(), 0.02),
    ("pipe-o4", lambda: G3.pipe_problem(j=2, order=4, lz=0.3), 0.01),
]


@pytest.mark.parametrize("k", range(len(CASES)), ids=[c[0] for c in CASES])
def test_dissipative_fixed_point_equals_direct_solve_3d(o3, k):
    """With the dissipation on, the direct discrete solution (tests/dhs3.py, which knows
    nothing of it) is still a fixed point of the map; the map itself changes away from the
    fixed point, and stays a contraction at these coefficients."""
    import dhs3
    name, make, nu = CASES[k]
    p = make()
    orc = o3.Oracle3(p, nu=nu)
    U = dhs3.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U)), name
    v = np.random.default_rng(5).standard_normal(p.n_total) * act
    assert np.max(np.abs(orc.iterate(v, True) - o3.Oracle3(p).iterate(v, True))) > 1e-8
    assert _rate(orc, p.n_total, act) < 1.0


def _checkerboard_amplitude(T, mu, nu_s):
    """The zero-forcing map on the grid-scale mode of a periodic cube, from the scheme's
    definition reduced to that mode: W^0 = 1, W^1 = 1 - mu/2, then
    W^{n+1} = (2 - mu) W^n - W^{n-1} - nu s ((W^n - W^{n-1}) - (cos w t^n - cos w t^{n-1})),
    filtered with the trapezoid weights (2 / T-bar) sigma_n dt (cos w t^n - alpha/2)."""
    import math
    dt, w, M, al = T.dt, T.omega_e, T.M, T.alpha

    def wf(n):
        return 2.0 / (M * dt) * (0.5 if n in (0, M) else 1.0) * dt * (math.cos(w * n * dt) - al / 2)
    Wm, Wc = 1.0, 1.0 - mu / 2.0
    V = wf(0) * Wm + wf(1) * Wc
    for n in range(1, M):
        dc = math.cos(w * n * dt) - math.cos(w * (n - 1) * dt)
        Wm, Wc = Wc, (2.0 - mu) * Wc - Wm - nu_s * ((Wc - Wm) - dc)
        V += wf(n + 1) * Wc
    return V, Wc


@pytest.mark.parametrize("order", [2, 4])
def test_dissipation_on_the_grid_scale_mode_of_the_periodic_cube(o3, order):
    """The grid-scale mode of a periodic cube is an eigenvector of the Laplacian (7-point:
    dt^2 L -> -mu, mu = 12 dt^2 / h^2; 13-point: mu = 16 dt^2 / h^2) and of the dissipation
    (symbol s = 12 for three axes of (-1, 2, -1), 48 for (1, -4, 6, -4, 1)): the dissipative
    map scales it by the closed-form amplitude of the scalar recurrence, to 1e-12.  That
    recurrence's roots leave the unit circle once nu > (4 - mu) / (2 s); below the limit the
    map contracts, well above it the map grows (just above it the filter still averages
    the alternating growth away)."""
    n = 12
    p = G3.unit_cube_problem(n, omega=5.0, b=20.0, bc=G.BC_PERIODIC, order=order)
    T = o3.Oracle3(p).time
    h = p.grids[0].h[0]
    mu = (12.0 if order == 2 else 16.0) * T.dt * T.dt / (h * h)
    sym = 12.0 if order == 2 else 48.0
    nu_star = (4.0 - mu) / (2.0 * sym)
    assert 0.0 < nu_star < 0.1
    i = np.arange(n)
    cb = ((-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])).ravel()
    for f in (0.3, 0.9, 1.1, 1.3):
        amp, last = _checkerboard_amplitude(T, mu, sym * f * nu_star)
        out = o3.Oracle3(p, nu=f * nu_star).iterate(cb, False)
        assert np.max(np.abs(out - amp * cb)) < 1e-12 * max(1.0, abs(last)), f
    act = np.ones(p.n_total, bool)
    assert _rate(o3.Oracle3(p, nu=0.9 * nu_star), p.n_total, act) < 1.0
    assert _rate(o3.Oracle3(p, nu=1.5 * nu_star), p.n_total, act) > 10.0


def test_negative_dissipation_refused_3d(o3):
    with pytest.raises(ValueError):
        o3.Oracle3(G3.unit_cube_problem(9, omega=5.0), nu=-0.1)
