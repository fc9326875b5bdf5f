"""Pins for the three-dimensional CPU oracle (second order): each test checks it against
something the paper or the mathematics fixes, never against itself (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


def _ext_coords(g):
    """Physical coordinates of every extended point of g, shape (3, e2, e1, e0)."""
    gh = g.ghosts()
    t = [np.arange(-gh[a], g.n[a] + gh[a]) * g.h[a] for a in range(3)]
    T2, T1, T0 = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    return g.mapping["map"](T0, T1, T2)


def _interior(g, out):
    """Values of an extended array at the grid's own points, shape (n2, n1, n0)."""
    gh = g.ghosts()
    return out[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]


def _single(g, omega=5.0):
    f = [np.zeros(g.mask.shape)]
    return G3.Problem3([g], G3.Interp3.empty(), omega, f)


# ------------------------------------------------------------------ operators

def test_cartesian_laplacian_exact_on_quadratics(o3):
    """D+D- is exact on quadratics: c^2 L_h u = c^2 * 2 tr(C) for u = x^T C x + d.x + e
    (Sec. 3.2), at every discretization and Dirichlet point, for a constant c^2."""
    rng = np.random.default_rng(3)
    g = G3.cartesian_grid3("box", (9, 7, 8), (-0.3, 0.1, -1.0), (0.9, 1.4, 0.2),
                           [G.BC_DIRICHLET] * 6)
    prob = _single(g)
    prob.c2 = [np.full(g.mask.shape, 1.7)]
    orc = o3.Oracle3(prob)
    Cm = rng.standard_normal((3, 3))
    Cm = Cm + Cm.T
    d = rng.standard_normal(3)
    X = _ext_coords(g)
    u = np.einsum("i...,ij,j...->...", X, Cm, X) + np.tensordot(d, X, 1) + 0.3
    out = _interior(g, orc.apply_lap(0, u))
    assert np.allclose(out, 1.7 * 2 * np.trace(Cm), rtol=1e-9, atol=1e-9)


def _smooth(X):
    return np.sin(2.0 * X[0] + 0.3) * np.cos(X[1]) * np.exp(0.5 * X[2])


def _smooth_lap(X):
    return (-4.0 - 1.0 + 0.25) * _smooth(X)


def _lap_error(o3, g):
    orc = o3.Oracle3(_single(g))
    X = _ext_coords(g)
    out = _interior(g, orc.apply_lap(0, _smooth(X)))
    ref = _interior(g, _smooth_lap(X))
    disc = g.mask == G.DISC
    return np.max(np.abs(out - ref)[disc])


@pytest.mark.parametrize("kind", ["shell", "patch"])
def test_mapped_laplacian_second_order(o3, kind):
    """The mapped Laplacian (Sec. 3.1) with metric-derived b_k converges at second order
    on the spherical shell (orthogonal) and on an orthographic pole patch (the mixed a-b
    term present), including the Neumann boundary layer with exact ghost values."""
    errs = []
    for s in (1, 2):
        if kind == "shell":
            # a 40-140 degree band: near 15 degrees the cot(th) and 1/sin(th)^2 metric
            # terms keep these coarse grids pre-asymptotic (rate ~1.6 at 64 x 31 x 15)
            g = G3.shell_grid("shell", 32 * s, 16 * s + 1 - s, 8 * s + 1 - s, 0.5, 0.3,
                              40.0, 140.0)
        else:
            g = G3.pole_patch_grid("north", 16 * s + 1 - s, 8 * s + 1 - s,
                                   math.sin(math.radians(30.0)), 0.5, 0.3, 1.0)
        errs.append(_lap_error(o3, g))
    rate = math.log2(errs[0] / errs[1])
    assert 1.8 < rate < 2.3, (errs, rate)


def test_mapped_laplacian_with_sound_speed(o3):
    """With c(x) on a curvilinear grid the operator is c(x)^2 times the mapped Laplacian
    (Eq. HelmholtzBVP, c^2 folded into every a_kl and b_k): second order against
    c^2 Lap u on the spherical shell."""
    errs = []
    for s in (1, 2):
        g = G3.shell_grid("shell", 32 * s, 16 * s + 1 - s, 8 * s + 1 - s, 0.5, 0.3, 40.0, 140.0)
        X = g.coords()
        c2 = (1.0 + 0.3 * np.sin(3.0 * X[0]) * np.cos(2.0 * X[2])) ** 2
        prob = _single(g)
        prob.c2 = [c2]
        orc = o3.Oracle3(prob)
        Xe = _ext_coords(g)
        out = _interior(g, orc.apply_lap(0, _smooth(Xe)))
        ref = c2 * _interior(g, _smooth_lap(Xe))
        errs.append(np.max(np.abs(out - ref)[g.mask == G.DISC]))
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.3, errs


def test_shell_coefficients_analytic(o3):
    """Spherical coordinates: Lap u = u_rr + (2/r) u_r + u_thth / r^2 + cot(th) u_th / r^2
    + u_phph / (r sin th)^2, so in the shell's parameters a00 = 1/(2 pi r sin th)^2,
    a11 = 1/(r dth)^2, a22 = 1/w^2, a_kl = 0 (k != l), b0 = 0, b1 = cot th/(r^2 dth) and
    b2 = 2/(r w).  The a_kl are products of the exact metrics; b_k come from second-order
    differences of the metrics (error O(h^2), asymptotic on a 40-140 degree band at these
    sizes)."""
    errs = []
    for s in (1, 2):
        nth, nr = 16 * s + 1 - s, 8 * s + 1 - s
        g = G3.shell_grid("shell", 32 * s, nth, nr, 0.5, 0.3, 40.0, 140.0)
        orc = o3.Oracle3(_single(g))
        th0, th1 = g.mapping["th"]
        dth = th1 - th0
        k, j, i = np.nonzero(g.mask == G.DISC)
        th = th0 + dth * j / (nth - 1)
        r = 0.5 + 0.3 * k / (nr - 1)
        co = {n: _interior(g, orc.coef(0, n))[k, j, i] for n in o3.COEF_NAMES}
        assert np.allclose(co["a00"], 1 / (2 * np.pi * r * np.sin(th)) ** 2, rtol=1e-12)
        assert np.allclose(co["a11"], 1 / (r * dth) ** 2, rtol=1e-12)
        assert np.allclose(co["a22"], 1 / 0.3 ** 2, rtol=1e-12)
        for n in ("a01", "a02", "a12"):
            assert np.all(co[n] == 0.0)
        e0 = np.max(np.abs(co["b0"])) / np.max(np.abs(co["b2"]))
        e1 = np.max(np.abs(co["b1"] - 1 / np.tan(th) / (r * r * dth)))
        e2 = np.max(np.abs(co["b2"] - 2 / (r * 0.3)))
        assert e0 < 1e-12
        errs.append((e1, e2))
    for q in range(2):
        assert math.log2(errs[0][q] / errs[1][q]) > 1.8, errs


# ---------------------------------------------------------- time setup

def test_time_setup_cartesian_cube(o3):
    """Eq. dtForCartesian in 3D at second order: c dt sqrt(3/h^2) <= 1, so dt_max =
    cfl h / sqrt(3); Recipe OmegaTildeExplicit and Eq. alphad give the rest."""
    prob = G3.unit_cube_problem(11, omega=7.0)
    ts = o3.Oracle3(prob).time
    h = 0.1
    assert ts.dt_max == pytest.approx(0.9 * h / math.sqrt(3.0), rel=1e-14)
    assert ts.dt <= ts.dt_max
    assert ts.dt == pytest.approx(2 / 7.0 * math.sin(math.pi / ts.Nt), rel=1e-15)
    assert 2 / 7.0 * math.sin(math.pi / (ts.Nt - 1)) > ts.dt_max
    assert ts.omega_e * ts.Nt * ts.dt == pytest.approx(2 * math.pi, rel=1e-14)
    assert ts.alpha == pytest.approx(math.tan(ts.omega_e * ts.dt / 2) /
                                     math.tan(ts.omega_e * ts.dt), rel=1e-14)


# ------------------------------------------------- the iteration map, spectral form

@pytest.mark.parametrize("bc", [G.BC_DIRICHLET, G.BC_NEUMANN])
def test_cube_eigenmodes_are_scaled_by_beta_d(o3, bc):
    """A discrete eigenmode of the 7-point Laplacian (sine modes with Dirichlet data,
    cosine modes with the centred Neumann rule) is an eigenvector of the zero-forcing
    iteration map with eigenvalue beta_d(lam~) (Eqs. waveHoltzFourierFPIexplicit, betad,
    discreteExplicitLambdaTilde): the whole march, first step, ghost rule and filter."""
    from oracle.oracle import beta_d_sum, lambda_tilde
    n = 13
    prob = G3.unit_cube_problem(n, omega=9.0, bc=bc)
    orc = o3.Oracle3(prob)
    ts = orc.time
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    rng = np.random.default_rng(5)
    v = np.zeros((n, n, n))
    expect = np.zeros_like(v)
    fn = np.sin if bc == G.BC_DIRICHLET else np.cos
    for mx, my, mz in ((1, 1, 1), (2, 3, 1), (5, 2, 4), (11, 10, 9)):
        phi = (fn(mz * np.pi * x)[:, None, None] * fn(my * np.pi * x)[None, :, None] *
               fn(mx * np.pi * x)[None, None, :])
        lam = sum(4 / h ** 2 * math.sin(m * math.pi * h / 2) ** 2 for m in (mx, my, mz))
        b = beta_d_sum(lambda_tilde(np.array([math.sqrt(lam)]), ts.dt), ts.omega_e, ts.dt,
                       ts.Nt, ts.alpha)[0]
        c = rng.standard_normal()
        v += c * phi
        expect += c * b * phi
    out = orc.iterate(v.ravel(), forcing=False).reshape(n, n, n)
    assert np.max(np.abs(out - expect)) < 1e-13 * np.max(np.abs(v))


# ------------------------------------------------------------ interpolation

def test_box_in_box_interpolation_exact_on_quadratics(o3):
    """Tensor-product Lagrange interpolation of width 3 (Sec. 3.1) reproduces every
    polynomial of degree <= 2 per axis between Cartesian grids."""
    prob = G3.box_in_box_problem()
    orc = o3.Oracle3(prob)
    rng = np.random.default_rng(2)
    c = rng.standard_normal((3, 3, 3))

    def poly(X):
        return sum(c[a, b, d] * X[0] ** a * X[1] ** b * X[2] ** d
                   for a in range(3) for b in range(3) for d in range(3))

    us = [poly(_ext_coords(g)) for g in prob.grids]
    got = orc.interpolate([u * (1.0 + 0.0) for u in us])
    for gi, g in enumerate(prob.grids):
        recv = g.mask == G.INTERP
        ext_recv = np.zeros(orc.ext_shape(gi), bool)
        _interior(g, ext_recv)[...] = recv
        assert np.allclose(got[gi][ext_recv], us[gi][ext_recv], rtol=1e-11, atol=1e-11)


def test_sphere_interpolation_third_order(o3):
    """On the sphere-in-box grids (curvilinear donors) width-3 Lagrange interpolation of a
    smooth function converges at third order (Sec. 3.1) under refinement."""
    errs = []
    for s in (1, 2):
        prob = G3.sphere_problem(nb=48 * s, nphi=64 * s, nth=32 * s, nr=10 * s,
                                 npatch=20 * s, width=0.5, r_hole=0.75, patch_deg=30.0,
                                 omega=6.0)
        orc = o3.Oracle3(prob)
        us = [_smooth(_ext_coords(g)) for g in prob.grids]
        got = orc.interpolate(us)
        e = 0.0
        for gi, g in enumerate(prob.grids):
            ext_recv = np.zeros(orc.ext_shape(gi), bool)
            _interior(g, ext_recv)[...] = g.mask == G.INTERP
            e = max(e, float(np.max(np.abs(got[gi] - us[gi])[ext_recv])))
        errs.append(e)
    assert math.log2(errs[0] / errs[1]) > 2.5, errs


def test_sphere_in_box_generator_invariants():
    """Every interpolation point is listed once, donors are discretization or Dirichlet
    points (explicit interpolation), and each axis' weights sum to 1."""
    prob = G3.sphere_problem(nb=48, nphi=64, nth=32, nr=10, npatch=20, width=0.5,
                             r_hole=0.75, patch_deg=30.0, omega=6.0)
    it = prob.interp
    G3.check_explicit_interp3(prob.grids, it)
    for w in (it.wx, it.wy, it.wz):
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
    keys = set(zip(it.recv_grid.tolist(), it.recv_i.tolist(), it.recv_j.tolist(),
                   it.recv_k.tolist()))
    assert len(keys) == it.n
    assert it.n == sum(int(np.count_nonzero(g.mask == G.INTERP)) for g in prob.grids)


# ------------------------------------------------------- fixed point = DHS

@pytest.mark.parametrize("make", [
    lambda: G3.box_in_box_problem(),
    lambda: G3.unit_cube_problem(9, omega=5.0, bc=G.BC_NEUMANN, b=20.0),
], ids=["box-in-box", "neumann-cube"])
def test_fixed_point_equals_direct_solve_3d(o3, make):
    """Sec. 6: the converged WaveHoltz solution equals the direct solution of the discrete
    Helmholtz system, assembled independently from the textbook 7-point stencil."""
    import dhs3
    from oracle.oracle import gmres
    prob = make()
    orc = o3.Oracle3(prob)
    U = dhs3.solve(prob)
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)) < 1e-11 * np.max(np.abs(U))
    v, its, hist = gmres(orc, tol=1e-13, restart=200, max_it=600)
    act = orc.active()
    assert np.max(np.abs(v - U)[act]) < 1e-9 * np.max(np.abs(U))


def test_rejects_neumann_on_non_orthogonal_axis(o3):
    """The centred Neumann rule is the normal derivative only when the normal grid axis
    is orthogonal to the tangential ones; the oracle refuses other grids."""
    g = G3.pole_patch_grid("north", 9, 5, 0.5, 0.5, 0.3, 1.0)
    g.ortho = 4  # declare (0, 2) non-orthogonal: the Neumann axis 2 then is not normal
    with pytest.raises(ValueError):
        o3.Oracle3(_single(g))


# ------------------------------------------------------- solution accuracy

@pytest.mark.parametrize("bc", [G.BC_DIRICHLET, G.BC_NEUMANN])
def test_eigenfunction_solution_second_order_3d(o3, bc):
    """Helmholtz solution phi = sin(pi x) sin(pi y) sin(pi z) on the Dirichlet cube and
    phi = cos(pi x) cos(pi y) cos(pi z) on the Neumann cube, with f = (omega^2 - 3 pi^2) phi:
    the WaveHoltz fixed point reached by the oracle's GMRES (Sec. 4.3) converges to phi at
    second order."""
    from oracle.oracle import gmres
    om = 3.0
    fn = np.sin if bc == G.BC_DIRICHLET else np.cos
    errs = []
    for n in (9, 17):
        prob = G3.unit_cube_problem(n, omega=om, bc=bc)
        X = prob.grids[0].coords()
        phi = fn(np.pi * X[0]) * fn(np.pi * X[1]) * fn(np.pi * X[2])
        prob.f = [(om ** 2 - 3 * np.pi ** 2) * phi]
        v, its, hist = gmres(o3.Oracle3(prob), tol=1e-12, restart=100, max_it=400)
        errs.append(np.max(np.abs(v.reshape(n, n, n) - phi)))
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.3, errs


def test_overset_solution_second_order_3d(o3):
    """On the box-in-box overset grid the solution of the Dirichlet problem with
    phi = prod sin(pi (x_m + 1) / 2) and f = (omega^2 - 3 pi^2 / 4) phi converges at second
    order (second-order march, third-order interpolation) under refinement of both grids."""
    from oracle.oracle import gmres
    om = 3.0
    errs = []
    for nb, ni in ((12, 10), (23, 19)):
        prob = G3.box_in_box_problem(nb=nb, ni=ni, omega=om)

        def phi(X):
            return (np.sin(np.pi * (X[0] + 1) / 2) * np.sin(np.pi * (X[1] + 1) / 2) *
                    np.sin(np.pi * (X[2] + 1) / 2))

        prob.f = [(om ** 2 - 3 * np.pi ** 2 / 4) * phi(g.coords()) for g in prob.grids]
        orc = o3.Oracle3(prob)
        v, its, hist = gmres(orc, tol=1e-12, restart=200, max_it=600)
        ref = np.concatenate([phi(g.coords()).ravel() for g in prob.grids])
        errs.append(np.max(np.abs(v - ref)[orc.active()]))
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.4, errs
