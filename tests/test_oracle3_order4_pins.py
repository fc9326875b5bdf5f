"""Pins for the three-dimensional CPU oracle at fourth order (Cartesian grids): each test
checks it against something the paper or the mathematics fixes, never against itself
(CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")
P, N, D = G.BC_PERIODIC, G.BC_NEUMANN, G.BC_DIRICHLET


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


def _ext_coords(g, order=4):
    gh = g.ghosts(order)
    t = [np.arange(-gh[a], g.n[a] + gh[a]) * g.h[a] for a in range(3)]
    T2, T1, T0 = np.meshgrid(t[2], t[1], t[0], indexing="ij")
    return g.mapping["map"](T0, T1, T2)


def _interior(g, out, order=4):
    gh = g.ghosts(order)
    return out[gh[2]:gh[2] + g.n[2], gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]


def _single(g, omega=5.0, order=4):
    return G3.Problem3([g], G3.Interp3.empty(), omega, [np.zeros(g.mask.shape)], order=order)


def _periodic_slab(n, bc):
    """[0, 1)^2 periodic in x and y (n points per period) times [0, 1] in z."""
    return G3.cartesian_grid3("slab", (n, n, n), (0.0, 0.0, 0.0),
                              ((n - 1) / n, (n - 1) / n, 1.0), bc)


# ------------------------------------------------------------------ operators

def test_fourth_order_laplacian_exact_on_quintics(o3):
    """D+D-(1 - h^2/12 D+D-) (Eq. SecondDerivOrderp, mu < 2) is exact on polynomials of
    degree <= 5 per axis: c^2 L_h u = c^2 Lap u at every point of the grid."""
    rng = np.random.default_rng(4)
    g = G3.cartesian_grid3("box", (9, 8, 10), (-0.3, 0.1, -1.0), (0.9, 1.4, 0.2), [D] * 6)
    prob = _single(g)
    prob.c2 = [np.full(g.mask.shape, 1.3)]
    orc = o3.Oracle3(prob)
    c = rng.standard_normal((3, 6))
    X = _ext_coords(g)
    u = sum(c[a, p] * X[a] ** p for a in range(3) for p in range(6)) + X[0] ** 2 * X[1] ** 3
    lap = (sum(c[a, p] * p * (p - 1) * X[a] ** (p - 2) for a in range(3) for p in range(2, 6))
           + 2 * X[1] ** 3 + 6 * X[0] ** 2 * X[1])
    out = _interior(g, orc.apply_lap(0, u))
    assert np.allclose(out, 1.3 * _interior(g, lap), rtol=1e-9, atol=1e-8)


def test_fourth_order_laplacian_error_decays_at_fourth_order(o3):
    errs = []
    for n in (11, 21):
        g = G3.cartesian_grid3("box", (n, n, n), (0.0,) * 3, (1.0,) * 3, [D] * 6)
        X = _ext_coords(g)
        u = np.sin(2.0 * X[0] + 0.3) * np.cos(X[1]) * np.exp(0.5 * X[2])
        lap = (-4.0 - 1.0 + 0.25) * u
        out = _interior(g, o3.Oracle3(_single(g)).apply_lap(0, u))
        errs.append(np.max(np.abs(out - _interior(g, lap))))
    assert 3.8 < math.log2(errs[0] / errs[1]) < 4.3, errs


def test_ghost_rules_reproduce_their_defining_conditions(o3):
    """After the boundary step the ghosts satisfy, per boundary point, the two conditions
    that define them: Dirichlet c^2 D_nn W_b = 0 (zero forcing) with the fifth-order
    extrapolation, Neumann the fourth-order centred D_n W = 0 with the same extrapolation;
    checked on the z faces of a periodic slab with random values."""
    rng = np.random.default_rng(8)
    n = 8
    for bc in ([P, P, P, P, N, D], [P, P, P, P, D, N]):
        g = _periodic_slab(n, bc)
        orc = o3.Oracle3(_single(g))
        u = rng.standard_normal(orc.ext_shape(0))
        # zero boundary values on the Dirichlet face, as the march keeps them
        zd = 2 if bc[4] == D else n + 1
        u[zd] = 0.0
        w = orc.apply_bc(0, u)
        for side in (4, 5):
            # rows along the inward normal: G2, G1, U0, U1, U2, U3
            idx = [0, 1, 2, 3, 4, 5] if side == 4 else [n + 3, n + 2, n + 1, n, n - 1, n - 2]
            G2, G1, U0, U1, U2, U3 = (w[k] for k in idx)
            ext = G2 - 5 * G1 + 10 * U0 - 10 * U1 + 5 * U2 - U3
            assert np.max(np.abs(ext)) < 1e-12
            if bc[side] == D:
                assert np.max(np.abs(-G2 + 16 * G1 - 30 * U0 + 16 * U1 - U2)) < 1e-12
            else:
                assert np.max(np.abs(8 * (U1 - G1) - (U2 - G2))) < 1e-12


def test_time_setup_fourth_order(o3):
    """Eq. dtForCartesian at fourth order: C = sqrt(3)/2, so dt_max = cfl (sqrt(3)/2) h /
    sqrt(3) = cfl h / 2 on the unit cube; Recipe OmegaTildeExplicit for the rest."""
    ts = o3.Oracle3(G3.unit_cube_problem(11, omega=7.0, order=4)).time
    assert ts.dt_max == pytest.approx(0.9 * 0.1 / 2.0, rel=1e-14)
    assert ts.dt == pytest.approx(2 / 7.0 * math.sin(math.pi / ts.Nt), rel=1e-15)
    assert 2 / 7.0 * math.sin(math.pi / (ts.Nt - 1)) > ts.dt_max


# ------------------------------------------------- the iteration map, spectral form

def test_periodic_fourier_modes_are_scaled_by_beta_d(o3):
    """On the fully periodic cube a Fourier mode is an eigenvector of the fourth-order
    Laplacian with eigenvalue -sum_a (4/h^2) s_a^2 (1 + s_a^2 / 3), s_a = sin(theta_a / 2),
    and so of the zero-forcing iteration map with eigenvalue beta_d(lam~) (Eqs.
    waveHoltzFourierFPIexplicit, betad, discreteExplicitLambdaTilde)."""
    from oracle.oracle import beta_d_sum, lambda_tilde
    n = 12
    g = G3.cartesian_grid3("torus", (n, n, n), (0.0,) * 3, ((n - 1) / n,) * 3, [P] * 6)
    orc = o3.Oracle3(_single(g, omega=9.0))
    ts = orc.time
    h = 1.0 / n
    i = np.arange(n)
    rng = np.random.default_rng(6)
    v = np.zeros((n, n, n))
    expect = np.zeros_like(v)
    for mx, my, mz in ((0, 0, 1), (1, 2, 3), (5, 4, 6), (6, 6, 6)):
        th = [2 * np.pi * m / n for m in (mx, my, mz)]
        ph = rng.uniform(0, 2 * np.pi, 3)
        phi = (np.cos(th[2] * i + ph[2])[:, None, None] * np.cos(th[1] * i + ph[1])[None, :, None]
               * np.cos(th[0] * i + ph[0])[None, None, :])
        # the product of cosines mixes +-theta per axis: all share the same eigenvalue
        lam = sum(4 / h ** 2 * math.sin(t / 2) ** 2 * (1 + math.sin(t / 2) ** 2 / 3) for t in th)
        b = beta_d_sum(lambda_tilde(np.array([math.sqrt(lam)]), ts.dt), ts.omega_e, ts.dt,
                       ts.Nt, ts.alpha)[0]
        c = rng.standard_normal()
        v += c * phi
        expect += c * b * phi
    out = orc.iterate(v.ravel(), forcing=False).reshape(n, n, n)
    assert np.max(np.abs(out - expect)) < 1e-13 * np.max(np.abs(v))


# ------------------------------------------------------------ interpolation

def test_box_in_box_width5_interpolation_exact_on_quartics(o3):
    """Tensor-product Lagrange interpolation of width 5 (Sec. 3.1) reproduces every
    polynomial of degree <= 4 per axis between the two Cartesian grids."""
    prob = G3.box_in_box_problem(nb=17, ni=15, order=4, hole=0.1)
    assert prob.interp.wx.shape[1] == 5
    orc = o3.Oracle3(prob)
    rng = np.random.default_rng(2)
    c = rng.standard_normal((5, 5, 5))

    def poly(X):
        return sum(c[a, b, d] * X[0] ** a * X[1] ** b * X[2] ** d
                   for a in range(5) for b in range(5) for d in range(5))

    us = [poly(_ext_coords(g)) for g in prob.grids]
    got = orc.interpolate([u.copy() for u in us])
    for gi, g in enumerate(prob.grids):
        ext_recv = np.zeros(orc.ext_shape(gi), bool)
        _interior(g, ext_recv)[...] = g.mask == G.INTERP
        assert ext_recv.any()
        assert np.allclose(got[gi][ext_recv], us[gi][ext_recv], rtol=1e-10, atol=1e-10)


def test_box_in_box_fourth_order_generator_invariants():
    """Interpolation layers two points thick, width-5 donor stencils of discretization or
    Dirichlet points only, weights summing to 1 per axis."""
    prob = G3.box_in_box_problem(nb=17, ni=15, order=4, hole=0.1)
    G3.check_explicit_interp3(prob.grids, prob.interp)
    for w in (prob.interp.wx, prob.interp.wy, prob.interp.wz):
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
    inner = prob.grids[1]
    assert np.all(inner.mask[:, :, :2] == G.INTERP) and np.all(inner.mask[:, :, -2:] == G.INTERP)
    assert np.all(inner.mask[2:-2, 2:-2, 2:-2] == G.DISC)


# ------------------------------------------------------- fixed point = DHS

def _forced(g, omega=5.0):
    """Order-4 problem on one grid with a Gaussian source centred in [0.3, 0.7]^3."""
    return G3.Problem3([g], G3.Interp3.empty(), omega,
                       [G3.gaussian3(g, np.array([0.45, 0.55, 0.6]), 1.0, 20.0)], order=4)


@pytest.mark.parametrize("make", [
    lambda: G3.unit_cube_problem(11, omega=5.0, b=20.0, order=4),
    # distinct spacings on the three axes
    lambda: _forced(G3.cartesian_grid3("box", (11, 9, 10), (0.0,) * 3, (1.0, 0.8, 1.1), [D] * 6)),
    lambda: _forced(_periodic_slab(10, [P, P, P, P, N, D])),
    lambda: _forced(_periodic_slab(10, [P, P, P, P, D, N])),
    lambda: G3.unit_cube_problem(10, omega=5.0, b=20.0, order=4, bc=[P, P, N, N, P, P]),
    lambda: G3.box_in_box_problem(nb=17, ni=15, order=4, hole=0.1),
], ids=["dirichlet-cube", "dirichlet-box", "neumann-dirichlet-slab", "dirichlet-neumann-slab",
        "neumann-slab", "box-in-box"])
def test_fixed_point_equals_direct_solve_fourth_order_3d(o3, make):
    """Sec. 6: the converged fourth-order WaveHoltz solution equals the direct solution of
    the fourth-order discrete Helmholtz system (13-point stencil, the two ghost rows per
    boundary point, width-5 interpolation), assembled independently."""
    import dhs3
    from oracle.oracle import gmres
    prob = make()
    orc = o3.Oracle3(prob)
    U = dhs3.solve(prob)
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)) < 1e-11 * np.max(np.abs(U))
    v, its, hist = gmres(orc, tol=1e-13, restart=200, max_it=600)
    act = orc.active()
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U))


# ------------------------------------------------------- solution accuracy

def test_dirichlet_cube_solution_fourth_order(o3):
    """phi = sin(pi x) sin(pi y) sin(pi z), f = (omega^2 - 3 pi^2) phi: the WaveHoltz fixed
    point reached by GMRES (Sec. 4.3) converges to phi at fourth order."""
    from oracle.oracle import gmres
    om, errs = 3.0, []
    for n in (9, 17):
        prob = G3.unit_cube_problem(n, omega=om, order=4)
        X = prob.grids[0].coords()
        phi = np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])
        prob.f = [(om ** 2 - 3 * np.pi ** 2) * phi]
        v, its, hist = gmres(o3.Oracle3(prob), tol=1e-12, restart=100, max_it=400)
        errs.append(np.max(np.abs(v.reshape(n, n, n) - phi)))
    assert 3.6 < math.log2(errs[0] / errs[1]) < 4.4, errs


def test_neumann_slab_solution_fourth_order(o3):
    """Periodic in x and y, Neumann in z: phi = cos(2 pi x) sin(2 pi y + 0.3) cos(pi z),
    f = (omega^2 - 9 pi^2) phi, fourth-order convergence."""
    from oracle.oracle import gmres
    om, errs = 3.0, []
    for n in (9, 17):
        g = _periodic_slab(n, [P, P, P, P, N, N])
        X = g.coords()
        phi = np.cos(2 * np.pi * X[0]) * np.sin(2 * np.pi * X[1] + 0.3) * np.cos(np.pi * X[2])
        prob = G3.Problem3([g], G3.Interp3.empty(), om, [(om ** 2 - 9 * np.pi ** 2) * phi],
                           order=4)
        v, its, hist = gmres(o3.Oracle3(prob), tol=1e-12, restart=100, max_it=400)
        errs.append(np.max(np.abs(v.reshape(n, n, n) - phi)))
    assert 3.4 < math.log2(errs[0] / errs[1]) < 4.4, errs


def test_overset_solution_fourth_order_3d(o3):
    """Box-in-box at fourth order (width-5 interpolation), phi = prod sin(pi (x_m + 1) / 2),
    f = (omega^2 - 3 pi^2 / 4) phi: fourth-order convergence under refinement of both
    grids (the finer level on the all-cores build of the same C source)."""
    from oracle.oracle import gmres
    om, errs = 3.0, []
    for nb, ni in ((17, 15), (33, 29)):
        prob = G3.box_in_box_problem(nb=nb, ni=ni, omega=om, order=4, hole=0.1)

        def phi(X):
            return (np.sin(np.pi * (X[0] + 1) / 2) * np.sin(np.pi * (X[1] + 1) / 2) *
                    np.sin(np.pi * (X[2] + 1) / 2))

        prob.f = [(om ** 2 - 3 * np.pi ** 2 / 4) * phi(g.coords()) for g in prob.grids]
        orc = o3.Oracle3(prob, openmp=nb > 17)
        v, its, hist = gmres(orc, tol=1e-12, restart=200, max_it=600)
        ref = np.concatenate([phi(g.coords()).ravel() for g in prob.grids])
        errs.append(np.max(np.abs(v - ref)[orc.active()]))
    assert 3.6 < math.log2(errs[0] / errs[1]) < 4.4, errs


# ------------------------------------------------------- what it refuses

def test_fourth_order_refusals(o3):
    """A curvilinear Dirichlet face whose normal axis is not orthogonal to the others, a
    Neumann face meeting another physical face, and Dirichlet data at fourth order are
    refused, as is an order other than 2 or 4."""
    g = G3.pole_patch_grid("north", 12, 8, 0.5, 0.5, 0.3, 1.0, order=4)
    o3.Oracle3(_single(g))  # Neumann sphere face, interpolation edges: taken
    g.bc[5] = D  # the radial axis is orthogonal to a and b: taken
    o3.Oracle3(_single(g))
    g.bc[0] = g.bc[1] = D  # the a axis is not orthogonal to b
    with pytest.raises(ValueError):
        o3.Oracle3(_single(g))
    with pytest.raises(ValueError):
        o3.Oracle3(G3.unit_cube_problem(9, order=4, bc=[N] * 6))
    with pytest.raises(ValueError):
        o3.Oracle3(G3.unit_cube_problem(9, order=4, bc=[P, P, N, N, D, D]))
    p = G3.with_boundary_data3(G3.unit_cube_problem(9, order=4), lambda x, y, z: 1.0 + x)
    with pytest.raises(ValueError):
        o3.Oracle3(p)
    assert o3.lib().o3_new_order(3) is None


# ---------------------------------------------- curvilinear grids (the sphere-in-box family)

def _smooth(X):
    return np.sin(2.0 * X[0] + 0.3) * np.cos(X[1]) * np.exp(0.5 * X[2])


def _lap_error(o3, g):
    orc = o3.Oracle3(_single(g))
    X = _ext_coords(g)
    out = _interior(g, orc.apply_lap(0, _smooth(X)))
    ref = _interior(g, (-4.0 - 1.0 + 0.25) * _smooth(X))
    return np.max(np.abs(out - ref)[g.mask == G.DISC])


@pytest.mark.parametrize("kind", ["shell", "patch"])
def test_mapped_laplacian_fourth_order(o3, kind):
    """The mapped Laplacian (Sec. 3.1) at fourth order -- D+D-(1 - h^2/12 D+D-), the first
    difference D0(1 - h^2/6 D+D-), its tensor product for the mixed a-b term of the pole
    patch, and b_k from fourth-order differences of the metrics -- converges at fourth order
    on a spherical shell and on an orthographic pole patch (Neumann layer included, exact
    ghost values)."""
    errs = []
    for s in (2, 4):
        if kind == "shell":
            g = G3.shell_grid("shell", 32 * s, 16 * s + 1 - s, 8 * s + 1 - s, 0.5, 0.3,
                              40.0, 140.0, order=4)
        else:
            g = G3.pole_patch_grid("north", 16 * s + 1 - s, 8 * s + 1 - s,
                                   math.sin(math.radians(25.0)), 1.5, 0.3, 1.0, order=4)
        errs.append(_lap_error(o3, g))
    assert 3.7 < math.log2(errs[0] / errs[1]) < 4.4, errs


def _affine_grid(n, B, bc, gw=2):
    """A curvilinear grid x = B t (B constant, columns not orthogonal), t in [0, 1]^3 on
    non-periodic axes and [0, 1) on periodic ones; interpolation layers gw thick on the
    faces without a condition."""
    h = tuple(1.0 / (m if bc[2 * a] == P else m - 1) for a, m in enumerate(n))
    gh = tuple(0 if bc[2 * a] == P else gw for a in range(3))
    ext = [n[a] + 2 * gh[a] for a in range(3)]
    Binv = np.linalg.inv(B)
    rx = np.empty((9, ext[2], ext[1], ext[0]))
    for k in range(3):
        for m in range(3):
            rx[3 * k + m] = Binv[k, m]
    mask = np.full((n[2], n[1], n[0]), G.DISC, np.int8)
    sl = [np.s_[:, :, :gw], np.s_[:, :, -gw:], np.s_[:, :gw, :], np.s_[:, -gw:, :],
          np.s_[:gw], np.s_[-gw:]]
    for s in range(6):
        if bc[s] == G.BC_NONE:
            mask[sl[s]] = G.INTERP
    ortho = 0
    for p, (a, b) in enumerate(((0, 1), (0, 2), (1, 2))):
        if abs(B[:, a] @ B[:, b]) < 1e-15:
            ortho |= 1 << p
    g = G3.Grid3("affine", G3.CURVILINEAR, tuple(n), list(bc), h, mask, ortho, rx)
    g.mapping = dict(map=lambda t0, t1, t2: np.einsum("ij,j...->i...", B,
                                                      np.stack([t0, t1, t2])))
    return g


def test_mapped_laplacian_exact_on_quartics_affine(o3):
    """Under an affine map with no orthogonal pair (every mixed term present, b_k = 0) the
    fourth-order mapped Laplacian is exact on polynomials of degree <= 4."""
    B = np.array([[1.0, 0.35, -0.2], [0.1, 0.9, 0.3], [-0.25, 0.15, 1.1]])
    g = _affine_grid((11, 10, 12), B, [G.BC_NONE] * 6)
    assert g.ortho == 0
    orc = o3.Oracle3(_single(g))
    x, y, z = _ext_coords(g)
    u = x ** 4 + 2 * x ** 2 * y * z - y ** 3 * z + 0.5 * z ** 4 + x * y * z + x * x * y * y
    lap = (12 * x ** 2 + 4 * y * z + 2 * y * y) + (-6 * y * z + 2 * x * x) + 6 * z ** 2
    out = _interior(g, orc.apply_lap(0, u))
    assert np.allclose(out[g.mask == G.DISC], _interior(g, lap)[g.mask == G.DISC],
                       rtol=1e-10, atol=1e-9)


def test_curvilinear_description_of_a_slab_equals_cartesian(o3):
    """A periodic/Neumann slab described as a curvilinear grid (x = diag(L) t) gives the
    Cartesian fourth-order operator and, through the curvilinear Neumann ghost rule, the
    same WaveHoltz iteration as the Cartesian description (the Cartesian path is pinned
    above)."""
    n, L = (12, 10, 14), (1.0, 0.8, 0.9)
    bc = [P, P, P, P, N, N]
    cart = G3.cartesian_grid3("s", n, (0.0,) * 3, (11 / 12, 0.8 * 9 / 10, 0.9), bc)
    curv = _affine_grid(n, np.diag(L), bc)
    assert curv.ortho == 7
    f = G3.gaussian3(cart, np.array([0.4, 0.35, 0.45]), 1.0, 20.0)
    po = [G3.Problem3([g], G3.Interp3.empty(), 6.0, [f], order=4) for g in (cart, curv)]
    oc, ov = (o3.Oracle3(p) for p in po)
    assert oc.time.M == ov.time.M and ov.time.dt == pytest.approx(oc.time.dt, rel=1e-13)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(oc.ext_shape(0))
    a, b = oc.apply_lap(0, u), ov.apply_lap(0, u)
    disc = np.zeros(u.shape, bool)
    _interior(cart, disc)[...] = cart.mask == G.DISC
    assert np.max(np.abs(a - b)[disc]) < 1e-12 * np.max(np.abs(a)[disc])
    v = G3.random_state3(po[0], 4)
    for forcing in (True, False):
        r1, r2 = oc.iterate(v, forcing), ov.iterate(v, forcing)
        assert np.max(np.abs(r1 - r2)) < 1e-12 * np.max(np.abs(r1))


def test_neumann_ghost_rule_on_the_sphere_fourth_order(o3):
    """On the shell's sphere face the fourth-order Neumann rule with the fifth-order
    extrapolation reproduces, at both ghost layers, a smooth function with zero normal
    derivative there, with errors that fall at least as h^4."""
    errs = []
    for s in (1, 2):
        g = G3.shell_grid("shell", 32 * s, 16 * s + 1 - s, 8 * s + 1 - s, 0.5, 0.3, 40.0,
                          140.0, order=4)
        orc = o3.Oracle3(_single(g))
        gh = g.ghosts(4)
        t = [np.arange(-gh[a], g.n[a] + gh[a]) * g.h[a] for a in range(3)]
        T2, T1, T0 = np.meshgrid(t[2], t[1], t[0], indexing="ij")
        ph, th = 2 * np.pi * T0, math.radians(40.0) + math.radians(100.0) * T1
        rr = 0.3 * T2  # r - r_in
        u = np.cos(2 * ph) * np.sin(th) ** 2 * (1 + 2 * rr ** 2) * np.exp(-rr ** 3)
        w = u.copy()
        w[:gh[2]] = 0.0
        out = orc.apply_bc(0, w)
        cols = np.zeros(u.shape[1:], bool)  # columns whose sphere point is a disc. point
        cols[gh[1]:gh[1] + g.n[1], :] = g.mask[0] == G.DISC
        errs.append(np.max(np.abs(out[:gh[2]] - u[:gh[2]])[:, cols]))
    assert math.log2(errs[0] / errs[1]) > 4.0, errs


def _sphere4(s):
    return G3.sphere_problem(nb=48 * s, nphi=96 * s, nth=64 * s, nr=16 * s, npatch=40 * s,
                             width=0.8, r_hole=0.83, patch_deg=38.0, omega=6.0, order=4,
                             box=1.5)


def test_sphere_in_box_fourth_order_generator_invariants():
    """Order-4 sphere-in-box: interpolation layers two points thick on the shell and the
    patches, width-5 donor stencils of discretization or Dirichlet points only (explicit
    interpolation), weights summing to 1 per axis, every interpolation point listed once."""
    prob = _sphere4(1)
    it = prob.interp
    assert it.wx.shape[1] == 5
    G3.check_explicit_interp3(prob.grids, it)
    for w in (it.wx, it.wy, it.wz):
        assert np.allclose(w.sum(axis=1), 1.0, atol=1e-13)
    keys = set(zip(it.recv_grid.tolist(), it.recv_i.tolist(), it.recv_j.tolist(),
                   it.recv_k.tolist()))
    assert len(keys) == it.n
    S = prob.grids[1]
    assert np.all(S.mask[-2:] == G.INTERP) and np.all(S.mask[:, :2] == G.INTERP)
    assert np.all(S.mask[:-2, 2:-2] == G.DISC)


def test_sphere_interpolation_fifth_order(o3):
    """Width-5 Lagrange interpolation on the order-4 sphere-in-box grids (curvilinear donors
    and receivers) converges at fifth order under refinement (> 4.3 at these sizes)."""
    errs = []
    for s in (1, 2):
        prob = _sphere4(s)
        orc = o3.Oracle3(prob)
        us = [_smooth(_ext_coords(g)) for g in prob.grids]
        got = orc.interpolate(us)
        e = 0.0
        for gi, g in enumerate(prob.grids):
            rec = np.zeros(orc.ext_shape(gi), bool)
            _interior(g, rec)[...] = g.mask == G.INTERP
            e = max(e, float(np.max(np.abs(got[gi] - us[gi])[rec])))
        errs.append(e)
    assert math.log2(errs[0] / errs[1]) > 4.3, errs
