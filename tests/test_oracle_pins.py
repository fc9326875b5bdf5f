"""Pins for the CPU oracle: each test checks it against something the paper or the
mathematics fixes, never against itself (CPU only)."""
import math

import numpy as np
import pytest
import scipy.fft as sfft

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _golden(name):
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as fh:
        for line in fh:
            line = line.split("#")[0].split()
            if line:
                rows.append(line)
    return rows


# ------------------------------------------------------------------ b_mu, stencils

def test_b_mu_matches_paper(oracle_mod):
    """Theorem uxxCoeff: b_0..b_4 = 1, 1/12, 1/90, 1/560, 1/3150."""
    L = oracle_mod.lib()
    for mu, num, den in _golden("b_mu.txt"):
        assert L.or_b_mu(int(mu)) == pytest.approx(int(num) / int(den), rel=1e-15)


@pytest.mark.parametrize("order", [2, 4])
def test_second_difference_symbol(oracle_mod, order):
    """Applied to e^{ikx} the order-p second difference has symbol
    -(4/h^2) sum_{mu<p/2} b_mu (4 sin^2(kh/2))^mu sin^2(kh/2) (App. C); for p = 4 this is
    -(4/h^2)(s^2 + s^4/3), s = sin(kh/2)."""
    n = 24
    prob = G.channel_problem(n, order, 5.0, bc=G.BC_NEUMANN)
    orc = oracle_mod.Oracle(prob)
    h = prob.grids[0].h[1]
    g = order // 2
    idx = np.arange(-g, n + g)
    for k in (1.0, 7.3, 19.0, 40.0):
        u = np.cos(k * h * idx)[:, None] * np.ones((1, n))  # varies along y only
        out = orc.apply_lap(0, u)
        s2 = math.sin(k * h / 2) ** 2
        sym = -(4.0 / h ** 2) * (s2 + (s2 * s2 / 3.0 if order == 4 else 0.0))
        inner = out[g + 1:g + n - 1, :]
        expect = sym * u[g + 1:g + n - 1, :]
        assert np.allclose(inner, expect, rtol=0, atol=1e-9 * abs(sym))


def test_cfl_constants(oracle_mod):
    """Eq. dtForCartesian: c dt sqrt(sum 1/dx_m^2) = C_{2,p} at CFL 1."""
    for p, cp in _golden("cfl_constants.txt"):
        prob = G.unit_square_problem(33, int(p), 10.0)
        orc = oracle_mod.Oracle(prob, cfl=1.0)
        h = prob.grids[0].h[0]
        assert orc.time.dt_max * math.sqrt(2.0) / h == pytest.approx(float(cp), rel=1e-14)


def test_time_setup_recipe(oracle_mod):
    """Recipe OmegaTildeExplicit on the 64^2 square; sin(omega_e dt/2)/(dt/2) = omega."""
    prob = G.unit_square_problem(64, 2, 10.0)
    ts = oracle_mod.Oracle(prob).time
    assert ts.Nt == int(dict(_golden("unit_square_setup.txt"))["Nt"])
    dt = 2.0 / 10.0 * math.sin(math.pi / ts.Nt)
    assert ts.dt == pytest.approx(dt, rel=1e-15)
    assert ts.omega_e == pytest.approx(2 * math.pi / (ts.Nt * dt), rel=1e-15)
    assert math.sin(ts.omega_e * ts.dt / 2) / (ts.dt / 2) == pytest.approx(10.0, rel=1e-14)
    assert ts.alpha == pytest.approx(math.tan(ts.omega_e * dt / 2) / math.tan(ts.omega_e * dt),
                                     rel=1e-14)
    assert ts.dt <= ts.dt_max
    # alpha_mode = 1 gives the plain alpha = 1/2 of Algorithm 1
    assert oracle_mod.Oracle(prob, alpha_mode=1).time.alpha == 0.5


# ---------------------------------------------------------------- filter functions

def test_beta_d_three_sincs_equals_trapezoid(oracle_mod):
    """Eq. discreteBetaThreeSincs equals the trapezoid sum Eq. betad away from the
    removable points z dt = 2 pi m."""
    O = oracle_mod
    for Nt in (5, 12, 63):
        w = 3.7
        dt = 2 * math.pi / (w * Nt)
        a = O.alpha_d(w, dt)
        lam = np.linspace(0.01, 3.0 * w, 997)
        bad = np.isclose(np.mod((w + lam) * dt, 2 * math.pi), 0, atol=1e-6)
        s1 = O.beta_d_sum(lam, w, dt, Nt, a)
        s2 = O.beta_d_sincs(lam, w, dt, Nt, a)
        assert np.max(np.abs(s1 - s2)[~bad]) < 1e-12


def test_beta_d_peak_at_omega(oracle_mod):
    """beta_d(omega) = 1 for any alpha; alpha_d makes d beta_d / d lambda vanish there
    (Eq. alphadII); alpha = 1/2 does not."""
    O = oracle_mod
    w, Nt = 2.0, 10
    dt = 2 * math.pi / (w * Nt)
    ad = O.alpha_d(w, dt)
    for a in (ad, 0.5):
        assert O.beta_d_sum([w], w, dt, Nt, a)[0] == pytest.approx(1.0, abs=1e-14)
    eps = 1e-5
    der = lambda a: (O.beta_d_sum([w + eps], w, dt, Nt, a)[0] -
                     O.beta_d_sum([w - eps], w, dt, Nt, a)[0]) / (2 * eps)
    assert abs(der(ad)) < 1e-8
    assert abs(der(0.5)) > 1e-3


def test_continuous_beta(oracle_mod):
    """Eq. filterThreeSincs with alpha = 1/2: beta(omega) = 1 and |beta| < 1 elsewhere."""
    O = oracle_mod
    w = 3.0
    T = 2 * math.pi / w
    lam = np.linspace(0, 10 * w, 20001)
    b = O.beta_continuous(lam, w, T)
    assert O.beta_continuous(np.array([w]), w, T)[0] == pytest.approx(1.0, abs=1e-15)
    far = np.abs(lam - w) > 1e-3
    assert np.max(np.abs(b[far])) < 1.0
    # the second closed form of Sec. 4.1, read with alpha/(2 lambda): integrating
    # Eq. filterFunction gives (2/T) sin(lam T) (lam/(lam^2 - w^2) - alpha/(2 lam)),
    # which is what the three-sinc form expands to (the printed alpha/lambda drops the 2)
    lam2 = lam[(lam > 0) & (np.abs(lam - w) > 1e-3)]
    alt = 2.0 / T * np.sin(lam2 * T) * (lam2 / (lam2 ** 2 - w ** 2) - 0.5 / (2 * lam2))
    assert np.allclose(O.beta_continuous(lam2, w, T), alt, atol=1e-12)


# -------------------------------------------------- iteration map: spectral closed form

def _square_closed_form(prob, ts, k_list):
    """Per-mode iterates v^(k) = sum_m (1 - beta_d(lam~_m)^k) U_m Phi_m on the square with
    DST-I modes (Sec. 4.2: Eqs. WhatExplicit, updateDiscreteExplicit, discrete
    eigenvalues of D+D- with Dirichlet data)."""
    n = prob.grids[0].n[0]
    h = prob.grids[0].h[0]
    f = prob.f[0][1:-1, 1:-1]
    fh = sfft.dstn(f, type=1, norm="ortho")
    m = np.arange(1, n - 1)
    sx = np.sin(m * np.pi * h / 2) ** 2
    lam2 = (4 / h ** 2) * (sx[None, :] + sx[:, None])
    from oracle.oracle import beta_d_sum, lambda_tilde
    lt = lambda_tilde(np.sqrt(lam2).ravel(), ts.dt)
    bd = beta_d_sum(lt, ts.omega_e, ts.dt, ts.Nt, ts.alpha).reshape(lam2.shape)
    U = fh / (prob.omega ** 2 - lam2)
    return {k: sfft.idstn((1 - bd ** k) * U, type=1, norm="ortho") for k in k_list}, bd


def test_unit_square_iterates_match_spectral_form(oracle_mod):
    """64^2 unit square, order 2, 20 fixed-point iterations from v = 0."""
    prob = G.unit_square_problem(64, 2, 10.0, seed=0)
    orc = oracle_mod.Oracle(prob)
    _, hist, res = oracle_mod.fpi(orc, 20)
    ref, bd = _square_closed_form(prob, orc.time, range(1, 21))
    for k in range(1, 21):
        got = hist[k].reshape(64, 64)
        assert np.max(np.abs(got[1:-1, 1:-1] - ref[k])) < 1e-13 * np.max(np.abs(ref[k]))
        assert np.all(got[0, :] == 0) and np.all(got[:, 0] == 0)
    # each discrete eigenmode is an eigenvector of S with eigenvalue beta_d(lam~_m)
    # (Eq. waveHoltzFourierFPIexplicit); the slowest decides the ACR of Theorem
    # FullyDiscreteExplicitWaveHoltzConvergenceRate (about 0.99965 here)
    h = prob.grids[0].h[0]
    x = np.arange(64) * h
    for (mx, my) in ((1, 1), (3, 2), (2, 3), (17, 40), (62, 62)):
        phi = np.outer(np.sin(my * np.pi * x), np.sin(mx * np.pi * x))
        out = orc.iterate(phi.ravel(), forcing=False).reshape(64, 64)
        assert np.max(np.abs(out - bd[my - 1, mx - 1] * phi)) < 1e-13
    assert np.max(np.abs(bd)) == pytest.approx(0.99965, abs=1e-5)


# ------------------------------------------------------- operators: order of accuracy

def _annulus_ext(A, order):
    gh = A.ghosts(order)
    nth, nr = A.n
    m = A.mapping
    s = np.arange(-gh[1], nr + gh[1]) / (nr - 1)
    t = np.arange(nth) / nth
    R = m["r_in"] + m["width"] * (np.exp(m["beta"] * s) - 1) / (np.exp(m["beta"]) - 1)
    return R[:, None] * np.cos(2 * np.pi * t)[None, :], R[:, None] * np.sin(2 * np.pi * t)[None, :]


def _smooth(x, y):
    return np.sin(1.3 * x + 0.4) * np.cos(0.7 * y) + x * y * y


def _smooth_lap(x, y):
    return -(1.3 ** 2 + 0.7 ** 2) * np.sin(1.3 * x + 0.4) * np.cos(0.7 * y) + 2 * x


@pytest.mark.parametrize("order", [2, 4])
def test_mapped_laplacian_order_annulus(oracle_mod, order):
    """Mapping method (Sec. 3.1) on the stretched annulus converges at order p."""
    errs = []
    for k in (2, 4):
        A = G.annulus_grid("a", 64 * k, 8 * k + 1, 0.5, 0.6, 1.5, order)
        prob = G.Problem([A], G.Interp.empty(order), order, 3.0, [np.zeros(A.mask.shape)])
        orc = oracle_mod.Oracle(prob)
        X, Y = _annulus_ext(A, order)
        out = orc.apply_lap(0, _smooth(X, Y))
        gh = A.ghosts(order)
        mk = np.zeros(X.shape, bool)
        mk[gh[1]:gh[1] + A.n[1], :] = A.mask == G.DISC
        errs.append(np.max(np.abs(out - _smooth_lap(X, Y))[mk]))
    assert math.log2(errs[0] / errs[1]) > order - 0.3


@pytest.mark.parametrize("order", [2, 4])
def test_mapped_laplacian_order_sheared(oracle_mod, order):
    """Non-orthogonal doubly periodic mapping: the mixed-derivative term is exercised."""
    errs = []
    for k in (1, 2):
        T = G.sheared_torus_grid("t", 32 * k, 32 * k, 0.1, 0.08, order)
        prob = G.Problem([T], G.Interp.empty(order), order, 3.0, [np.zeros(T.mask.shape)])
        orc = oracle_mod.Oracle(prob)
        X, Y = T.xy
        # periodic smooth function of the torus coordinates
        u = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) + 0.5 * np.cos(4 * np.pi * X)
        lu = -8 * np.pi ** 2 * np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y) \
            - 8 * np.pi ** 2 * np.cos(4 * np.pi * X)
        errs.append(np.max(np.abs(orc.apply_lap(0, u) - lu)))
    assert math.log2(errs[0] / errs[1]) > order - 0.3


def test_annulus_coefficients_analytic(oracle_mod):
    """a_kl and b_k of the polar mapping against their closed forms:
    a11 = 1/(2 pi r)^2, a12 = 0, a22 = 1/r'(s)^2, b1 = Lap t = 0, b2 = Lap s."""
    order = 4
    A = G.annulus_grid("a", 256, 33, 0.5, 0.3, 1.5, order)
    prob = G.Problem([A], G.Interp.empty(order), order, 3.0, [np.zeros(A.mask.shape)])
    orc = oracle_mod.Oracle(prob)
    gh = A.ghosts(order)
    X, Y = _annulus_ext(A, order)
    r = np.hypot(X, Y)
    m = A.mapping
    eb = math.exp(m["beta"]) - 1
    s = np.log1p((r - m["r_in"]) * eb / m["width"]) / m["beta"]
    rs = m["width"] * m["beta"] * np.exp(m["beta"] * s) / eb
    rss = m["beta"] * rs
    a11, a22 = 1 / (2 * np.pi * r) ** 2, 1 / rs ** 2
    # s(r) radial: Lap s = s'' + s'/r, s' = 1/r', s'' = -r''/r'^3
    b2 = -rss / rs ** 3 + 1 / (rs * r)
    mk = np.zeros(X.shape, bool)
    mk[gh[1]:gh[1] + A.n[1], :] = A.mask == G.DISC
    for which, ref, tol in ((0, a11, 1e-12), (2, a22, 1e-12), (3, 0 * r, 1e-9), (4, b2, 2e-5)):
        got = orc.coef(0, which)
        assert np.max(np.abs(got - ref)[mk]) <= tol * np.max(np.abs(ref) + 1)
    assert np.max(np.abs(orc.coef(0, 1)[mk])) < 1e-12


# ------------------------------------------------------------------- ghost rules

@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_order4_ghost_values_converge(oracle_mod, kind):
    """The order-4 ghost rules reproduce the ghost values of a smooth function that
    satisfies the boundary condition (and, for Dirichlet, c^2 Lap u = f on the
    boundary) with error falling at least like h^4."""
    errs = []
    for n in (21, 41):
        if kind == "neumann":
            prob = G.channel_problem(n, 4, 5.0, bc=G.BC_NEUMANN)
            g = prob.grids[0]
            X = np.broadcast_to((np.arange(n) / n)[None, :], (n + 4, n))
            Y = np.broadcast_to((np.arange(-2, n + 2) * g.h[1])[:, None], (n + 4, n))
            u = np.cos(2 * np.pi * X) * np.cos(np.pi * Y) + np.cos(3 * np.pi * Y)
            orc = oracle_mod.Oracle(prob)
            w = u.copy()
            w[:2, :] = w[-2:, :] = 0.0
            out = orc.apply_bc(0, w, 1.0)
            errs.append(max(np.max(np.abs(out[:2] - u[:2])), np.max(np.abs(out[-2:] - u[-2:]))))
            continue
        prob = G.unit_square_problem(n, 4, 5.0, bc=G.BC_DIRICHLET)
        g = prob.grids[0]
        h = g.h[0]
        idx = np.arange(-2, n + 2) * h
        X, Y = np.meshgrid(idx, idx)
        if True:
            u = np.sin(np.pi * X) * np.sin(2 * np.pi * Y) * np.exp(X + Y)
            # f with c^2 Lap u = f on the boundary points
            lap = (np.exp(X + Y) * (np.sin(2 * np.pi * Y) * ((1 - np.pi ** 2) * np.sin(np.pi * X)
                   + 2 * np.pi * np.cos(np.pi * X)) + np.sin(np.pi * X) *
                   ((1 - 4 * np.pi ** 2) * np.sin(2 * np.pi * Y) + 4 * np.pi * np.cos(2 * np.pi * Y))))
            prob.f = [lap[2:-2, 2:-2]]
        orc = oracle_mod.Oracle(prob)
        w = u.copy()
        w[:2, :] = w[-2:, :] = 0.0
        w[:, :2] = w[:, -2:] = 0.0
        out = orc.apply_bc(0, w, 1.0)
        # ghost points next to non-corner boundary points
        err = max(np.max(np.abs(out[2:-2, :2] - u[2:-2, :2])[1:-1]),
                  np.max(np.abs(out[:2, 2:-2] - u[:2, 2:-2])[:, 1:-1]))
        errs.append(err)
    assert math.log2(errs[0] / errs[1]) > 3.8


# ------------------------------------------------------------------ interpolation

@pytest.mark.parametrize("order", [2, 4])
def test_lagrange_weights_exact_on_polynomials(order):
    """Width-(p+1) Lagrange weights reproduce polynomials of degree <= p (Sec. 3.1)."""
    xi = np.linspace(-0.7, order + 0.7, 31)
    w = G.lagrange_weights(xi, order + 1)
    nodes = np.arange(order + 1)
    for d in range(order + 1):
        assert np.allclose(w @ nodes ** d, xi ** d, atol=1e-12 * (order + 1) ** d)


@pytest.mark.parametrize("order", [2, 4])
def test_overset_interpolation_order(oracle_mod, order):
    """Receivers interpolated from a smooth function converge at order p+1."""
    errs = []
    for k in (2, 4):
        prob = G.disk_problem(nb=40 * k + 1, nth=80 * k, nr=8 * k + 1, order=order, omega=3.0,
                              width=0.8, r_cut=0.7)
        orc = oracle_mod.Oracle(prob)
        exts, truth = [], []
        for gi, g in enumerate(prob.grids):
            gh = g.ghosts(order)
            e = np.zeros(orc.ext_shape(gi))
            e[gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]] = _smooth(*g.xy)
            exts.append(e)
            truth.append(_smooth(*g.xy))
        # receivers start from garbage so that only the interpolation sets them
        for gi, g in enumerate(prob.grids):
            gh = g.ghosts(order)
            blk = exts[gi][gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]
            blk[g.mask == G.INTERP] = 1e3
        out = orc.interpolate(exts)
        err = 0.0
        for gi, g in enumerate(prob.grids):
            gh = g.ghosts(order)
            blk = out[gi][gh[1]:gh[1] + g.n[1], gh[0]:gh[0] + g.n[0]]
            m = g.mask == G.INTERP
            err = max(err, np.max(np.abs(blk - truth[gi])[m]))
        errs.append(err)
    assert math.log2(errs[0] / errs[1]) > order + 1 - 0.5


def test_explicit_interpolation_invariant():
    """Donor stencils contain only discretization points (explicit interpolation)."""
    prob = G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0)
    G.check_explicit_interp(prob.grids, prob.interp, 4)
    it = prob.interp
    assert it.n > 0
    assert np.all(prob.grids[0].mask[it.recv_j[it.recv_grid == 0], it.recv_i[it.recv_grid == 0]]
                  == G.INTERP)
    assert np.allclose(it.wx.sum(1), 1) and np.allclose(it.wy.sum(1), 1)


# ---------------------------------------------- fixed point = direct discrete solve

DHS_CASES = [
    ("square-o2", lambda: G.unit_square_problem(16, 2, 10.0), 1e-11),
    ("square-o4", lambda: G.unit_square_problem(20, 4, 10.0), 1e-11),
    ("channel-neumann-o2", lambda: G.channel_problem(20, 2, 5.0, bc=G.BC_NEUMANN), 1e-11),
    ("channel-neumann-o4", lambda: G.channel_problem(20, 4, 5.0, bc=G.BC_NEUMANN), 1e-11),
    ("channel-dirichlet-o4", lambda: G.channel_problem(20, 4, 5.0, bc=G.BC_DIRICHLET), 1e-11),
    ("torus-o2", lambda: G.sheared_torus_problem(24, 20, 2), 1e-11),
    ("torus-o4", lambda: G.sheared_torus_problem(24, 20, 4), 1e-11),
    ("disk-o2", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=4.0, width=0.8,
                                       r_cut=0.75), 1e-9),
    ("disk-o4", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8,
                                       r_cut=0.75), 1e-9),
    ("ellipse-disk-o2", lambda: _two_bodies(2), 1e-9),
    ("ellipse-disk-o4", lambda: _two_bodies(4), 1e-9),
]


def _two_bodies(order):
    """An ellipse (elliptic-coordinate grid) and a disk in a 64^2 background."""
    bodies = [G.Body((-0.8, -0.3), 0.4, 0.22, 0.6, 64, 12, beta=1.0, cut=0.6),
              G.Body((0.85, 0.45), 0.3, 0.3, 0.6, 56, 12, beta=1.0, cut=0.6)]
    return G.bodies_problem(64, bodies, order=order, omega=4.0, seed=1)


@pytest.mark.parametrize("name,make,tol", DHS_CASES, ids=[c[0] for c in DHS_CASES])
def test_fixed_point_equals_direct_solve(oracle_mod, name, make, tol):
    """Sec. 6: the converged WaveHoltz solution equals the direct solution of the
    discrete Helmholtz system; the oracle's GMRES (Sec. 4.3) reaches it."""
    import dhs
    prob = make()
    orc = oracle_mod.Oracle(prob)
    U = dhs.solve(prob)
    # the direct solution is a fixed point of the iteration map
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)) < 1e-11 * np.max(np.abs(U))
    v, its, hist = oracle_mod.gmres(orc, tol=1e-13, restart=200, max_it=400)
    act = orc.active()
    assert np.max(np.abs(v - U)[act]) < tol * np.max(np.abs(U))


@pytest.mark.parametrize("order,bc", [(2, G.BC_DIRICHLET), (4, G.BC_DIRICHLET),
                                      (2, G.BC_NEUMANN), (4, G.BC_NEUMANN)])
def test_eigenfunction_solution_order(oracle_mod, order, bc):
    """Helmholtz solution phi = sin(pi x) sin(2 pi y) on the Dirichlet square, and
    phi = cos(2 pi x) cos(pi y) on the periodic channel with Neumann walls, with
    f = (omega^2 - 5 pi^2) phi: the oracle's WaveHoltz solution converges at order p."""
    om = 3.0
    fn = (lambda x, y: np.sin(np.pi * x) * np.sin(2 * np.pi * y)) if bc == G.BC_DIRICHLET else \
        (lambda x, y: np.cos(2 * np.pi * x) * np.cos(np.pi * y))
    errs = []
    for n in (17, 33):
        prob = G.unit_square_problem(n, order, om, bc=bc) if bc == G.BC_DIRICHLET else \
            G.channel_problem(n, order, om, bc=bc)
        X, Y = prob.grids[0].xy
        prob.f = [(om ** 2 - 5 * np.pi ** 2) * fn(X, Y)]
        orc = oracle_mod.Oracle(prob)
        v, its, hist = oracle_mod.gmres(orc, tol=1e-12, restart=100, max_it=300)
        errs.append(np.max(np.abs(v.reshape(n, n) - fn(X, Y))))
    assert math.log2(errs[0] / errs[1]) > order - 0.3


@pytest.mark.slow
def test_overset_self_convergence(oracle_mod):
    """Richardson-style self-convergence on three nested disk grids (Sec. 6.4): the
    order-4 direct discrete solution (equal to the oracle's fixed point) converges at
    better than third order; order 2 at second order."""
    import dhs

    def diff(pc, uc, pf, uf):
        d = 0.0
        for gi, (a, b) in enumerate(zip(pc.split(uc), pf.split(uf))):
            m = (pc.grids[gi].mask != 0) & (pf.grids[gi].mask[::2, ::2] != 0)
            d = max(d, np.max(np.abs(a - b[::2, ::2])[m]))
        return d

    for order, ks, rate in ((2, (1, 2, 4), 1.8), (4, (2, 4, 8), 2.7)):
        sols = []
        for k in ks:
            p = G.disk_problem(nb=40 * k + 1, nth=80 * k, nr=8 * k + 1, order=order, omega=3.0,
                               width=0.6 if order == 2 else 0.8, r_cut=0.7)
            p.f = [G.gaussian(g.xy, (1.0, 0.8), 1.0, 20.0) for g in p.grids]
            sols.append((p, dhs.solve(p)))
        e1 = diff(*sols[0], *sols[1])
        e2 = diff(*sols[1], *sols[2])
        assert math.log2(e1 / e2) > rate


# ----------------------------------------------------------------- rejected input

def test_rejects_unsupported_grids(oracle_mod):
    # physical sides on a non-orthogonal grid are defined at order 2 only
    T = G.sheared_torus_grid("t", 16, 16, 0.1, 0.1, 4)
    T.bc = [G.BC_DIRICHLET] * 4
    prob = G.Problem([T], G.Interp.empty(4), 4, 3.0, [np.zeros(T.mask.shape)])
    with pytest.raises(ValueError):
        oracle_mod.Oracle(prob)
    for bcs in ([G.BC_DIRICHLET, G.BC_DIRICHLET, G.BC_NEUMANN, G.BC_NEUMANN],
                [G.BC_NEUMANN] * 4):
        g = G.cartesian_grid("c", 8, 8, 0, 1, 0, 1, bcs, 2)
        prob = G.Problem([g], G.Interp.empty(2), 2, 3.0, [np.zeros(g.mask.shape)])
        with pytest.raises(ValueError):
            oracle_mod.Oracle(prob)
