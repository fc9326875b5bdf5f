"""Pins for the implicit-time-stepping WaveHoltz oracle (``oracle/implicit.py``; the
implicit scheme, Eq. WaveSchemeImplicit, Recipe OmegaTildeImplicit): each test checks it
against something the paper or the mathematics fixes, never against itself (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G


@pytest.fixture(scope="module")
def imp():
    from oracle import implicit
    return implicit


def test_recipe_omega_tilde_implicit(imp):
    """Recipe OmegaTildeImplicit: N_t dt omega_i = 2 pi and cos(omega_i dt) = 1 / (1 +
    (omega dt)^2 / 2) (Eq. cosOmegaTilde); dt depends on omega and N_t only (not on the
    mesh); alpha_d from Eq. alphad; fewer than 5 steps per period are refused."""
    for omega, nt in ((10.0, 5), (10.0, 10), (37.5, 7), (3.0, 40)):
        T = imp.implicit_time_setup(omega, nt)
        assert T["omega_i"] * nt * T["dt"] == pytest.approx(2 * math.pi, rel=1e-14)
        assert math.cos(T["omega_i"] * T["dt"]) == pytest.approx(
            1.0 / (1.0 + (omega * T["dt"]) ** 2 / 2.0), rel=1e-13)
        assert T["alpha"] == pytest.approx(
            math.tan(T["omega_i"] * T["dt"] / 2) / math.tan(T["omega_i"] * T["dt"]), rel=1e-14)
    # many steps per period: omega_i -> omega, dt -> T / N_t
    T = imp.implicit_time_setup(2.0, 4000)
    assert T["omega_i"] == pytest.approx(2.0, rel=1e-6)
    with pytest.raises(ValueError):
        imp.implicit_time_setup(10.0, 4)


def test_lambda_implicit_range(imp):
    """Eq. lambdaTildeImplicit maps [0, inf) onto [0, pi / (2 dt)) monotonically, the range
    the paper gives as [0, omega N_t / 4] for many steps per period, and omega onto omega_i
    (Eq. omegaTildeImplicitII)."""
    T = imp.implicit_time_setup(1.0, 200)
    lam = np.array([0.0, 0.5, 1.0, 10.0, 1e3, 1e8])
    li = imp.lambda_implicit(lam, T["dt"])
    assert np.all(np.diff(li) > 0) and li[0] == 0.0
    assert li[-1] < math.pi / (2 * T["dt"])
    assert li[-1] == pytest.approx(1.0 * 200 / 4, rel=1e-3)
    # the mode at lambda = omega goes to omega_i exactly (where beta_d = 1)
    for omega, nt in ((1.0, 200), (10.0, 5), (7.0, 12)):
        T = imp.implicit_time_setup(omega, nt)
        assert imp.lambda_implicit(omega, T["dt"]) == pytest.approx(T["omega_i"], rel=1e-13)


@pytest.mark.parametrize("nt,periods", [(5, 1), (10, 1), (10, 2), (16, 3)])
def test_eigenmodes_are_scaled_by_beta_d_implicit(imp, nt, periods):
    """Theorem FullyDiscreteImplicitWaveHoltzConvergenceRate: a sine mode of the Dirichlet
    unit square (an eigenvector of the 5-point Laplacian with eigenvalue -lambda^2) is an
    eigenvector of the zero-forcing implicit map with eigenvalue
    beta_d(lambda_i; omega_i, T-tilde, alpha_d), lambda_i from Eq. lambdaTildeImplicit: the
    implicit first step, the implicit march, the boundary rows and the filter together."""
    from oracle.oracle import beta_d_sum
    n = 24
    orc = imp.ImplicitOracle(G.unit_square_problem(n, 2, 10.0), n_its=nt, periods=periods)
    T = orc.time
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    rng = np.random.default_rng(nt)
    v = np.zeros((n, n))
    expect = np.zeros_like(v)
    for mx, my in ((1, 1), (2, 3), (7, 5), (20, 21), (22, 22)):
        phi = np.sin(my * np.pi * x)[:, None] * np.sin(mx * np.pi * x)[None, :]
        lam = math.sqrt(4 / h ** 2 * (math.sin(mx * math.pi * h / 2) ** 2 +
                                      math.sin(my * math.pi * h / 2) ** 2))
        b = beta_d_sum(imp.lambda_implicit(lam, T["dt"]), T["omega_i"], T["dt"], T["Nt"],
                       T["alpha"], periods)[0]
        c = rng.standard_normal()
        v += c * phi
        expect += c * b * phi
    out = orc.iterate(v.ravel(), False).reshape(n, n)
    assert np.max(np.abs(out - expect)) < 1e-13 * np.max(np.abs(v))


def _boundary_forcing(prob):
    """The same problem with a forcing that does not vanish on the Dirichlet sides, so that
    the order-4 compatibility rows carry it."""
    import copy
    p = copy.copy(prob)
    p.f = [np.cos(g.xy[0] + 2.0 * g.xy[1]) + 0.5 for g in prob.grids]
    return p


CASES = [
    ("square-o2", lambda: G.unit_square_problem(24, 2, 10.0)),
    ("square-o4-boundary-forcing", lambda: _boundary_forcing(
        G.unit_square_problem(25, 4, 10.0, seed=2))),
    ("disk-o4-boundary-forcing", lambda: _boundary_forcing(
        G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75))),
    ("square-o4", lambda: G.unit_square_problem(25, 4, 10.0, seed=2)),
    ("channel-neumann-o4", lambda: G.channel_problem(30, 4, 5.0, bc=G.BC_NEUMANN)),
    ("disk-o2", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=4.0, width=0.8,
                                       r_cut=0.75)),
    ("disk-o4", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8,
                                       r_cut=0.75)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_implicit_fixed_point_equals_direct_solve(imp, name, make):
    """Recipe OmegaTildeImplicit removes the time discretization error: the discrete
    Helmholtz solution U (assembled independently from textbook stencil tables in
    tests/dhs.py) is a fixed point of the implicit map, and GMRES on the implicit map
    (Sec. 4.3) reaches it."""
    import dhs
    from oracle.oracle import gmres
    prob = make()
    orc = imp.ImplicitOracle(prob, n_its=10)
    U = dhs.solve(prob)
    act = orc.active()
    defect = orc.iterate(U, True) - U
    assert np.max(np.abs(defect)[act]) < 1e-11 * np.max(np.abs(U)), name
    v, its, hist = gmres(orc, tol=1e-12, restart=150, max_it=400)
    assert np.max(np.abs(v - U)[act]) < 1e-9 * np.max(np.abs(U)), (name, its)


def test_time_steps_independent_of_the_mesh(imp):
    """Sec. 4.5: with N_t = 10 implicit steps per period the number of GMRES iterations, and
    so of time steps, does not grow as the mesh is refined; the explicit scheme's steps per
    period grow as 1/h (its CFL bound)."""
    from oracle.oracle import Oracle, gmres
    its_i, steps_e = [], []
    for n in (24, 48):
        prob = G.unit_square_problem(n, 2, 10.0)
        _, its, _ = gmres(imp.ImplicitOracle(prob, n_its=10), tol=1e-10, restart=200, max_it=400)
        its_i.append(its)
        orc = Oracle(prob)
        _, its2, _ = gmres(orc, tol=1e-10, restart=200, max_it=400)
        steps_e.append(its2 * orc.time.M)
    assert its_i[0] == its_i[1], its_i
    assert steps_e[1] > 1.8 * steps_e[0] and steps_e[0] > 10 * its_i[0], steps_e


def test_implicit_refusals(imp):
    with pytest.raises(ValueError):
        imp.ImplicitOracle(G.unit_square_problem(16, 2, 10.0), n_its=4)
    p = G.with_boundary_data(G.unit_square_problem(16, 2, 10.0), lambda x, y: 1.0 + x)
    with pytest.raises(ValueError):
        imp.ImplicitOracle(p)


def test_implicit_eigenvalues_and_deflation_on_the_knife_edge(imp):
    """On the overset knife edge: the slowest eigenvalues of the zero-forcing implicit map
    (ARPACK on S) equal beta_d(lambda_i; omega_i, T-tilde, alpha_d) of their own spatial
    eigenvalues (Rayleigh quotients; Theorem FullyDiscreteImplicitWaveHoltzConvergenceRate);
    and deflating them with the exact inflation (Sec. 4.4, Algorithm 3's purpose: the WH +
    implicit + deflation combination of Sec. 7) reaches the direct solution in fewer GMRES
    products."""
    import dhs
    from oracle import deflation as D
    from oracle.oracle import beta_d_sum, gmres
    p = G.knife_edge_problem(order=2, j=8, omega=20.0, width=0.04, height=0.3, b=300.0)
    orc = imp.ImplicitOracle(p, n_its=10)
    T = orc.time
    Phi, lam2, beta = D.wave_eigenpairs(orc, 8, tol=1e-12)
    theory = beta_d_sum(imp.lambda_implicit(np.sqrt(lam2), T["dt"]), T["omega_i"], T["dt"],
                        T["Nt"], T["alpha"], T["periods"])
    assert np.max(np.abs(beta - theory)) < 1e-8, (beta, theory)
    U = dhs.solve(p)
    act = orc.active()
    u, its_d, _ = D.deflated_gmres_schur(orc, Phi, D.rayleigh_matrix(orc, Phi), tol=1e-12,
                                         restart=200, max_it=600)
    assert np.max(np.abs(u - U)[act]) < 1e-9 * np.max(np.abs(U))
    _, its_p, _ = gmres(orc, tol=1e-12, restart=200, max_it=600)
    assert its_d < 0.8 * its_p, (its_d, its_p)


# ------------------------------------------------------------- three dimensions

def test_eigenmodes_are_scaled_by_beta_d_implicit_3d(imp):
    """The same theorem in three dimensions: sine modes of the Dirichlet unit cube
    (eigenvectors of the 7-point Laplacian, -lambda^2 = -sum_a (4/h^2) sin^2(pi m_a h / 2))
    are eigenvectors of the zero-forcing implicit map with eigenvalue beta_d(lambda_i)."""
    from paper_2504_03074_gb300 import grids3 as G3
    from oracle.oracle import beta_d_sum
    n = 11
    orc = imp.ImplicitOracle(G3.unit_cube_problem(n, omega=6.0), n_its=10, periods=2)
    T = orc.time
    h = 1.0 / (n - 1)
    x = np.arange(n) * h
    rng = np.random.default_rng(3)
    v = np.zeros((n, n, n))
    expect = np.zeros_like(v)
    for m in ((1, 1, 1), (2, 3, 1), (5, 4, 7), (9, 9, 8)):
        phi = (np.sin(m[2] * np.pi * x)[:, None, None] * np.sin(m[1] * np.pi * x)[None, :, None]
               * np.sin(m[0] * np.pi * x)[None, None, :])
        lam = math.sqrt(sum(4 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2 for k in m))
        b = beta_d_sum(imp.lambda_implicit(lam, T["dt"]), T["omega_i"], T["dt"], T["Nt"],
                       T["alpha"], 2)[0]
        c = rng.standard_normal()
        v += c * phi
        expect += c * b * phi
    out = orc.iterate(v.ravel(), False).reshape(n, n, n)
    assert np.max(np.abs(out - expect)) < 1e-13 * np.max(np.abs(v))


def _cases3():
    from paper_2504_03074_gb300 import grids3 as G3
    return [
        ("cube-o2", lambda: G3.unit_cube_problem(9, omega=5.0, b=20.0)),
        ("cube-o4", lambda: G3.unit_cube_problem(9, omega=5.0, b=20.0, order=4)),
        ("box-in-box-o2", lambda: G3.box_in_box_problem()),
        # the paper's implicit pipe run is fourth order (Sec. 6); a shorter period here
        ("pipe-o4", lambda: G3.pipe_problem(j=2, order=4, lz=0.3)),
    ]


@pytest.mark.parametrize("k", range(4), ids=["cube-o2", "cube-o4", "box-in-box-o2", "pipe-o4"])
def test_implicit_fixed_point_equals_direct_solve_3d(imp, k):
    """In three dimensions too the direct discrete solution (tests/dhs3.py) is a fixed point
    of the implicit map (Cartesian cubes at orders 2 and 4, the box-in-box overset grid,
    the pipe at order 4 with the paper's source), and GMRES on the implicit map reaches it."""
    import dhs3
    from oracle.oracle import gmres
    name, make = _cases3()[k]
    prob = make()
    orc = imp.ImplicitOracle(prob, n_its=10)
    U = dhs3.solve(prob)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U)), name
    v, its, hist = gmres(orc, tol=1e-12, restart=150, max_it=300)
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U)), (name, its)
