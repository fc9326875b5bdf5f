"""Pins for the dissipative variant of the 2D oracle's march (the paper's upwind-dissipation
variant, whose form it leaves to its reference): the dissipation acts on the march's
deviation from the periodic motion of the iterate, so that the discrete Helmholtz solution
stays the fixed point exactly -- the "additional correction" the paper asks for -- while
the grid-scale growth of an unstable boundary rule is damped (CPU only)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G


@pytest.fixture(scope="module")
def orc_mod():
    from oracle import oracle
    return oracle


def _rate(orc, n, act=None):
    """Largest |eigenvalue| of the zero-forcing map by power iteration."""
    v = np.random.default_rng(0).standard_normal(n)
    if act is not None:
        v = v * act
    for _ in range(60):
        w = orc.iterate(v, False)
        rate = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    return rate


CASES = [
    ("sheared-channel-53deg-o2", lambda: G.sheared_channel_problem(shear=0.8), 0.1),
    ("square-o4", lambda: G.unit_square_problem(33, 4, 10.0), 0.01),
    ("disk-o4", lambda: G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8,
                                       r_cut=0.75), 0.01),
    ("disk-o2-gn", lambda: G.with_neumann_data(
        G.disk_problem(nb=48, nth=96, nr=10, order=2, omega=4.0, width=0.8, r_cut=0.75),
        lambda x, y: (np.cos(x), -np.sin(y))), 0.02),
]


@pytest.mark.parametrize("name,make,nu", CASES, ids=[c[0] for c in CASES])
def test_dissipative_fixed_point_equals_direct_solve(orc_mod, name, make, nu):
    """With the dissipation on, the direct discrete solution (tests/dhs.py, which knows
    nothing of the dissipation) is still a fixed point of the map, to rounding."""
    import dhs
    p = make()
    orc = orc_mod.Oracle(p, nu=nu)
    U = dhs.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(U, True) - U)[act]) < 1e-12 * np.max(np.abs(U))
    # and the dissipation does change the map away from the fixed point
    v = G.random_state(p, 5)
    assert np.max(np.abs(orc.iterate(v, True) - orc_mod.Oracle(p).iterate(v, True))) > 1e-8


def test_dissipation_stabilizes_the_sheared_neumann_channel(orc_mod):
    """Neumann walls crossed at 53 degrees make the plain march unstable (the zero-forcing
    map has an eigenvalue far above 1); the dissipation brings every |eigenvalue| below 1,
    and GMRES on the dissipative map reaches the direct solution."""
    import dhs
    p = G.sheared_channel_problem(shear=0.8)
    assert _rate(orc_mod.Oracle(p), p.n_total) > 10.0
    orc = orc_mod.Oracle(p, nu=0.1)
    assert _rate(orc, p.n_total) < 1.0
    U = dhs.solve(p)
    v, its, hist = orc_mod.gmres(orc, tol=1e-12, restart=200, max_it=600)
    act = orc.active()
    assert np.max(np.abs(v - U)[act]) < 1e-10 * np.max(np.abs(U)), its


def test_negative_dissipation_refused(orc_mod):
    with pytest.raises(ValueError):
        orc_mod.Oracle(G.unit_square_problem(16, 2, 10.0), nu=-0.1)
