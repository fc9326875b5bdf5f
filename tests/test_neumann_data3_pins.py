"""Pins for Neumann data in the 3D oracle: the ghost rules make the outward normal
derivative gn cos(omega t) instead of 0 (order 2: the centred D0; order 4: the fourth-order
D_n with the extrapolation row), as in two dimensions (CPU only)."""
import math

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

N, P = G.BC_NEUMANN, G.BC_PERIODIC


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3
    return oracle3


def _slab(n, order, om):
    """Periodic in x and y, Neumann at z = 0 and 1, with the manufactured solution
    u = sin(Kx) cos(Ky) cos(z + 0.4) + 0.3 (K the periodic wavenumber), f = Lap u +
    omega^2 u, and its normal derivatives as Neumann data."""
    p = G3.unit_cube_problem(n, omega=om, b=20.0, order=order, bc=[P] * 4 + [N, N])
    g = p.grids[0]
    K = 2 * np.pi / (g.n[0] * g.h[0])

    def U(x, y, z):
        return np.sin(K * x) * np.cos(K * y) * np.cos(z + 0.4) + 0.3

    def grad(x, y, z):
        return (K * np.cos(K * x) * np.cos(K * y) * np.cos(z + 0.4),
                -K * np.sin(K * x) * np.sin(K * y) * np.cos(z + 0.4),
                -np.sin(K * x) * np.cos(K * y) * np.sin(z + 0.4))
    X = g.coords()
    p.f = [(om ** 2 - 2 * K * K - 1.0) * (U(*X) - 0.3) + om ** 2 * 0.3]
    return G3.with_neumann_data3(p, grad), U(*X).ravel()


@pytest.mark.parametrize("order,lo,hi", [(2, 1.75, 2.3), (4, 3.4, 4.5)])
def test_neumann_data_slab_fixed_point_and_convergence(o3, order, lo, hi):
    """The fixed point with Neumann data equals the direct solve of tests/dhs3.py (whose
    rows take the data from the normal-derivative definition), and converges to the
    manufactured solution at the scheme's order (9^3 -> 17^3: 1.86 and 3.62)."""
    import dhs3
    errs = []
    for n in (9, 17):
        p, u = _slab(n, order, 2.0)
        orc = o3.Oracle3(p)
        V = dhs3.solve(p)
        act = orc.active()
        assert np.max(np.abs(orc.iterate(V, True) - V)[act]) < 1e-12 * np.max(np.abs(V))
        errs.append(np.max(np.abs(V - u)))
    assert lo < math.log2(errs[0] / errs[1]) < hi, errs


@pytest.mark.parametrize("order", [2, 4])
def test_neumann_data_on_a_curvilinear_grid(o3, order):
    """On the annular cylinder (Neumann walls at r = a and b; |grad r| != 1 there) the
    fixed point with Neumann data equals the direct solve, and the data change it."""
    import dhs3
    p0 = G3.annular_cylinder_problem(order=order, bc_in=N, bc_out=N)
    p = G3.with_neumann_data3(p0, lambda x, y, z: (np.cos(x) + 0 * y, 0.5 + 0 * x,
                                                    np.sin(2 * np.pi * z)))
    assert max(np.max(np.abs(x)) for x in p.gn) > 0.5
    orc = o3.Oracle3(p)
    V = dhs3.solve(p)
    act = orc.active()
    assert np.max(np.abs(orc.iterate(V, True) - V)[act]) < 1e-12 * np.max(np.abs(V))
    assert np.max(np.abs(V - dhs3.solve(p0))) > 1e-3


def test_neumann_data_where_faces_meet_refused():
    """One value per point cannot hold the data of two faces: the helper refuses Neumann
    data on a cube whose Neumann faces meet."""
    p = G3.unit_cube_problem(9, omega=2.0, bc=N)
    with pytest.raises(ValueError):
        G3.with_neumann_data3(p, lambda x, y, z: (1.0 + 0 * x, 1.0 + 0 * y, 1.0 + 0 * z))
