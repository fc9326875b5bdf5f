"""Parity of the three-dimensional CUDA path (through the C ABI) with the 3D CPU oracle."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G
from paper_2504_03074_gb300 import grids3 as G3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from oracle import oracle3 as O3
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    assert torch.cuda.is_available()
    return torch, O3, W


def _small_sphere(omega=6.0):
    # 48^3 background (tiles of 32: one ragged column), 64 x 32 x 10 shell, 20^2 x 10 patches
    return G3.sphere_problem(nb=48, nphi=64, nth=32, nr=10, npatch=20, width=0.5,
                             r_hole=0.75, patch_deg=30.0, omega=omega)


def _cube_c2(n=13):
    prob = G3.unit_cube_problem(n, omega=8.0)
    g = prob.grids[0]
    X = g.coords()
    c = 1.0 + 0.3 * np.exp(-((X[0] - 0.4) ** 2 + (X[1] - 0.6) ** 2 + (X[2] - 0.5) ** 2) / 0.05)
    prob.c2 = [c * c]
    return prob


def _sphere_c2():
    # c(x) = 1 + 0.2 exp(-|x - x1|^2 / 0.2^2) on every grid (per-point weights on the
    # background, c^2 folded into the shell's and patches' coefficients)
    prob = _small_sphere()
    c2 = []
    for g in prob.grids:
        X = g.coords()
        c = 1.0 + 0.2 * np.exp(-((X[0] - 0.55) ** 2 + (X[1] + 0.3) ** 2 + (X[2] - 0.4) ** 2) / 0.04)
        c2.append(c * c)
    prob.c2 = c2
    return prob


CASES = [
    ("sphere-in-box-48", _small_sphere),
    ("box-in-box", lambda: G3.box_in_box_problem()),
    ("dirichlet-cube-37", lambda: G3.unit_cube_problem(37, omega=9.0)),
    ("neumann-cube-21", lambda: G3.unit_cube_problem(21, omega=7.0, bc=G.BC_NEUMANN, b=20.0)),
    ("periodic-cube-17", lambda: G3.unit_cube_problem(17, omega=5.0, bc=G.BC_PERIODIC, b=20.0)),
    ("cube-c(x)-13", _cube_c2),
    ("sphere-in-box-48-c(x)", _sphere_c2),
]


def _rel(got, ref, act):
    return np.max(np.abs(got - ref)[act]) / np.max(np.abs(ref)[act])


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_iteration_matches_oracle_3d(env, name, make):
    """One FP64 WaveHoltz iteration, forcing on and off, from a random state: within 1e-12
    relative max-norm of the oracle; exactly 2M + 3 launches."""
    torch, O3, W = env
    prob = make()
    orc = O3.Oracle3(prob)
    s = W.Solver(prob)
    ti = s.prepare()
    assert ti.Nt == orc.time.Nt and ti.M == orc.time.M
    assert ti.dt == pytest.approx(orc.time.dt, rel=1e-14)
    assert ti.alpha == pytest.approx(orc.time.alpha, rel=1e-13)
    assert ti.n_active == prob.n_active and ti.n_total == prob.n_total
    act = orc.active()
    v = G3.random_state3(prob, 11)
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    for forcing in (True, False):
        s.iterate(vi, vo, forcing)
        torch.cuda.synchronize()
        assert s.L.wh_last_launch_count(s.h) == 2 * ti.M + 3
        got = vo.cpu().numpy()
        ref = orc.iterate(v, forcing)
        assert _rel(got, ref, act) <= 1e-12, (name, forcing, _rel(got, ref, act))
        assert np.all(got[~act] == 0.0)


def test_iteration_host_buffers_3d(env):
    """wh_iterate_host (host in, host out) gives the device call's result bit for bit."""
    torch, O3, W = env
    prob = G3.box_in_box_problem()
    s = W.Solver(prob)
    s.prepare()
    v = G3.random_state3(prob, 3)
    out_h = s.iterate_host(v, True)
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    s.iterate(vi, vo, True)
    torch.cuda.synchronize()
    assert np.array_equal(out_h, vo.cpu().numpy())


def test_fp32_march_within_bound_3d(env):
    """The FP32 march (FP64 filter and interpolation weights) stays within 1e-4 relative
    max-norm of the FP64 oracle per iteration on the small sphere-in-box."""
    torch, O3, W = env
    prob = _small_sphere()
    orc = O3.Oracle3(prob)
    s = W.Solver(prob, precision=W.FP32)
    s.prepare()
    act = orc.active()
    v = G3.random_state3(prob, 5)
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    for forcing in (True, False):
        s.iterate(vi, vo, forcing)
        torch.cuda.synchronize()
        err = _rel(vo.cpu().numpy(), orc.iterate(v, forcing), act)
        assert err <= 1e-4, err


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gmres_matches_direct_solve_3d(env, precision):
    """GMRES on the GPU (Sec. 4.3; the FP32 form: FP32 wave solves, then FP64 ones) reaches
    the direct solution of the discrete Helmholtz system, assembled on the CPU from the
    textbook stencil, on the box-in-box overset grid."""
    import dhs3
    torch, O3, W = env
    prob = G3.box_in_box_problem()
    U = dhs3.solve(prob)
    s = W.Solver(prob, precision=W.FP32 if precision == "fp32" else W.FP64)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-11, max_it=800, restart=200)
    assert st.converged == 1, st.status
    if precision == "fp32":
        assert st.products_fp32 > 0
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    got = u.cpu().numpy()
    assert np.max(np.abs(got - U)[act]) <= 1e-8 * np.max(np.abs(U))


def test_full_size_sphere_in_box(env):
    """The 320^3 + 256 x 128 x 24 + 2 x 96^2 x 24 sphere-in-box at full size: the time setup
    agrees with the oracle's (coefficients and the CFL bound computed on both sides), the
    zero-forcing map is linear to rounding, FP64 and FP32 iterations agree to the FP32
    bound, and a forcing-on iteration equals the zero-forcing one plus W_h(0, f)."""
    torch, O3, W = env
    prob = G3.sphere_problem()
    orc = O3.Oracle3(prob)
    s = W.Solver(prob)
    ti = s.prepare()
    assert (ti.Nt, ti.M) == (orc.time.Nt, orc.time.M)
    assert ti.dt_max == pytest.approx(orc.time.dt_max, rel=1e-12)
    n = prob.n_total
    rng = np.random.default_rng(4)
    act = torch.from_numpy(np.concatenate([(g.mask != 0).ravel() for g in prob.grids])).cuda()
    a = torch.from_numpy(rng.standard_normal(n)).cuda() * act
    b = torch.from_numpy(rng.standard_normal(n)).cuda() * act
    Sa, Sb, Sab, out = (torch.empty_like(a) for _ in range(4))
    s.iterate(a, Sa, False)
    s.iterate(b, Sb, False)
    s.iterate(a + 2.0 * b, Sab, False)
    torch.cuda.synchronize()
    lin = (Sab - Sa - 2.0 * Sb).abs().max().item() / Sab.abs().max().item()
    assert lin < 1e-12, lin
    z = torch.zeros_like(a)
    s.iterate(z, out, True)
    Sf = out.clone()
    s.iterate(a, out, True)
    torch.cuda.synchronize()
    aff = (out - Sa - Sf).abs().max().item() / out.abs().max().item()
    assert aff < 1e-12, aff
    s32 = W.Solver(prob, precision=W.FP32)
    s32.prepare()
    out32 = torch.empty_like(a)
    s32.iterate(a, out32, True)
    torch.cuda.synchronize()
    err = (out32 - out).abs().max().item() / out.abs().max().item()
    assert err < 1e-4, err
