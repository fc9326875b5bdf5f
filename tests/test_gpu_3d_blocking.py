"""Temporal blocking of the three-dimensional FP32 march: K steps per launch on the units
whose widened box holds no receiver and no rewritten ghost, single steps with the ghost
rules and interpolation in between elsewhere.  Every point's update is the same FP32
arithmetic in the same order, so a blocked iteration must equal the single-step one bit for
bit, on problems with and without overset coupling, at every depth and unit depth."""
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
    return G3.sphere_problem(nb=48, nphi=64, nth=32, nr=10, npatch=20, width=0.5,
                             r_hole=0.75, patch_deg=30.0, omega=omega)


CASES = [
    ("dirichlet-cube-70", lambda: G3.unit_cube_problem(70, omega=9.0)),
    ("neumann-cube-70", lambda: G3.unit_cube_problem(70, omega=7.0, bc=G.BC_NEUMANN, b=20.0)),
    ("sphere-in-box-48", _small_sphere),
    ("box-in-box", lambda: G3.box_in_box_problem()),
]


def _launches(M, K, ctiles_nonempty=True):
    """Launches of one blocked iteration: input, level-0 gather, first step + gather, per
    block of K steps the blocked kernel and K (coupled march + gather), single steps for the
    rest, output."""
    sup = (M - 1) // K
    rest = M - 1 - sup * K
    cm = 1 if ctiles_nonempty else 0
    return 2 + 1 + 2 + sup * (1 + K * (cm + 1)) + 2 * rest


def _iterate(torch, s, v, forcing):
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    s.iterate(vi, vo, forcing)
    torch.cuda.synchronize()
    return vo.cpu().numpy()


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_blocked_iteration_equals_single_step_bitwise(env, name, make):
    torch, O3, W = env
    prob = make()
    s = W.Solver(prob, precision=W.FP32)
    ti = s.prepare()
    v = G3.random_state3(prob, 7)
    s.set_tuning(temporal_depth=1)
    assert s.get_tuning()["blocked_points"] == 0
    ref = {f: _iterate(torch, s, v, f) for f in (True, False)}
    assert s.last_launch_count() == 2 * ti.M + 3
    blocked_any = False
    for K in (2, 3, 4):
        for uz in (8, 32, 64):
            s.set_tuning(temporal_depth=K, unit_depth=uz)
            t = s.get_tuning()
            assert t["temporal_depth"] == K and t["unit_depth"] == uz
            blocked_any |= t["blocked_points"] > 0
            for f in (True, False):
                got = _iterate(torch, s, v, f)
                assert np.array_equal(got, ref[f]), (name, K, uz, f,
                                                     np.max(np.abs(got - ref[f])))
            if t["blocked_points"] > 0:
                n = s.last_launch_count()
                assert n in (_launches(ti.M, K, True), _launches(ti.M, K, False)), n
    if name in ("dirichlet-cube-70", "neumann-cube-70"):
        assert blocked_any


def test_blocked_fp32_within_bound_of_oracle(env):
    """The default (blocked) FP32 march stays within the FP32 form's 1e-4 bound of the FP64
    oracle on the small sphere-in-box, and GMRES with it (two phases) reaches the direct
    discrete solution on the box-in-box grid."""
    import dhs3
    torch, O3, W = env
    prob = _small_sphere()
    orc = O3.Oracle3(prob)
    s = W.Solver(prob, precision=W.FP32)
    s.prepare()
    act = orc.active()
    v = G3.random_state3(prob, 5)
    for f in (True, False):
        got = _iterate(torch, s, v, f)
        ref = orc.iterate(v, f)
        assert np.max(np.abs(got - ref)[act]) <= 1e-4 * np.max(np.abs(ref)[act])
    bp = G3.box_in_box_problem()
    U = dhs3.solve(bp)
    sb = W.Solver(bp, precision=W.FP32)
    sb.prepare()
    sb.set_tuning(temporal_depth=3, unit_depth=8)
    u = torch.zeros(bp.n_total, dtype=torch.float64, device="cuda")
    st = sb.solve(u, W.GMRES, tol=1e-11, max_it=800, restart=200)
    assert st.converged == 1 and st.products_fp32 > 0
    act = np.concatenate([(g.mask != 0).ravel() for g in bp.grids])
    assert np.max(np.abs(u.cpu().numpy() - U)[act]) <= 1e-8 * np.max(np.abs(U))


def test_autotune_3d_depths(env):
    """The 3D autotuner times depths 1..4 with three unit depths and keeps a layout whose
    iteration still equals the single-step one bit for bit."""
    torch, O3, W = env
    prob = G3.unit_cube_problem(70, omega=9.0)
    s = W.Solver(prob, precision=W.FP32)
    s.prepare()
    t = s.autotune(reps=1)
    assert t["candidates"] == 10 and 1 <= t["temporal_depth"] <= 4
    v = G3.random_state3(prob, 2)
    got = _iterate(torch, s, v, True)
    s.set_tuning(temporal_depth=1)
    assert np.array_equal(got, _iterate(torch, s, v, True))
    with pytest.raises(W.WHError):
        s.set_tuning(temporal_depth=5)
    with pytest.raises(W.WHError):
        s.set_tuning(fold_gather=1)


def test_full_size_sphere_blocked_equals_single_step(env):
    """At the full sphere-in-box size (320^3 + shell + 2 patches), depth 4 with 128-plane
    units (a layout the bench's autotuner times), the blocked FP32 iteration equals the
    single-step one bit for bit, and most points advance K steps per launch."""
    torch, O3, W = env
    prob = G3.sphere_problem()
    s = W.Solver(prob, precision=W.FP32)
    s.prepare()
    assert s.get_tuning()["temporal_depth"] == 1  # the library's choice here (86% blocked)
    s.set_tuning(temporal_depth=4, unit_depth=128)
    t = s.get_tuning()
    assert t["temporal_depth"] == 4 and t["blocked_points"] > 0.7 * prob.n_total
    rng = np.random.default_rng(9)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    v = rng.standard_normal(prob.n_total) * act
    a = _iterate(torch, s, v, True)
    s.set_tuning(temporal_depth=1)
    b = _iterate(torch, s, v, True)
    assert np.array_equal(a, b)
