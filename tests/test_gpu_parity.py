"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the same
seeded inputs.  FP64 bar: 1e-12 relative max-norm per WaveHoltz iteration."""
import time

import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available(), "GPU tests need a CUDA device"
    return T


@pytest.fixture(scope="module")
def W():
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz
    return waveholtz


def rel_err(a, b, active):
    return np.max(np.abs(a - b)[active]) / max(np.max(np.abs(b)[active]), 1e-300)


def gpu_iterate(torch, solver, v, forcing):
    vi = torch.from_numpy(v).cuda()
    vo = torch.empty_like(vi)
    solver.iterate(vi, vo, forcing)
    torch.cuda.synchronize()
    return vo.cpu().numpy()


CASES = [
    ("square64-o2", lambda: G.unit_square_problem(64, 2, 10.0), {}),
    ("square37-o4-ragged", lambda: G.unit_square_problem(37, 4, 10.0, seed=2), {}),
    ("channel-neumann-o2", lambda: G.channel_problem(40, 2, 5.0, bc=G.BC_NEUMANN), {}),
    ("channel-neumann-o4", lambda: G.channel_problem(45, 4, 5.0, bc=G.BC_NEUMANN), {}),
    ("channel-dirichlet-o4", lambda: G.channel_problem(40, 4, 5.0, bc=G.BC_DIRICHLET), {}),
    ("torus-o2", lambda: G.sheared_torus_problem(40, 36, 2), {}),
    ("torus-o4", lambda: G.sheared_torus_problem(40, 36, 4), {}),
    ("disk-o2", lambda: G.disk_problem(nb=96, nth=192, nr=14, order=2, omega=8.0, width=0.6,
                                       r_cut=0.7), {}),
    ("disk-o4", lambda: G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0), {}),
    ("disk-o4-cx", lambda: G.disk_problem(nb=96, nth=192, nr=16, order=4, omega=6.0, c_bumps=8,
                                          width=0.6, r_cut=0.7), {}),
    ("disk-o4-2src-Np2-alpha-half", lambda: G.disk_problem(nb=80, nth=160, nr=14, order=4,
                                                           omega=7.0, n_src=2, width=0.6,
                                                           r_cut=0.7, seed=3),
     dict(periods=2, alpha_mode=1)),
    # several bodies: two ellipses on elliptic-coordinate grids and a disk (4 grids)
    ("ellipses-o4", lambda: G.ellipses_problem(nb=192, omega=12.0), {}),
    ("ellipses-o4-Np3", lambda: G.ellipses_problem(nb=160, omega=8.0, seed=2),
     dict(periods=3)),
]


def _two_bodies(order):
    """An ellipse (elliptic-coordinate grid) and a disk in a 64^2 background."""
    bodies = [G.Body((-0.8, -0.3), 0.4, 0.22, 0.6, 64, 12, beta=1.0, cut=0.6),
              G.Body((0.85, 0.45), 0.3, 0.3, 0.6, 56, 12, beta=1.0, cut=0.6)]
    return G.bodies_problem(64, bodies, order=order, omega=4.0, seed=1)


@pytest.mark.parametrize("mode", ["persistent", "graph"])
@pytest.mark.parametrize("name,make,kw", CASES, ids=[c[0] for c in CASES])
def test_iteration_parity(torch, W, oracle_mod, name, make, kw, mode):
    prob = make()
    orc = oracle_mod.Oracle(prob, **kw)
    s = W.Solver(prob, launch_mode=W.PERSISTENT if mode == "persistent" else W.GRAPH, **kw)
    ti = s.prepare()
    assert (ti.Nt, ti.M) == (orc.time.Nt, orc.time.M)
    assert abs(ti.dt - orc.time.dt) <= 1e-15 * orc.time.dt
    assert abs(ti.alpha - orc.time.alpha) <= 1e-14
    act = orc.active()
    for seed, forcing in ((1, True), (2, False)):
        v = G.random_state(prob, seed)
        ref = orc.iterate(v, forcing)
        got = gpu_iterate(torch, s, v, forcing)
        assert rel_err(got, ref, act) <= TOL, (name, forcing, rel_err(got, ref, act))
        assert np.all(got[~act] == 0.0)
    s.close()


def test_unit_square_twenty_iterations(torch, W, oracle_mod):
    """64^2 unit square, order 2, 20 fixed-point iterations from v = 0."""
    prob = G.unit_square_problem(64, 2, 10.0, seed=0)
    orc = oracle_mod.Oracle(prob)
    s = W.Solver(prob)
    s.prepare()
    act = orc.active()
    v_ref = orc.zeros()
    vg = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    out = torch.empty_like(vg)
    for k in range(20):
        v_ref = orc.iterate(v_ref, True)
        s.iterate(vg, out, True)
        vg, out = out, vg
        got = vg.cpu().numpy()
        assert rel_err(got, v_ref, act) <= TOL, (k, rel_err(got, v_ref, act))


def test_full_size_disk_iteration(torch, W, oracle_mod):
    """The full disk-in-square workload (1024^2 background + 2048x64 annulus, order 4,
    omega = 40): one iteration from a seeded random state, every output point."""
    prob = G.disk_problem()
    orc = oracle_mod.Oracle(prob)
    s = W.Solver(prob)
    ti = s.prepare()
    assert ti.M == orc.time.M == 165
    v = G.random_state(prob, 11)
    got = gpu_iterate(torch, s, v, True)
    ref = orc.iterate(v, True)
    assert rel_err(got, ref, orc.active()) <= TOL
    # few ghost-rule/interpolation units next to the march blocks: they are folded into the
    # march launches (init, level 0's ghost rules + interpolation, M steps, output)
    assert s.last_launch_count() == ti.M + 3
    # the FP32-march form at full size (TMA-staged background, annulus by ticket) against the
    # same oracle iteration, within the form's stated bound
    s32 = W.Solver(prob, precision=W.FP32)
    s32.prepare()
    got32 = gpu_iterate(torch, s32, v, True)
    assert rel_err(got32, ref, orc.active()) <= 1e-4


def test_folded_gather_order2(torch, W, oracle_mod):
    """Order 2 with the ghost rules and interpolation folded into the march launches
    (Neumann cylinder, 256^2 background + 512x16 annulus)."""
    prob = G.disk_problem(nb=256, nth=512, nr=16, order=2, omega=10.0, seed=4)
    orc = oracle_mod.Oracle(prob)
    s = W.Solver(prob)
    ti = s.prepare()
    v = G.random_state(prob, 12)
    for forcing in (True, False):
        got = gpu_iterate(torch, s, v, forcing)
        ref = orc.iterate(v, forcing)
        assert rel_err(got, ref, orc.active()) <= TOL
    assert s.last_launch_count() == ti.M + 3


def test_determinism_and_zero(torch, W):
    prob = G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0)
    s = W.Solver(prob)
    s.prepare()
    v = G.random_state(prob, 5)
    a = gpu_iterate(torch, s, v, True)
    b = gpu_iterate(torch, s, v, True)
    assert np.array_equal(a, b)
    z = gpu_iterate(torch, s, np.zeros(prob.n_total), False)
    assert np.all(z == 0.0)
    # host-buffer path equals the device path
    c = s.iterate_host(v, True)
    assert np.array_equal(a, c)
    # init, level 0's ghost rules + interpolation, the steps (M march launches folding in
    # the next level's ghost rules and interpolation, or M pairs), output
    assert s.last_launch_count() in (s.info.M + 3, 2 * s.info.M + 3)
    p = W.Solver(prob, launch_mode=W.PERSISTENT)
    p.prepare()
    d = gpu_iterate(torch, p, v, True)
    assert p.last_launch_count() == 1  # one persistent launch per iteration
    assert np.max(np.abs(d - a)) <= 1e-13 * np.max(np.abs(a))


def test_barrier_timeout_is_reported(torch, W):
    """A grid barrier that runs out of polls makes every block leave the persistent
    kernel; the call reports WH_ERR_TIMEOUT and the GPU context stays usable."""
    prob = G.disk_problem(nb=64, nth=128, nr=12, order=4, omega=5.0, width=0.8, r_cut=0.75)
    s = W.Solver(prob, launch_mode=W.PERSISTENT, barrier_spin_limit=1)
    s.prepare()
    v = G.random_state(prob, 1)
    with pytest.raises(W.WHError) as e:
        s.iterate_host(v, True)
    assert e.value.status == -5
    ok = W.Solver(prob, launch_mode=W.PERSISTENT)
    ok.prepare()
    out = ok.iterate_host(v, True)
    assert np.all(np.isfinite(out))
    assert float(torch.ones(4, device="cuda").sum()) == 4.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_graph_path_wait_timeout_is_reported(torch, W, oracle_mod, prec):
    """The graph path's bounded waits (folded gather's step flags in FP64, TMA stages in
    FP32; copies in flight are drained first) with a spin limit of 1: an iteration either
    completes or reports WH_ERR_TIMEOUT (each poll of an mbarrier may itself wait a while,
    so whether a limit of 1 runs out is up to the hardware), the context stays usable, and
    a solver with the normal limit still gives the oracle's iteration."""
    prob = G.disk_problem(nb=256, nth=512, nr=16, order=4, omega=10.0, seed=6)
    pr = W.FP64 if prec == "fp64" else W.FP32
    s = W.Solver(prob, precision=pr, barrier_spin_limit=1)
    s.prepare()
    v = G.random_state(prob, 13)
    reported = 0
    for _ in range(3):
        try:
            out = s.iterate_host(v, True)
            assert np.all(np.isfinite(out))
        except W.WHError as e:
            assert e.status == -5
            reported += 1
    ok = W.Solver(prob, precision=pr)
    ok.prepare()
    ref = oracle_mod.Oracle(prob).iterate(v, True)
    got = ok.iterate_host(v, True)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    assert rel_err(got, ref, act) <= (TOL if prec == "fp64" else 1e-4)
    assert float(torch.ones(4, device="cuda").sum()) == 4.0


def test_gmres_reaches_direct_solution(torch, W):
    import dhs
    prob = G.disk_problem(nb=48, nth=96, nr=10, order=4, omega=4.0, width=0.8, r_cut=0.75)
    U = dhs.solve(prob)
    s = W.Solver(prob)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-12, max_it=400, restart=200)
    assert st.converged == 1, (st.status, st.residual)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    assert rel_err(u.cpu().numpy(), U, act) < 1e-9
    assert st.history[0] == pytest.approx(1.0)


@pytest.mark.parametrize("order", [2, 4])
def test_gmres_reaches_direct_solution_two_bodies(torch, W, order):
    """An ellipse and a disk in one background (three grids, two of them curvilinear):
    GPU GMRES equals the direct solution of the discrete Helmholtz system."""
    import dhs
    prob = _two_bodies(order)
    U = dhs.solve(prob)
    s = W.Solver(prob)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-12, max_it=400, restart=200)
    assert st.converged == 1, (st.status, st.residual)
    act = np.concatenate([(g.mask != 0).ravel() for g in prob.grids])
    assert rel_err(u.cpu().numpy(), U, act) < 1e-9


def test_fpi_matches_oracle_iterates(torch, W, oracle_mod):
    prob = G.unit_square_problem(40, 4, 10.0, seed=4)
    orc = oracle_mod.Oracle(prob)
    v_ref, _, res = oracle_mod.fpi(orc, 6)
    s = W.Solver(prob)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.FPI, tol=1e-30, max_it=6)
    assert st.iterations == 6 and st.status == "WH_ERR_NOT_CONVERGED"
    assert rel_err(u.cpu().numpy(), v_ref, orc.active()) <= TOL


def test_dot(torch, W):
    prob = G.unit_square_problem(16, 2, 3.0)
    s = W.Solver(prob)
    x = torch.randn(1_000_003, dtype=torch.float64, device="cuda")
    y = torch.randn(1_000_003, dtype=torch.float64, device="cuda")
    d = s.dot(x, y)
    ref = float(np.dot(x.cpu().numpy(), y.cpu().numpy()))
    assert abs(d - ref) <= 1e-12 * np.linalg.norm(x.cpu().numpy()) * np.linalg.norm(y.cpu().numpy())
    assert s.dot(x[:0], y[:0]) == 0.0


def test_errors_on_device(torch, W):
    prob = G.disk_problem(nb=64, nth=128, nr=12, order=4, omega=5.0, width=0.8, r_cut=0.75)
    # a donor that is an interpolation point: explicit interpolation violated
    bad = prob.interp
    k = int(np.nonzero(bad.recv_grid == 1)[0][0])
    bad.donor_j0 = bad.donor_j0.copy()
    bad.donor_grid = bad.donor_grid.copy()
    bad.donor_grid[k] = 0
    bad.donor_i0 = bad.donor_i0.copy()
    jj, ii = np.nonzero(prob.grids[0].mask == G.INTERP)
    bad.donor_i0[k], bad.donor_j0[k] = ii[0] - 1, jj[0] - 1
    s = W.Solver(prob)
    with pytest.raises(W.WHError) as e:
        s.prepare()
    assert e.value.status == -7


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_launch_layout_and_autotune(torch, W, oracle_mod, prec):
    """Every launch layout (persistent; graph with the gather folded; separate gather with
    tiles by ticket or by stride; TMA-staged or plain FP32 march) gives the oracle's
    iteration, and so does the layout the autotuner keeps."""
    prob = G.disk_problem(nb=256, nth=512, nr=16, order=4, omega=10.0, seed=6)
    orc = oracle_mod.Oracle(prob)
    act = orc.active()
    v = G.random_state(prob, 13)
    ref = orc.iterate(v, True)
    tol = TOL if prec == "fp64" else 1e-4
    s = W.Solver(prob, precision=W.FP64 if prec == "fp64" else W.FP32)
    s.prepare()
    layouts = [(W.PERSISTENT, -1, -1, -1, -1), (W.GRAPH, 1, -1, 0, 1), (W.GRAPH, 0, 1, 0, 1),
               (W.GRAPH, 0, 0, 0, 0), (W.GRAPH, 1, -1, 0, 0)]
    if prec == "fp32":
        layouts += [(W.GRAPH, 1, -1, 1, 1), (W.GRAPH, 0, -1, 1, 1), (W.GRAPH, 1, -1, 1, 0)]
    for lay in layouts:
        s.set_tuning(*lay)
        got = gpu_iterate(torch, s, v, True)
        assert rel_err(got, ref, act) <= tol, lay
    t = s.autotune(reps=2)
    assert t["candidates"] >= (7 if prec == "fp64" else 9) and t["ms_per_iteration"] > 0
    got = gpu_iterate(torch, s, v, True)
    assert rel_err(got, ref, act) <= tol, t
