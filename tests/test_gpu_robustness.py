"""GPU checks of the library's service paths: the FP32 -> FP64 widening of the FP32 march's
filter against the hardware conversion (bit for bit), the FP64 throughput probe, the folded
gather's fallbacks (a residency cap, an expired wait), divergence detection, and deflated
GMRES against the oracle."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


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


def _rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_widen_matches_hardware_conversion(torch, W):
    """Every exponent with both signs and edge fractions, signed zeros, subnormals,
    infinities, NaNs and a stride-257 sweep of all 2^32 bit patterns: the integer widening
    gives exactly the bits of the hardware float -> double conversion."""
    fr = np.array([0, 1, 2, 0x3FF, 0x400000, 0x555555, 0x7FFFFE, 0x7FFFFF], np.uint32)
    exps = np.arange(256, dtype=np.uint32)
    pats = [(s << 31) | (e << 23) | f for s in (0, 1) for e in exps for f in fr]
    sweep = np.arange(0, 2 ** 32, 257, dtype=np.uint64).astype(np.uint32)
    bits = np.concatenate([np.array(pats, np.uint32), sweep])
    x = torch.from_numpy(bits.view(np.float32)).cuda()
    out = torch.empty(x.numel(), dtype=torch.float64, device="cuda")
    W.widen_f32(x, out)
    ref = x.double()
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint64)
    want = ref.cpu().numpy().view(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (bad[:5], bits[bad[:5]])
    assert x.numel() > 16_000_000


def test_fp64_probe_is_plausible(torch, W):
    """The FP64 FMA probe reports a throughput within a plausible band for this part."""
    tf, ms = W.probe_fp64(3)
    assert 0.2 < tf < 5.0 and ms > 0


def _disk():
    return G.disk_problem(nb=256, nth=512, nr=16, order=4, omega=10.0, seed=6)


def test_resident_cap_uses_separate_gather(torch, W, oracle_mod):
    """With a residency cap below the folded layout's grid the ghost rules and
    interpolation run as their own kernel after every march launch (2M + 3 launches) and
    the persistent kernel's grid is capped; both still give the oracle's iteration."""
    prob = _disk()
    v = G.random_state(prob, 3)
    ref = oracle_mod.Oracle(prob).iterate(v, True)
    s = W.Solver(prob, resident_blocks=4)
    ti = s.prepare()
    got = s.iterate_host(v, True)
    assert s.last_launch_count() == 2 * ti.M + 3
    assert _rel(got, ref) <= 1e-12
    p = W.Solver(prob, launch_mode=W.PERSISTENT, resident_blocks=8)
    p.prepare()
    assert _rel(p.iterate_host(v, True), ref) <= 1e-12


def test_folded_wait_timeout_falls_back(torch, W, oracle_mod):
    """A folded gather unit whose bounded wait expires (a spin limit of 1) is reported as
    WH_ERR_TIMEOUT once; the context then runs the gather as its own kernel and gives the
    oracle's iteration."""
    prob = _disk()
    v = G.random_state(prob, 4)
    ref = oracle_mod.Oracle(prob).iterate(v, True)
    s = W.Solver(prob, barrier_spin_limit=1)
    ti = s.prepare()
    reported = 0
    for _ in range(4):
        try:
            s.iterate_host(v, True)
        except W.WHError as e:
            assert e.status == -5
            reported += 1
    got = s.iterate_host(v, True)
    assert reported <= 1
    if reported:
        assert s.last_launch_count() == 2 * ti.M + 3
    assert _rel(got, ref) <= 1e-12


@pytest.mark.parametrize("method", ["fpi", "gmres"])
def test_unstable_march_is_reported_as_diverged(torch, W, method):
    """A time step above the stability limit (cfl 1.6) makes the march grow without bound;
    the solvers stop with WH_ERR_DIVERGED (growth of the FPI differences, or a GMRES product
    far above the bound of a stable map) instead of iterating to the limit."""
    prob = G.unit_square_problem(32, 2, 6.0, seed=1)
    s = W.Solver(prob, cfl=1.6)
    s.prepare()
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    with pytest.raises(W.WHError) as e:
        s.solve(u, W.FPI if method == "fpi" else W.GMRES, tol=1e-10, max_it=200, restart=30)
    assert e.value.status == -4
    ok = W.Solver(prob)
    ok.prepare()
    st = ok.solve(torch.zeros_like(u), W.GMRES, tol=1e-8, max_it=300, restart=60)
    assert st.converged


def _square_modes(prob, ts, K):
    """The K DST-I modes of the unit square with |beta_d| nearest 1 (orthonormal, compact)
    and their eigenvalues lambda_h^2."""
    import scipy.fft as sfft
    from oracle.oracle import beta_d_sum, lambda_tilde
    n, h = prob.grids[0].n[0], prob.grids[0].h[0]
    m = np.arange(1, n - 1)
    sx = np.sin(m * np.pi * h / 2) ** 2
    lam2 = (4 / h ** 2) * (sx[None, :] + sx[:, None])
    bd = beta_d_sum(lambda_tilde(np.sqrt(lam2).ravel(), ts.dt), ts.omega_e, ts.dt, ts.Nt,
                    ts.alpha).reshape(lam2.shape)
    Phi, l2 = [], []
    for q in np.argsort(-np.abs(bd).ravel())[:K]:
        i, j = np.unravel_index(q, bd.shape)
        z = np.zeros((n - 2, n - 2))
        z[i, j] = 1.0
        phi = np.zeros((n, n))
        phi[1:-1, 1:-1] = sfft.idstn(z, type=1, norm="ortho")
        Phi.append(phi.ravel())
        l2.append(lam2[i, j])
    return np.array(Phi), np.array(l2)


def test_deflated_gmres_matches_oracle_and_direct_solve(torch, W, oracle_mod):
    """GMRES on the deflated fixed-point iteration of Algorithm 3 (8 DST modes of the 48^2
    unit square, the self-adjoint case where the inflation is exact) reaches the oracle's
    deflated GMRES solution and the direct solution of the discrete Helmholtz system."""
    import dhs
    from oracle import deflation as D
    prob = G.unit_square_problem(48, 2, 10.0, seed=2)
    orc = oracle_mod.Oracle(prob)
    Phi, l2 = _square_modes(prob, orc.time, 8)
    f = prob.f[0].ravel()
    ref, its, _ = D.deflated_gmres(orc, Phi, l2, f, prob.omega, tol=1e-12)
    U = dhs.solve(prob)
    s = W.Solver(prob)
    s.prepare()
    phi = torch.from_numpy(Phi).cuda().contiguous()
    s.set_deflation(phi, l2)
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.GMRES, tol=1e-12, max_it=2000, restart=100)
    assert st.converged
    got = u.cpu().numpy()
    assert _rel(got, ref) <= 1e-9
    assert _rel(got, U) <= 1e-9
    # the deflated problem needs fewer products than the plain one
    s.set_deflation(None)
    u0 = torch.zeros_like(u)
    st0 = s.solve(u0, W.GMRES, tol=1e-12, max_it=4000, restart=100)
    assert st0.converged and st.iterations < st0.iterations


def test_rejected_forcing_leaves_the_problem_unchanged(torch, W):
    """A wh_set_forcing refused for non-finite values stores nothing: after it (and a new
    prepare) an iteration gives the result it gave before the refused call, bit for bit."""
    prob = G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0, seed=5)
    s = W.Solver(prob)
    s.prepare()
    v = G.random_state(prob, 6)
    before = s.iterate_host(v, True)
    bad = np.array(prob.f[0], dtype=np.float64, copy=True)
    bad.flat[17] = np.inf
    with pytest.raises(W.WHError) as e:
        s.set_forcing(0, bad)
    assert e.value.status == -1
    s.prepare()
    assert np.array_equal(s.iterate_host(v, True), before)


def test_new_forcing_after_a_deflated_solve(torch, W, oracle_mod):
    """A new forcing (which rebuilds the device layout at the next prepare) after solves that
    allocated the deflation and checkpoint buffers: the next deflated GMRES solve runs on
    fresh buffers and reaches the oracle's solution for the new source (the 48^2 unit
    square, 8 DST modes)."""
    import dhs
    prob = G.unit_square_problem(48, 2, 10.0, seed=2)
    s = W.Solver(prob)
    orc = oracle_mod.Oracle(prob)
    s.prepare()
    Phi, l2 = _square_modes(prob, orc.time, 8)
    phi = torch.from_numpy(Phi).cuda().contiguous()
    s.set_deflation(phi, l2)
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    s.solve(u, W.GMRES, tol=1e-12, max_it=30, restart=20)  # stops: a saved state exists
    p2 = G.unit_square_problem(48, 2, 10.0, seed=7)
    s.set_forcing(0, p2.f[0])
    s.prepare()
    u2 = torch.zeros_like(u)
    st = s.solve(u2, W.GMRES, tol=1e-12, max_it=2000, restart=100)
    assert st.converged
    U = dhs.solve(p2)
    assert _rel(u2.cpu().numpy(), U) <= 1e-9
    with pytest.raises(W.WHError):
        s.get_state()  # the stopped solve belonged to the old layout
