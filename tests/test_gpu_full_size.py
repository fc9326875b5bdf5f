"""Parity at the full sizes the bench times, on outputs the oracle can compute one by one:
the 256-instance uneven batch (disk-in-square, N ~ U{256..1024}, omega ~ U[10, 50], 1-4
sources) in the autotuned launch layout, FP64 and the FP32 march, checked on sampled
instances; and the sound-speed inversion geometry (512^2 + 1024x32, c with 8 bumps) in
FP64.  The oracle runs its all-cores build (the same arithmetic as the single-thread one,
bit for bit)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu
# FP32 march: 1e-4 up to 165 steps, growing about as the square of the step count beyond
# (the state is rounded every step and each rounding is carried by the wave for the rest
# of the iteration): 1e-4 (M / 165)^2


def fp32_bound(M):
    return 1e-4 * max(1.0, (M / 165.0) ** 2)
# FP64: the two sides round in different orders (folded stencil weights against
# 2 W - W_prev + dt^2 L W), and the difference grows with the step count: 1e-12 up to
# 100 steps, 1e-14 per step beyond (measured 4.2e-15 and 5.1e-15 per step at M = 495 for
# a white-noise state and for the forced iteration from rest)
FP64_STEP_BOUND = 1e-14


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    return T


@pytest.fixture(scope="module")
def W():
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz
    return waveholtz


def _rel(a, b, act):
    return np.max(np.abs(a - b)[act]) / np.max(np.abs(b)[act])


def test_full_batch_256_sampled_instances(torch, W, oracle_mod):
    """Two inputs: a white-noise state with forcing, and the forced iteration from rest
    (GMRES's right-hand side b = W_h(0, f))."""
    bp, probs = G.batch_disk_problem(256, seed=100)
    offs = np.cumsum([0] + [p.n_total for p in probs])
    v = G.random_state(bp, 4)
    got, Ms = {}, None
    for prec in (W.FP64, W.FP32):
        s = W.Solver(bp, precision=prec)
        infos = s.prepare()
        Ms = [t.M for t in infos]
        s.autotune(reps=1)  # the layout the bench times
        for name, x in (("noise", v), ("rest", np.zeros_like(v))):
            vi = torch.from_numpy(x).cuda()
            vo = torch.empty_like(vi)
            s.iterate(vi, vo, True)
            got[prec, name] = vo.cpu().numpy()
        s.close()
    assert min(Ms) < max(Ms)
    # sampled: the shortest and the longest instance, and one drawn by seed
    pick = sorted({int(np.argmin(Ms)), int(np.argmax(Ms)),
                   int(np.random.default_rng(3).integers(len(probs)))})
    for k in pick:
        p = probs[k]
        orc = oracle_mod.Oracle(p, openmp=True)
        assert orc.time.M == Ms[k]
        seg = slice(offs[k], offs[k + 1])
        act = orc.active()
        for name, x in (("noise", v[seg]), ("rest", np.zeros(p.n_total))):
            ref = orc.iterate(x, True)
            b64 = max(1e-12, FP64_STEP_BOUND * Ms[k])
            assert _rel(got[W.FP64, name][seg], ref, act) <= b64, (name, k, Ms[k])
            # FP32: the state is rounded every step at the input's scale; the filter leaves
            # little of white noise, so that case is measured against the input's scale
            scale = np.max(np.abs(x)[act]) if name == "noise" else np.max(np.abs(ref)[act])
            err = np.max(np.abs(got[W.FP32, name][seg] - ref)[act]) / scale
            assert err <= fp32_bound(Ms[k]), (name, k, Ms[k], err)


def test_full_size_inversion_geometry_iteration(torch, W, oracle_mod):
    prob = G.misfit_problem(nb=512, omega=20.0, seed=0)
    orc = oracle_mod.Oracle(prob, openmp=True)
    s = W.Solver(prob)
    ti = s.prepare()
    assert ti.M == orc.time.M
    v = G.random_state(prob, 9)
    for forcing in (True, False):
        vi = torch.from_numpy(v).cuda()
        vo = torch.empty_like(vi)
        s.iterate(vi, vo, forcing)
        got = vo.cpu().numpy()
        ref = orc.iterate(v, forcing)
        assert _rel(got, ref, orc.active()) <= 1e-12, forcing
