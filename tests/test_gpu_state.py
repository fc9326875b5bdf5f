"""Checkpoint and resume of a solve (wh_get_state / wh_set_state): a solve stopped at its
product budget, saved, loaded into a fresh context and continued equals the uninterrupted
solve bit for bit (GMRES stopped inside a restart cycle, the FP32-then-FP64 form, the
fixed-point iteration, deflated GMRES)."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    assert torch.cuda.is_available()
    return torch, W


def _disk():
    return G.disk_problem(nb=128, nth=256, nr=16, order=4, omega=10.0, seed=2)


def _solve(torch, s, n, method, max_it, restart=40):
    u = torch.zeros(n, dtype=torch.float64, device="cuda")
    st = s.solve(u, method, tol=1e-14, max_it=max_it, restart=restart)
    torch.cuda.synchronize()
    return u.cpu().numpy(), st


@pytest.mark.parametrize("case", ["gmres-fp64", "gmres-fp32", "fpi", "gmres-deflated"])
def test_interrupted_and_resumed_equals_uninterrupted(env, case):
    torch, W = env
    prob = _disk()
    n = prob.n_total
    prec = W.FP32 if case == "gmres-fp32" else W.FP64
    method = W.FPI if case == "fpi" else W.GMRES
    total, first = (20, 7) if case == "fpi" else (150, 77)  # 77: inside the second cycle

    def solver():
        s = W.Solver(prob, precision=prec)
        s.prepare()
        if case == "gmres-deflated":
            Q, T, beta, lam2, st = s.eigs(4, tol=1e-10, max_products=2000, passes=1)
            s.set_deflation_basis(Q, T)
            s._keep = Q
        return s

    a = solver()
    ref, st_ref = _solve(torch, a, n, method, total)
    assert st_ref.status == "WH_ERR_NOT_CONVERGED" and st_ref.iterations >= total
    b = solver()
    part, st1 = _solve(torch, b, n, method, first)
    assert st1.status == "WH_ERR_NOT_CONVERGED"
    state = b.get_state()
    c = solver()
    c.set_state(state)
    got, st2 = _solve(torch, c, n, method, total)
    assert np.array_equal(got, ref), np.max(np.abs(got - ref))
    assert st2.iterations == st_ref.iterations
    assert (st2.products_fp32, st2.products_fp64) == (st_ref.products_fp32, st_ref.products_fp64)


def test_state_errors(env):
    torch, W = env
    prob = _disk()
    s = W.Solver(prob)
    s.prepare()
    with pytest.raises(W.WHError) as e:
        s.get_state()  # no stopped solve
    assert e.value.status == -3
    _solve(torch, s, prob.n_total, W.GMRES, 30)
    state = s.get_state()
    other = W.Solver(G.disk_problem(nb=64, nth=128, nr=12, order=4, omega=5.0, width=0.8, r_cut=0.75))
    other.prepare()
    with pytest.raises(W.WHError) as e:
        other.set_state(state)  # another problem
    assert e.value.status == -3
    with pytest.raises(W.WHError) as e:
        s.set_state(b"garbage" * 40)
    assert e.value.status == -1
    s.set_state(state)
    with pytest.raises(W.WHError) as e:  # a resumed GMRES with another restart length
        s.solve(torch.zeros(prob.n_total, dtype=torch.float64, device="cuda"), W.GMRES,
                tol=1e-14, max_it=60, restart=20)
    assert e.value.status == -3
