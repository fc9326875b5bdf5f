"""Batching form: independent Helmholtz instances (uneven grids, their own omega, time
step, Nt and alpha) advanced by the same kernel launches.  Each instance's part of a
batched WaveHoltz iteration must equal the oracle's iteration of that instance alone."""
import numpy as np
import pytest

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


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


@pytest.fixture(scope="module")
def batch():
    bp, probs = G.batch_disk_problem(5, seed=3, nb_range=(40, 72), omega_range=(3.0, 9.0),
                                     width=0.8, r_cut=0.75)
    return bp, probs


@pytest.mark.parametrize("mode", ["graph", "persistent"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_iteration_matches_each_instance(torch, W, oracle_mod, batch, mode, prec):
    bp, probs = batch
    s = W.Solver(bp, precision=W.FP32 if prec == "fp32" else W.FP64,
                 launch_mode=W.PERSISTENT if mode == "persistent" else W.GRAPH)
    infos = s.prepare()
    assert len(infos) == len(probs)
    Ms = [ti.M for ti in infos]
    assert len(set(Ms)) > 1  # uneven step counts
    tol = 1e-12 if prec == "fp64" else 1e-4
    vs = [G.random_state(p, 10 + k) for k, p in enumerate(probs)]
    v = np.concatenate(vs)
    for forcing in (True, False):
        vi = torch.from_numpy(v).cuda()
        vo = torch.empty_like(vi)
        s.iterate(vi, vo, forcing)
        got = vo.cpu().numpy()
        off = 0
        for k, p in enumerate(probs):
            orc = oracle_mod.Oracle(p)
            assert orc.time.M == infos[k].M and abs(orc.time.dt - infos[k].dt) < 1e-15
            ref = orc.iterate(vs[k], forcing)
            seg = got[off:off + p.n_total]
            act = orc.active()
            err = np.max(np.abs(seg - ref)[act]) / np.max(np.abs(ref)[act])
            assert err <= tol, (k, forcing, err)
            off += p.n_total


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-11, 1e-8), ("fp32", 1e-11, 1e-6)])
def test_batched_solve_reaches_each_direct_solution(torch, W, batch, prec, tol, bound):
    import dhs
    bp, probs = batch
    s = W.Solver(bp, precision=W.FP32 if prec == "fp32" else W.FP64)
    s.prepare()
    u = torch.zeros(bp.n_total, dtype=torch.float64, device="cuda")
    stats = s.solve_batch(u, tol=tol, max_it=3000, restart=300)
    assert all(st.converged == 1 for st in stats), [(st.residual, st.iterations) for st in stats]
    sol = u.cpu().numpy()
    off = 0
    for k, p in enumerate(probs):
        U = dhs.solve(p)
        act = np.concatenate([(g.mask != 0).ravel() for g in p.grids])
        seg = sol[off:off + p.n_total]
        err = np.max(np.abs(seg - U)[act]) / np.max(np.abs(U)[act])
        assert err <= bound, (k, err, stats[k].iterations)
        off += p.n_total
    if prec == "fp32":
        assert all(st.products_fp32 > 0 and st.products_fp64 > 0 for st in stats)
