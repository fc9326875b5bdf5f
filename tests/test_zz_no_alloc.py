"""The allocation-free inner-product entry point (wh_multidot_noalloc), for callers that
cannot call cudaMalloc: its results must equal the context-based wh_dot on two calls in
a row (the shared scratch array keeps the previous call's contents), and sizes beyond its
fixed scratch must be refused."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import grids as G
    from paper_2504_03074_gb300 import waveholtz as W
    solver = W.Solver(G.unit_square_problem(16, 2, 3.0))  # a context for wh_dot
    return torch, W, solver


def _noalloc(torch, W, X, y, nv, n, ldx):
    out = torch.full((nv,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    st = W.lib().wh_multidot_noalloc(C.c_void_p(X.data_ptr()), ldx, nv,
                                     C.c_void_p(y.data_ptr()), n, C.c_void_p(out.data_ptr()),
                                     C.c_void_p(stream.cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_matches_wh_dot_on_two_calls_in_a_row(env):
    torch, W, solver = env
    g = torch.Generator(device="cuda").manual_seed(0)
    cases = [(7, 1_234_567), (64, 40_001)]   # second call: more vectors, fewer entries
    for nv, n in cases:
        ldx = n + 3
        X = torch.randn(nv * ldx, dtype=torch.float64, device="cuda", generator=g)
        y = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
        got = _noalloc(torch, W, X, y, nv, n, ldx)
        for k in range(nv):
            xk = X[k * ldx:k * ldx + n]
            ref = solver.dot(xk, y)
            scale = float(torch.linalg.norm(xk) * torch.linalg.norm(y))
            assert abs(got[k] - ref) <= 1e-12 * scale, (nv, n, k, got[k], ref)


def test_refuses_sizes_beyond_its_scratch(env):
    torch, W, _ = env
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(128, dtype=torch.float64, device="cuda")
    L = W.lib()
    p = lambda t: C.c_void_p(t.data_ptr())
    assert L.wh_multidot_noalloc(p(x), 8, 65, p(x), 8, p(out), None) == -1   # nv > 64
    assert L.wh_multidot_noalloc(p(x), 8, 0, p(x), 8, p(out), None) == -1
    assert L.wh_multidot_noalloc(p(x), 4, 2, p(x), 8, p(out), None) == -1    # ldx < n
    assert L.wh_multidot_noalloc(p(x), 8, 1, p(x), -1, p(out), None) == -1
    torch.cuda.synchronize()
    assert float(out.abs().sum()) == 0.0   # nothing was launched
