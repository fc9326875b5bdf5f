"""Deflation (Algorithm 3) through the C ABI against the oracle's Algorithm 3."""
import numpy as np
import pytest
import scipy.fft as sfft

from paper_2504_03074_gb300 import grids as G

pytestmark = pytest.mark.gpu


def _modes(prob, ts, K):
    """The K DST-I modes of the unit square with |beta_d| nearest 1, orthonormal in the
    compact inner product, and their eigenvalues lambda_h^2."""
    from oracle.oracle import beta_d_sum, lambda_tilde
    n = prob.grids[0].n[0]
    h = prob.grids[0].h[0]
    m = np.arange(1, n - 1)
    sx = np.sin(m * np.pi * h / 2) ** 2
    lam2 = (4 / h ** 2) * (sx[None, :] + sx[:, None])
    bd = beta_d_sum(lambda_tilde(np.sqrt(lam2).ravel(), ts.dt), ts.omega_e, ts.dt, ts.Nt,
                    ts.alpha).reshape(lam2.shape)
    pick = np.argsort(-np.abs(bd).ravel())[:K]
    Phi, l2 = [], []
    for q in pick:
        i, j = np.unravel_index(q, bd.shape)
        z = np.zeros((n - 2, n - 2))
        z[i, j] = 1.0
        phi = np.zeros((n, n))
        phi[1:-1, 1:-1] = sfft.idstn(z, type=1, norm="ortho")
        Phi.append(phi.ravel())
        l2.append(lam2[i, j])
    return np.array(Phi), np.array(l2)


@pytest.mark.parametrize("K", [1, 8])
def test_deflated_fpi_matches_oracle(K):
    """12 deflated fixed-point iterations from 0 on the 64^2 unit square (the library's FPI
    with a deflation set of K DST modes, then the inflation) equal the oracle's Algorithm 3
    within 1e-12 relative max-norm."""
    import torch
    from oracle import deflation as D
    from oracle import oracle as O
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz as W
    prob = G.unit_square_problem(64, 2, 10.0, seed=0)
    orc = O.Oracle(prob)
    Phi, l2 = _modes(prob, orc.time, K)
    ref, hist, res = D.deflated_fpi(orc, Phi, l2, prob.f[0].ravel(), prob.omega, 12)
    s = W.Solver(prob)
    s.prepare()
    phi_d = torch.from_numpy(Phi).cuda().contiguous()
    s.set_deflation(phi_d, l2)
    u = torch.zeros(prob.n_total, dtype=torch.float64, device="cuda")
    st = s.solve(u, W.FPI, tol=1e-300, max_it=12)
    assert st.status == "WH_ERR_NOT_CONVERGED" and st.iterations == 12
    got = u.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # residuals ||v_{k+1} - v_k|| / ||v_{k+1}|| fall to 2e-4 here, so rounding differences of
    # ~1e-14 in the iterates show up at ~1e-10 in them
    assert np.allclose(st.history[:12], [r / max(np.linalg.norm(hist[k + 1]), 1e-300)
                                          for k, r in enumerate(res)], rtol=1e-8)
    s.set_deflation(None)
