"""The host side of the GPU eigensolver (wh_eigs): the small dense eigenproblems of its
projected matrices, by Householder reduction to Hessenberg form and the shifted QR
algorithm, against numpy's LAPACK routine and the definition A v = w v (CPU only)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def W():
    from paper_2504_03074_gb300 import build
    build.build()
    from paper_2504_03074_gb300 import waveholtz
    return waveholtz


def _match(w, ref):
    """Every computed eigenvalue matched to a distinct reference one (greedy)."""
    ref = list(ref)
    err = 0.0
    for x in sorted(w, key=lambda z: (z.real, z.imag)):
        j = int(np.argmin([abs(x - r) for r in ref]))
        err = max(err, abs(x - ref[j]))
        ref.pop(j)
    return err


@pytest.mark.parametrize("kind", ["general", "symmetric", "hessenberg", "rotation",
                                  "repeated", "defective", "zero", "one"])
def test_dense_eig_against_lapack_and_definition(W, kind):
    rng = np.random.default_rng(3)
    m = 40
    if kind == "general":
        A = rng.standard_normal((m, m))
    elif kind == "symmetric":
        B = rng.standard_normal((m, m))
        A = B + B.T
    elif kind == "hessenberg":  # the shape Arnoldi produces: decaying subdiagonal
        A = np.triu(rng.standard_normal((m, m)), -1)
        A[np.arange(1, m), np.arange(m - 1)] *= np.logspace(0, -6, m - 1)
    elif kind == "rotation":  # complex pairs only
        A = np.zeros((m, m))
        for b in range(0, m, 2):
            t = 0.1 * (b + 1)
            A[b:b + 2, b:b + 2] = [[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]]
        Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = Qr @ A @ Qr.T
    elif kind == "repeated":  # eigenvalue 2 four times, diagonalisable
        d = np.concatenate([np.full(4, 2.0), rng.standard_normal(m - 4)])
        Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = Qr @ np.diag(d) @ Qr.T
    elif kind == "defective":  # a Jordan block: eigenvalues converge only to sqrt(eps)
        m = 6
        A = np.eye(m) * 0.5 + np.diag(np.ones(m - 1), 1)
    elif kind == "zero":
        A = np.zeros((m, m))
    else:
        m = 1
        A = np.array([[3.5]])
    w, V = W.dense_eig(A)
    ref = np.linalg.eigvals(A)
    scale = max(1.0, np.max(np.abs(ref)))
    tol = 1e-6 if kind == "defective" else 1e-10
    assert _match(w, ref) <= tol * scale
    res = np.abs(A @ V - V * w[None, :]).max()
    assert res <= 1e-10 * scale
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-12)


def test_dense_eig_rejects_bad_arguments(W):
    import ctypes as C
    L = W.lib()
    assert L.wh_dense_eig(0, None, None, None) == -1
    A = np.eye(2)
    assert L.wh_dense_eig(2, A.ctypes.data, None, None) == -1


@pytest.mark.parametrize("kind", ["general", "rotation", "near-defective"])
def test_invariant_basis_spans_an_invariant_subspace(W, kind):
    """The Schur-reordered basis of the p eigenvalues of largest modulus: orthonormal, A Q =
    Q (Q^T A Q) to rounding, and Q^T A Q carries exactly those eigenvalues (tested through
    wh_eigs' host routine on matrices with complex pairs and a nearly defective pair)."""
    rng = np.random.default_rng(5)
    m = 30
    if kind == "general":
        A = rng.standard_normal((m, m))
    elif kind == "rotation":
        A = np.zeros((m, m))
        for b in range(0, m, 2):
            t = 0.2 * (b + 1)
            r = 1.0 + 0.01 * b
            A[b:b + 2, b:b + 2] = r * np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
        Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = Qr @ A @ Qr.T
    else:  # eigenvalue 2 with a Jordan-like coupling of 1e-8, then random ones below 1
        J = np.diag(np.concatenate([[2.0, 2.0], 0.9 * rng.random(m - 2)]))
        J[0, 1] = 1.0
        J[1, 0] = 1e-16
        Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
        A = Qr @ J @ Qr.T
    import ctypes as C
    # through the binding: the basis of the 4 (or 5) largest eigenvalues
    from paper_2504_03074_gb300 import waveholtz as WH
    Q, w = WH.invariant_basis(A, 4)
    p = Q.shape[1]
    assert p in (4, 5)
    assert np.allclose(Q.T @ Q, np.eye(p), atol=1e-12)
    T = Q.T @ A @ Q
    assert np.max(np.abs(A @ Q - Q @ T)) < 1e-10 * np.max(np.abs(A))
    ref = np.linalg.eigvals(A)
    top = ref[np.argsort(-np.abs(ref))][:p]
    assert _match(np.linalg.eigvals(T), top) < 1e-6


def test_invariant_basis_keeps_a_split_nearly_real_pair_whole(W):
    """A conjugate pair whose imaginary part (1e-9) is below the pairing threshold, cut by
    the selection: the returned real basis spans the pair's whole real invariant subspace
    (one column more than asked), and A Q = Q (Q^T A Q) holds to rounding."""
    from paper_2504_03074_gb300 import waveholtz as WH
    rng = np.random.default_rng(11)
    m = 20
    J = np.diag(np.concatenate([[2.0, 1.5, 1.5], 0.5 * rng.random(m - 3)]))
    J[1, 2], J[2, 1] = 1e-9, -1e-9  # 1.5 +- 1e-9 i
    Qr, _ = np.linalg.qr(rng.standard_normal((m, m)))
    A = Qr @ J @ Qr.T
    Q, p = WH.invariant_basis(A, 2)
    assert p == 3
    T = Q.T @ A @ Q
    assert np.max(np.abs(A @ Q - Q @ T)) < 1e-12


@pytest.mark.parametrize("m,want", [(48, 48), (144, 96), (96, 48)])
def test_invariant_basis_large_selections(W, m, want):
    """Selections covering most or all of the spectrum (the eigensolver's thick restarts and
    its final k of a k-wide matrix): the basis stays orthonormal and invariant to rounding
    (an earlier version built it from a degenerate Gram eigenproblem and lost both)."""
    from paper_2504_03074_gb300 import waveholtz as WH
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, m)) / np.sqrt(m) + np.diag(np.linspace(1, 0.2, m))
    Q, p = WH.invariant_basis(A, want)
    assert want <= p <= want + 1
    assert np.max(np.abs(Q.T @ Q - np.eye(p))) < 1e-13
    T = Q.T @ A @ Q
    assert np.max(np.abs(A @ Q - Q @ T)) < 1e-12
