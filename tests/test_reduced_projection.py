"""The identity behind the reduced projections of the barrier Hessians (CPU
only, numpy).

A pair's Hessian in its 3n vertex coordinates is C^T Hz C, where Hz lives in
the R = 3k reduced variables z = C y and C = coef (x) I3: point-point w = p - a
(k = 1, n = 2), point-edge (w, e) (k = 2, n = 3), point-plane and line-line
(w, e1, e2) (k = 3, n = 4).  With C C^T = L L^T the rows of Q = L^-1 C are
orthonormal and C = L Q, so the PSD projection of the 3n x 3n Hessian equals
Q^T Project(L^T Hz L) Q.  Checked here against numpy.linalg.eigh on the full
matrix for random symmetric Hz of every type, including ones that are already
PSD or entirely negative.
"""
import numpy as np
import pytest

COEF = {
    "point-point": np.array([[1, -1]], float),
    "point-edge": np.array([[1, -1, 0], [0, -1, 1]], float),
    "point-plane": np.array([[1, -1, 0, 0], [0, -1, 1, 0], [0, -1, 0, 1]], float),
    "line-line": np.array([[1, 0, -1, 0], [-1, 1, 0, 0], [0, 0, -1, 1]], float),
}


def project(A):
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    return (V * np.maximum(lam, 0.0)) @ V.T


@pytest.mark.parametrize("kind", sorted(COEF))
@pytest.mark.parametrize("shift", [0.0, 5.0, -5.0])
def test_projection_through_the_reduced_space(kind, shift):
    rng = np.random.default_rng(7)
    C = np.kron(COEF[kind], np.eye(3))  # R x 3n, rows (variable group, component)
    R = C.shape[0]
    L = np.linalg.cholesky(C @ C.T)
    Q = np.linalg.solve(L, C)
    assert np.allclose(Q @ Q.T, np.eye(R), atol=1e-14)
    assert np.allclose(L @ Q, C, atol=1e-14)
    for _ in range(20):
        B = rng.normal(size=(R, R))
        H9 = 0.5 * (B + B.T) + shift * np.eye(R)
        full = project(C.T @ H9 @ C)
        reduced = Q.T @ project(L.T @ H9 @ L) @ Q
        assert np.abs(full - reduced).max() <= 1e-12 * max(np.abs(full).max(), 1.0)


def test_factor_is_block_constant():
    """L is chol(coef coef^T) (x) I3: one 3x3 factor per distance type."""
    for coef in COEF.values():
        L3 = np.linalg.cholesky(coef @ coef.T)
        L = np.linalg.cholesky(np.kron(coef @ coef.T, np.eye(3)))
        assert np.allclose(L, np.kron(L3, np.eye(3)), atol=1e-15)
