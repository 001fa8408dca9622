"""Oracle pins of the Baraff-Witkin cloth membrane (stretch and shear, Baraff
and Witkin 1998, the cloth of the paper's benchmarks, Sec. "Cloths on Bunny on
Cloth"; CPU).

Psi(F) = k_st/2 ((|f_u| - 1)^2 + (|f_v| - 1)^2) + k_sh/2 (f_u . f_v)^2 with
F = [f_u f_v] the deformation gradient over the triangle's rest (u, v) frame
(u along its first edge), energy = area * thickness * Psi.  Pinned by closed
forms (rest state, uniaxial stretch along u and along v, pure shear), rigid
motion invariance, central differences of the energy and of the gradient,
and the F-space projection (PSD, rank at most 6, identity on a PSD Hessian).
"""
import numpy as np
import pytest

import oracle
import scenes

KST, KSH, TH = 3.357e4, 1.00607e5, 1e-3


def rest_triangle():
    # first edge along (1, 1, 0)/sqrt2, in a tilted plane
    a = np.array([0.01, 0.02, 0.03])
    u = np.array([1.0, 1.0, 0.0]) / np.sqrt(2)
    n = np.array([0.0, 0.0, 1.0]) + 0.3 * np.array([1.0, -1.0, 0.0])
    v = np.cross(n, u)
    v /= np.linalg.norm(v)
    X = np.array([a, a + 0.02 * u, a + 0.012 * u + 0.017 * v])
    return X, u, v


def frame_map(X, u, v, M):
    """Positions after the in-plane map M (2x2, acting on (u, v) coordinates)."""
    x = X.copy()
    for k in range(3):
        d = X[k] - X[0]
        c = np.array([d @ u, d @ v])
        c2 = M @ c
        x[k] = X[0] + c2[0] * u + c2[1] * v
    return x


def area(X):
    return 0.5 * np.linalg.norm(np.cross(X[1] - X[0], X[2] - X[0]))


def test_rest_state_is_stress_free():
    X, _, _ = rest_triangle()
    E, g, H = oracle.bw_local(X, X, KST, KSH, TH, project=False)
    assert abs(E) < 1e-20 and np.abs(g).max() < 1e-14


@pytest.mark.parametrize("axis", [0, 1])
def test_uniaxial_stretch_closed_form(axis):
    X, u, v = rest_triangle()
    lam = 1.13
    M = np.eye(2)
    M[axis, axis] = lam
    E, _, _ = oracle.bw_local(frame_map(X, u, v, M), X, KST, KSH, TH)
    assert E == pytest.approx(area(X) * TH * 0.5 * KST * (lam - 1.0) ** 2, rel=1e-12)


def test_pure_shear_closed_form():
    X, u, v = rest_triangle()
    gam = 0.21
    M = np.array([[1.0, gam], [0.0, 1.0]])  # f_u = u, f_v = v + gam u
    E, _, _ = oracle.bw_local(frame_map(X, u, v, M), X, KST, KSH, TH)
    want = 0.5 * KST * (np.sqrt(1 + gam * gam) - 1.0) ** 2 + 0.5 * KSH * gam * gam
    assert E == pytest.approx(area(X) * TH * want, rel=1e-12)


def test_rigid_motion_invariance():
    X, u, v = rest_triangle()
    rng = np.random.default_rng(4)
    x = frame_map(X, u, v, np.array([[1.1, 0.07], [-0.03, 0.94]]))
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    xr = x @ q.T + rng.normal(size=3)
    E0, g0, _ = oracle.bw_local(x, X, KST, KSH, TH)
    E1, g1, _ = oracle.bw_local(xr, X, KST, KSH, TH)
    assert E1 == pytest.approx(E0, rel=1e-12)
    assert np.allclose(g1.reshape(3, 3), g0.reshape(3, 3) @ q.T, rtol=0, atol=1e-12 * np.abs(g0).max())


def test_derivatives_match_central_differences():
    X, u, v = rest_triangle()
    rng = np.random.default_rng(5)
    x = frame_map(X, u, v, np.array([[1.08, 0.1], [0.05, 0.9]])) + 1e-4 * rng.normal(size=(3, 3))
    E, g, H = oracle.bw_local(x, X, KST, KSH, TH, project=False)
    h = 1e-7
    gfd = np.zeros(9)
    Hfd = np.zeros((9, 9))
    for i in range(9):
        e = np.zeros(9)
        e[i] = h
        gfd[i] = (oracle.bw_local((x.ravel() + e).reshape(3, 3), X, KST, KSH, TH)[0]
                  - oracle.bw_local((x.ravel() - e).reshape(3, 3), X, KST, KSH, TH)[0]) / (2 * h)
        Hfd[:, i] = (oracle.bw_local((x.ravel() + e).reshape(3, 3), X, KST, KSH, TH, project=False)[1]
                     - oracle.bw_local((x.ravel() - e).reshape(3, 3), X, KST, KSH, TH, project=False)[1]) / (2 * h)
    assert np.abs(g - gfd).max() <= 1e-6 * np.abs(g).max()
    assert np.abs(H - Hfd).max() <= 1e-5 * np.abs(H).max()


def test_fspace_projection():
    X, u, v = rest_triangle()
    # a compressed state: the stretch Hessian has negative curvature (|f| < 1)
    x = frame_map(X, u, v, np.array([[0.7, 0.2], [0.0, 0.8]]))
    _, _, H = oracle.bw_local(x, X, KST, KSH, TH, project=False)
    _, _, P = oracle.bw_local(x, X, KST, KSH, TH, project=True)
    w = np.linalg.eigvalsh(H)
    wp = np.linalg.eigvalsh(P)
    assert w.min() < -1e-6 * np.abs(w).max()  # the exact Hessian is indefinite here
    assert wp.min() >= -1e-12 * np.abs(wp).max()
    assert np.sum(wp > 1e-9 * wp.max()) <= 6  # J_F^T P_F J_F: at most the 6 F-space directions
    # stretched state (|f_u|, |f_v| > 1, no shear): PSD already, projection is the identity
    xs = frame_map(X, u, v, np.diag([1.2, 1.1]))
    _, _, Hs = oracle.bw_local(xs, X, KST, KSH, TH, project=False)
    _, _, Ps = oracle.bw_local(xs, X, KST, KSH, TH, project=True)
    assert np.abs(Hs - Ps).max() <= 1e-10 * np.abs(Hs).max()


def test_bw_scene_step_descends_without_crossing():
    s = scenes.bw_cloth_scene(cloth_n=9, cloth_size=0.3, blob_h=0.02, blob_radius=0.05)
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    xt = O.xtilde(x, v)
    E0 = O.energy(x, xt)
    x1, v1, rc, st = O.step(x, v)
    assert rc == 0 and O.energy(x1, xt) <= E0
    assert O.positions(x1)[:, 1].min() > 0
