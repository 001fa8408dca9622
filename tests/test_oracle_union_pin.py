"""Pins of the oracle's UNION map and its scatter onto affine-body nodes.

Sec. "UNION" and Sec. "Differentiation of Unioned Attributes" (App. A): an
affine-body vertex with body-relative rest offset r sits at
p = t + r1 A_1 + r2 A_2 + r3 A_3, so its Jacobian with respect to the body's
four nodes (t, A_1, A_2, A_3) is (1, r1, r2, r3) (x) I3, and a pair whose
vertices share a body adds their contributions into the same node rows
(the local merge before the scatter, Sec. "Hessian Code Generation").

These tests check the oracle against things outside it:
  * the position map against that definition written out here, with r taken
    from the scene's rest geometry and A, t random;
  * the assembled gradient and exact Hessian against central differences of
    the oracle's energy, on a scene where every free/affine pair combination
    (point-triangle both ways, edge-edge, point-ground) is active;
  * the barrier part alone (kappa = 1 minus kappa = 0) against differences of
    the barrier term, row by row on the body nodes.
A transposed weight, a wrong r, or a dropped or doubled merged node changes
the scattered rows or blocks of the bodies and fails one of them.
"""
import numpy as np
import pytest

import oracle
import scenes


def _perturbed_state(O, s, rng):
    x, v = O.initial_state()
    nb = len(s["body_mass"])
    for b in range(nb):
        n0 = O.nfree + 4 * b
        x[n0] += rng.uniform(-2e-5, 2e-5, 3)
        x[n0 + 1:n0 + 4] += rng.uniform(-1.5e-3, 1.5e-3, (3, 3))
    x[:O.nfree] += rng.uniform(-2e-5, 2e-5, (O.nfree, 3))
    return x, v


@pytest.fixture(scope="module")
def union_scene():
    s = scenes.union_contact_scene()
    O = oracle.OracleSystem(s)
    x, v = _perturbed_state(O, s, np.random.default_rng(7))
    return s, O, x, v


def test_union_position_map_definition():
    """p = t + A r for body vertices, the node itself for free ones."""
    s = scenes.union_contact_scene()
    O = oracle.OracleSystem(s)
    x0, _ = O.initial_state()
    rest = s["rest_pos"]
    vb = s["vert_body"]
    nb = len(s["body_mass"])
    # at rest every body has A = I: its vertices sit at t0 + r, so r = rest - t0
    t0 = np.array([x0[O.nfree + 4 * b] for b in range(nb)])
    for b in range(nb):
        assert np.allclose(x0[O.nfree + 4 * b + 1:O.nfree + 4 * b + 4], np.eye(3), atol=0)
    r = rest - np.where(vb[:, None] >= 0, t0[np.maximum(vb, 0)], 0.0)
    rng = np.random.default_rng(3)
    x = x0.copy()
    A = rng.normal(size=(nb, 3, 3))
    t = rng.normal(size=(nb, 3))
    for b in range(nb):
        x[O.nfree + 4 * b] = t[b]
        x[O.nfree + 4 * b + 1:O.nfree + 4 * b + 4] = A[b].T  # node k+1 holds column A_k
    x[:O.nfree] = rng.normal(size=(O.nfree, 3))
    P = O.positions(x)
    free = np.nonzero(vb < 0)[0]
    assert np.array_equal(P[free], x[:O.nfree])  # free vertices in increasing order
    for vtx in np.nonzero(vb >= 0)[0]:
        b = vb[vtx]
        want = t[b] + A[b] @ r[vtx]
        assert np.allclose(P[vtx], want, rtol=0, atol=1e-14 * (1 + np.abs(want).max()))


def test_union_scene_covers_every_combination(union_scene):
    s, O, x, _ = union_scene
    pt, ee, pg = O.pairs(x, brute=True)
    vb = s["vert_body"]
    st, se = s["surf_tris"], s["surf_edges"]
    kinds_pt = {(vb[a] >= 0, bool((vb[st[b]] >= 0).all())) for a, b, _ in pt}
    assert kinds_pt == {(False, True), (True, True), (True, False)}
    kinds_ee = {(vb[se[a][0]] >= 0, vb[se[b][0]] >= 0) for a, b, _ in ee}
    assert (True, True) in kinds_ee and ((True, False) in kinds_ee or (False, True) in kinds_ee)
    assert {vb[a] >= 0 for a, _, _ in pg} == {True, False}
    assert np.isfinite(O.energy(x, O.xtilde(x, union_scene[3])))


def _fd(f, x, h):
    out = []
    for i in range(x.size):
        e = np.zeros_like(x)
        e.flat[i] = h
        out.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack(out, axis=-1)


def test_union_gradient_matches_fd_of_energy(union_scene):
    s, O, x, v = union_scene
    xt = O.xtilde(x, v)
    g = O.assemble(x, xt, project=False).ravel()
    gfd = _fd(lambda y: np.array(O.energy(y.reshape(-1, 3), xt)), x.ravel(), 1e-8)
    scale = np.abs(gfd).max()
    err = np.abs(g - gfd)
    assert np.all(err <= 1e-6 * scale + 1e-5 * np.abs(gfd)), err.max() / scale


def test_union_barrier_rows_on_body_nodes(union_scene):
    """Barrier part only (kappa 1 minus kappa 0), each body node row on its own."""
    s, _, x, v = union_scene
    O1 = oracle.OracleSystem(s, kappa=1.0)
    O0 = oracle.OracleSystem(s, kappa=0.0)
    xt = O1.xtilde(x, v)
    gB = (O1.assemble(x, xt, project=False) - O0.assemble(x, xt, project=False)).ravel()
    fB = lambda y: np.array(O1.energy(y.reshape(-1, 3), xt, terms=True)[1][5])
    gfd = _fd(fB, x.ravel(), 1e-9)
    body = np.arange(3 * O1.nfree, 3 * O1.nn)
    assert np.abs(gfd[body]).max() > 1e-3 * np.abs(gfd).max()  # the bodies do take barrier forces
    for i in range(O1.nn):
        rows = slice(3 * i, 3 * i + 3)
        ref = gfd[rows]
        tol = 1e-7 * np.abs(gfd).max() + 1e-5 * np.abs(ref).max()
        assert np.abs(gB[rows] - ref).max() <= tol, (i, gB[rows], ref)


def test_union_exact_hessian_blocks_match_fd(union_scene):
    s, O, x, v = union_scene
    xt = O.xtilde(x, v)
    O.assemble(x, xt, project=False)
    H = O.dense_hessian()
    Hfd = _fd(lambda y: O.assemble(y.reshape(-1, 3), xt, project=False).ravel(), x.ravel(), 1e-9)
    Hfd = 0.5 * (Hfd + Hfd.T)
    floor = 1e-7 * np.abs(Hfd).max()
    n = O.nn
    for i in range(n):
        for j in range(n):
            B = H[3 * i:3 * i + 3, 3 * j:3 * j + 3]
            R = Hfd[3 * i:3 * i + 3, 3 * j:3 * j + 3]
            assert np.abs(B - R).max() <= floor + 1e-5 * np.abs(R).max(), (i, j)
