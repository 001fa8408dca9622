"""Pins of the FP64 oracle to things other than itself.

Each test checks the oracle against what the paper or the mathematics fixes:
closed forms, invariants, special cases that reduce to a library routine,
brute force on tiny inputs, finite differences of its own energies (which pins
the jets' derivatives to the energy), and the sizes the paper prints.
"""
import json
import os

import numpy as np
import pytest

import oracle
import scenes

rng = np.random.default_rng(1234)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def fd_grad(f, x, h):
    g = np.zeros_like(x)
    for i in range(x.size):
        e = np.zeros_like(x)
        e.flat[i] = h
        g.flat[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def fd_jac(f, x, h):
    cols = []
    for i in range(x.size):
        e = np.zeros_like(x)
        e.flat[i] = h
        cols.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack(cols, axis=1)


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# ----------------------------------------------------------------- EVD / PSD
@pytest.mark.parametrize("n", [3, 6, 9, 12])
def test_eig_matches_numpy(n):
    A = rng.normal(size=(n, n))
    A = A + A.T
    w, V = oracle.eig_sym(A)
    assert np.allclose(np.sort(w), np.linalg.eigvalsh(A), atol=1e-12 * np.abs(A).max())
    assert np.allclose(V @ np.diag(w) @ V.T, A, atol=1e-12 * np.abs(A).max())
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)


@pytest.mark.parametrize("n", [6, 9, 12])
def test_project_psd_properties(n):
    A = rng.normal(size=(n, n))
    A = A + A.T
    P = oracle.project_psd(A)
    # nearest PSD matrix in Frobenius norm = clamp eigenvalues (numpy eigh as the library primitive)
    w, V = np.linalg.eigh(A)
    ref = V @ np.diag(np.maximum(w, 0)) @ V.T
    assert np.allclose(P, ref, atol=1e-12 * np.abs(A).max())
    assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.abs(A).max()
    assert np.allclose(oracle.project_psd(P), P, atol=1e-12 * np.abs(A).max())  # idempotent
    B = A @ A.T
    assert np.allclose(oracle.project_psd(B), B, atol=1e-11 * np.abs(B).max())  # identity on PSD


# ----------------------------------------------------------------- SNH
def test_snh_rest_stability_and_identity_value():
    mu, lam = oracle.lame(1e5, 0.4)
    psi, P, H = oracle.snh_Fspace(np.eye(3), mu, lam)
    # rest stability: with alpha = 1 + 3 mu / (4 lam) the stress vanishes at F = I
    assert np.abs(P).max() < 1e-9 * mu
    # Psi(I) = -mu/2 ln 4 + lam/2 (3 mu / (4 lam))^2
    assert psi == pytest.approx(-0.5 * mu * np.log(4.0) + 0.5 * lam * (0.75 * mu / lam) ** 2, rel=1e-14)


def test_snh_hessian_at_identity_closed_form():
    # d2Psi/dF2 at F = I derived by hand: (3mu/4) I9 + (mu/8 + lam) f f^T - (3 mu / 4) d2(det)/dF2(I)
    mu, lam = oracle.lame(1e5, 0.4)
    _, _, H = oracle.snh_Fspace(np.eye(3), mu, lam)
    f = np.eye(3).ravel()
    HJ = np.zeros((9, 9))
    for i in range(3):
        for j in range(3):
            if i != j:
                HJ[3 * i + i, 3 * j + j] = 1.0   # d2 det / dF_ii dF_jj
                HJ[3 * i + j, 3 * j + i] = -1.0  # d2 det / dF_ij dF_ji
    ref = 0.75 * mu * np.eye(9) + (mu / 8 + lam) * np.outer(f, f) - 0.75 * mu * HJ
    assert np.allclose(H, ref, rtol=0, atol=1e-9 * lam)


def test_snh_rotation_invariance_and_fd():
    mu, lam = oracle.lame(3e4, 0.3)
    F = np.eye(3) + 0.3 * rng.normal(size=(3, 3))
    R = scenes.random_rotations(rng, 1)[0]
    p1, _, _ = oracle.snh_Fspace(F, mu, lam)
    p2, _, _ = oracle.snh_Fspace(R @ F, mu, lam)
    assert p1 == pytest.approx(p2, rel=1e-12)
    # local element: gradient / exact Hessian against central differences of its energy
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    x = X + 0.01 * rng.normal(size=(4, 3))
    e = lambda y: oracle.snh_local(y.reshape(4, 3), X, mu, lam, project=False)[0]
    gf = lambda y: oracle.snh_local(y.reshape(4, 3), X, mu, lam, project=False)[1]
    E, g, H = oracle.snh_local(x, X, mu, lam, project=False)
    assert rel(g, fd_grad(e, x.ravel(), 1e-7)) < 1e-6
    assert rel(H, fd_jac(gf, x.ravel(), 1e-7)) < 1e-6
    # projected Hessian: PSD and equal to J^T Project(d2Psi/dF2) J (never worse than exact on PSD input)
    _, _, Hp = oracle.snh_local(x, X, mu, lam, project=True)
    assert np.linalg.eigvalsh(Hp).min() >= -1e-10 * np.abs(Hp).max()
    assert np.allclose(Hp, Hp.T)


def test_snh_fspace_projection_size():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["tet_projection"]
    mu, lam = oracle.lame(1e5, 0.4)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    x = X.copy()
    x[3] = [0.2, 0.1, -0.6]  # inverted-ish, indefinite Hessian
    _, _, Hp = oracle.snh_local(x, X, mu, lam, project=True)
    # J_F^T P J_F has rank <= 9 (F-space), the 12x12 position-space matrix is rank deficient by 3
    assert Hp.shape == (g["position_space"],) * 2
    assert np.sum(np.linalg.eigvalsh(Hp) > 1e-9 * np.abs(Hp).max()) <= g["F_space"]


# ----------------------------------------------------------------- membrane / bending / ABD
def test_stvk_rest_rigid_and_fd():
    mu, lam = oracle.lame_plane_stress(1e6, 0.3)
    X = np.array([[0, 0, 0], [0.01, 0, 0], [0.003, 0, 0.009]])
    R = scenes.random_rotations(rng, 1)[0]
    E0, g0, _ = oracle.stvk_local(X @ R.T + 0.5, X, mu, lam, 1e-3)
    assert abs(E0) < 1e-20 and np.abs(g0).max() < 1e-12
    x = X + 1e-3 * rng.normal(size=(3, 3))
    e = lambda y: oracle.stvk_local(y.reshape(3, 3), X, mu, lam, 1e-3, project=False)[0]
    gf = lambda y: oracle.stvk_local(y.reshape(3, 3), X, mu, lam, 1e-3, project=False)[1]
    E, g, H = oracle.stvk_local(x, X, mu, lam, 1e-3, project=False)
    assert rel(g, fd_grad(e, x.ravel(), 1e-8)) < 1e-6
    assert rel(H, fd_jac(gf, x.ravel(), 1e-8)) < 1e-6
    # uniaxial stretch by (1+e) along the first rest edge: Green strain e + e^2/2,
    # Psi = A t (mu E00^2 + lam/2 E00^2)
    eps = 0.1
    x2 = X.copy()
    x2[:, 0] *= 1 + eps
    area = 0.5 * 0.01 * 0.009
    E00 = eps + 0.5 * eps * eps
    ref = area * 1e-3 * (mu * E00 ** 2 + 0.5 * lam * E00 ** 2)
    assert oracle.stvk_local(x2, X, mu, lam, 1e-3)[0] == pytest.approx(ref, rel=1e-12)


def test_bending_angle_closed_form_and_fd():
    X = np.array([[0, 0, 0], [1, 0, 0], [0.5, 0, 1], [0.5, 0, -1]], float)  # flat hinge in the y=0 plane
    th0, w = oracle.hinge_rest(X)
    assert abs(th0) < 1e-15
    assert w == pytest.approx(3.0 * 1.0 / (0.5 + 0.5))
    for ang in (0.3, 1.0, -0.7, 2.5):
        # rotate the wing b about the shared edge (x axis) by ang: dihedral angle magnitude = ang
        x = X.copy()
        x[3] = [0.5, np.sin(ang) * 1.0, -np.cos(ang) * 1.0]
        E, _, _ = oracle.bend_local(x, X, 2.0, project=False)
        assert E == pytest.approx(2.0 * w * ang ** 2, rel=1e-12)
    x = X + 0.05 * rng.normal(size=(4, 3))
    e = lambda y: oracle.bend_local(y.reshape(4, 3), X, 2.0, project=False)[0]
    gf = lambda y: oracle.bend_local(y.reshape(4, 3), X, 2.0, project=False)[1]
    E, g, H = oracle.bend_local(x, X, 2.0, project=False)
    assert rel(g, fd_grad(e, x.ravel(), 1e-7)) < 1e-6
    assert rel(H, fd_jac(gf, x.ravel(), 1e-7)) < 1e-5


def test_abd_orthogonality():
    R = scenes.random_rotations(rng, 1)[0]
    E, g, H = oracle.abd_ortho_local(R.T.ravel(), 6400.0)  # columns of R
    assert abs(E) < 1e-20 and np.abs(g).max() < 1e-10
    A = np.eye(3) + 0.1 * rng.normal(size=(3, 3))
    cols = A.T.ravel()
    e = lambda y: oracle.abd_ortho_local(y, 3.0, project=False)[0]
    gf = lambda y: oracle.abd_ortho_local(y, 3.0, project=False)[1]
    E, g, H = oracle.abd_ortho_local(cols, 3.0, project=False)
    # closed form: 1/2 ||A^T A - I||_F^2
    assert E == pytest.approx(1.5 * np.sum((A.T @ A - np.eye(3)) ** 2), rel=1e-12)
    assert rel(g, fd_grad(e, cols, 1e-7)) < 1e-7
    assert rel(H, fd_jac(gf, cols, 1e-7)) < 1e-6


# ----------------------------------------------------------------- distances
def _tri_brute(p, a, b, c, n=400):
    u = np.linspace(0, 1, n)
    U, V = np.meshgrid(u, u)
    m = U + V <= 1
    pts = a + U[m, None] * (b - a) + V[m, None] * (c - a)
    d = np.sum((pts - p) ** 2, axis=1)
    return d.min()


def test_point_triangle_distance_vs_sampling():
    for trial in range(40):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 1.5
        st, s = oracle.pt_classify(p, a, b, c)
        ref = _tri_brute(p, a, b, c)
        assert s <= ref + 1e-12
        assert s == pytest.approx(ref, rel=2e-2, abs=1e-4)


def test_point_triangle_special_cases():
    a, b, c = np.array([0., 0, 0]), np.array([1., 0, 0]), np.array([0., 1, 0])
    st, s = oracle.pt_classify(np.array([0.2, 0.2, 0.3]), a, b, c)
    assert st == 6 and s == pytest.approx(0.09, rel=1e-14)   # interior: plane distance
    st, s = oracle.pt_classify(np.array([-1.0, -1.0, 0.5]), a, b, c)
    assert st == 0 and s == pytest.approx(2.25, rel=1e-14)   # vertex region
    st, s = oracle.pt_classify(np.array([0.5, -1.0, 0.0]), a, b, c)
    assert st == 3 and s == pytest.approx(1.0, rel=1e-14)    # edge ab region


def test_edge_edge_distance_vs_sampling_and_closed_form():
    for trial in range(40):
        a0, a1, b0, b1 = rng.normal(size=(4, 3))
        st, s = oracle.ee_classify(a0, a1, b0, b1)
        u = np.linspace(0, 1, 500)
        P = a0 + u[:, None] * (a1 - a0)
        Q = b0 + u[:, None] * (b1 - b0)
        ref = np.min(np.sum((P[:, None, :] - Q[None, :, :]) ** 2, axis=2))
        assert s <= ref + 1e-12
        assert s == pytest.approx(ref, rel=2e-2, abs=1e-4)
    # perpendicular crossing edges at height 0.3
    st, s = oracle.ee_classify(np.array([-1., 0, 0]), np.array([1., 0, 0]), np.array([0., -1, 0.3]), np.array([0., 1, 0.3]))
    assert st == 0 and s == pytest.approx(0.09, rel=1e-14)
    # parallel edges: falls back to point-edge distances
    st, s = oracle.ee_classify(np.array([0., 0, 0]), np.array([1., 0, 0]), np.array([0.5, 0.2, 0]), np.array([1.5, 0.2, 0]))
    assert st != 0 and s == pytest.approx(0.04, rel=1e-13)


# ----------------------------------------------------------------- barrier
@pytest.mark.parametrize("form", [0, 1])
def test_barrier_closed_form_and_smoothness(form):
    sh = 1e-6
    for s in (1e-9, 1e-8, 3e-7, 9.9e-7):
        b, db, d2b = oracle.barrier_scalar(s, sh, form)
        L = np.log(s / sh)
        ref = -(s - sh) ** 2 * L if form == 0 else (s - sh) ** 2 * L * L
        assert b == pytest.approx(ref, rel=1e-13)
        h = s * 1e-5
        bp = oracle.barrier_scalar(s + h, sh, form)
        bm = oracle.barrier_scalar(s - h, sh, form)
        assert db == pytest.approx((bp[0] - bm[0]) / (2 * h), rel=1e-6)
        assert d2b == pytest.approx((bp[1] - bm[1]) / (2 * h), rel=1e-6)
    # vanishes with its first two derivatives at dhat (C2 activation)
    b, db, d2b = oracle.barrier_scalar(sh * (1 - 1e-9), sh, form)
    assert abs(b) < 1e-27 and abs(db) < 1e-20 and abs(d2b) < 1e-7
    assert oracle.barrier_scalar(sh, sh, form) == (0.0, 0.0, 0.0)
    assert oracle.barrier_scalar(1e-20, sh, form)[0] > oracle.barrier_scalar(1e-12, sh, form)[0] > 0


@pytest.mark.parametrize("kind", [0, 1])
def test_pair_local_fd_and_psd(kind):
    sh = 1e-6
    for trial in range(6):
        base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float) * 0.01
        if kind == 0:
            p = np.array([0.002 + 0.004 * rng.random(), 0.002 + 0.004 * rng.random(), 4e-4 + 3e-4 * rng.random()])
            if trial % 2:
                p[:2] = [-0.0003, -0.0002]  # vertex / edge region
            x = np.vstack([p, base])
        else:
            x = np.array([[-0.005, 0.001, 0.0], [0.005, 0.002, 0.0],
                          [0.0, -0.005, 5e-4 + 2e-4 * rng.random()], [0.001, 0.005, 6e-4]])
        E, g, H, st = oracle.pair_local(kind, x, kappa=1e4, shat=sh, project=False)
        assert E > 0
        e = lambda y: oracle.pair_local(kind, y.reshape(4, 3), kappa=1e4, shat=sh, project=False)[0]
        gf = lambda y: oracle.pair_local(kind, y.reshape(4, 3), kappa=1e4, shat=sh, project=False)[1]
        assert rel(g, fd_grad(e, x.ravel(), 1e-9)) < 1e-5
        assert rel(H, fd_jac(gf, x.ravel(), 1e-9)) < 1e-4
        _, _, Hp, _ = oracle.pair_local(kind, x, kappa=1e4, shat=sh, project=True)
        assert np.linalg.eigvalsh(Hp).min() >= -1e-10 * np.abs(Hp).max()


# ----------------------------------------------------------------- CCD
def test_accd_conservative_and_exact_approach():
    # point falling straight onto a triangle interior from distance d0 with speed |dx|:
    # true impact at t* = d0 / |dx|; ACCD must return t <= t* and stop with gap >= s*d0
    tri = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float)
    for d0, vz in ((1e-3, 4e-3), (2e-3, 1e-3), (1e-3, 0.5e-3)):
        x = np.vstack([[0.2, 0.2, d0], tri])
        dx = np.zeros((4, 3))
        dx[0, 2] = -vz
        t, it = oracle.accd(0, x, dx, gap_s=0.1, tmax=1.0)
        tstar = d0 / vz
        if tstar > 1.0:
            assert t == 1.0
        else:
            assert t <= tstar
            assert d0 - t * vz >= 0.1 * d0 * (1 - 1e-9)
            assert t >= 0.8 * tstar * 0.9
    # random trajectories: no crossing on [0, t]
    for trial in range(30):
        x = rng.normal(size=(4, 3)) * 0.01
        dx = rng.normal(size=(4, 3)) * 0.02
        for kind in (0, 1):
            t, _ = oracle.accd(kind, x, dx, gap_s=0.1)
            d0 = np.sqrt(oracle.pt_classify(*x)[1] if kind == 0 else oracle.ee_classify(*x)[1])
            for tau in np.linspace(0, t, 60):
                y = x + tau * dx
                s = oracle.pt_classify(*y)[1] if kind == 0 else oracle.ee_classify(*y)[1]
                assert np.sqrt(s) >= 0.1 * d0 * 0.999


def test_point_ground_ccd():
    pl = np.array([0, 1, 0, 0.0])
    t = oracle.pg_ccd(np.array([0, 1e-3, 0]), np.array([0, -2e-3, 0]), pl, gap_s=0.1)
    assert t == pytest.approx(0.9 * 0.5, rel=1e-14)
    assert oracle.pg_ccd(np.array([0, 1e-3, 0]), np.array([0, 2e-3, 0]), pl) == 1.0


# ----------------------------------------------------------------- system level
@pytest.fixture(scope="module")
def cubes_contact():
    s = scenes.cubes_scene(n=2)
    O = oracle.OracleSystem(s, pcg_tol=1e-10)
    x, v = O.initial_state()
    for _ in range(3):
        x, v, rc, st = O.step(x, v)
        assert rc == 0
    return s, O, x, v


def test_ccd_bound_invariant_under_common_translation(cubes_contact):
    """The distance between two primitives at any time of the step does not
    change when every vertex gets the same extra displacement, so neither does
    a time of impact.  The swept-box candidates are taken in the frame that
    moves with the mean displacement, which makes the bound (CCD over those
    candidates) invariant too; a horizontal shift also leaves the ground plane
    distances unchanged.  The grid broadphase gives the brute-force bound."""
    s, O, x, v = cubes_contact
    assert len(s["fixed"]) == 0 and len(s["body_mass"]) == 0  # every vertex is a free node
    xt = O.xtilde(x, v)
    p, _, _ = O.pcg(O.assemble(x, xt), tol=1e-10)
    c = np.broadcast_to(np.array([0.3, 0.0, -0.2]), x.shape)
    for scale in (1.0, 20.0, 200.0):
        a0 = O.ccd_bound(x, scale * p)
        assert 0.0 < a0 <= 1.0
        assert O.ccd_bound(x, scale * p, brute=True) == a0
        assert O.ccd_bound(x, scale * p - c) == pytest.approx(a0, rel=1e-9)
    assert O.ccd_bound(x, 200.0 * p) < 1.0  # the large steps are bounded


def test_ccd_bound_depends_on_relative_motion_only():
    """Two cubes 50 mm apart rise together by 100 mm while the lower one closes
    in to 3 mm of the upper one: ACCD (gap 0.1) would stop that approach, but
    the pair never comes within dhat, so it is no candidate and the step is
    not bounded.  Seen from the frame that removes the common rise the motion
    is the same, and so is the bound; boxes swept in place would overlap in the
    first view only (their union covers the common rise) and bound the step
    there."""
    s = scenes.cubes_scene(n=2)
    O = oracle.OracleSystem(s)
    x, _ = O.initial_state()
    x = x.copy()
    n = len(x) // 2  # cube 0 (lower) first, every vertex a free node
    x[n:, 1] += 0.048
    D = np.zeros_like(x)
    D[:n, 1] = 0.147
    D[n:, 1] = 0.100
    a = O.ccd_bound(x, -D)
    assert a == 1.0
    assert O.ccd_bound(x, -(D - D.mean(0))) == a
    # the same approach ending 0.5 mm apart (within dhat) is bounded
    D[:n, 1] = 0.1495
    assert O.ccd_bound(x, -D) < 1.0


def test_dof_layout_sizes():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["gradient_length"]
    s = scenes.mixed_scene(sphere_h=0.03, cloth_n=5, n_boxes=1)
    O = oracle.OracleSystem(s)
    n_free = len(s["rest_pos"]) - np.sum(s["vert_body"] >= 0) - len(s["fixed"])
    assert 3 * O.nn == g["per_free_vertex"] * n_free + g["per_affine_body"] * len(s["body_mass"])


def test_pairs_grid_equals_bruteforce(cubes_contact):
    s, O, x, v = cubes_contact
    a = O.pairs(x, brute=False)
    b = O.pairs(x, brute=True)
    assert sum(len(p) for p in a) > 0
    for pa, pb in zip(a, b):
        assert np.array_equal(pa, pb)


def test_assembly_matches_dense_fd(cubes_contact):
    s, O, x, v = cubes_contact
    xt = O.xtilde(x, v)
    g = O.assemble(x, xt, project=False)
    # gradient and exact Hessian of the total incremental potential vs central differences
    f = lambda y: O.energy(y.reshape(-1, 3), xt)
    gfd = fd_grad(f, x.ravel(), 1e-8)
    assert rel(g.ravel(), gfd) < 1e-5
    H = O.dense_hessian()
    gf = lambda y: O.assemble(y.reshape(-1, 3), xt, project=False).ravel()
    Hfd = fd_jac(gf, x.ravel(), 1e-8)
    assert rel(H, Hfd) < 1e-4
    # upper-only unique sorted sparsity
    rowptr, col, vals, diag = O.bsr(0)
    for r in range(O.nn):
        c = col[rowptr[r]:rowptr[r + 1]]
        assert np.all(c > r) and np.all(np.diff(c) > 0)


def test_pcg_matches_dense_solve(cubes_contact):
    s, O, x, v = cubes_contact
    xt = O.xtilde(x, v)
    g = O.assemble(x, xt, project=True)
    H = O.dense_hessian()
    assert np.linalg.eigvalsh(H).min() > 0
    p, it, rc = O.pcg(g, tol=1e-12)
    ref = np.linalg.solve(H, g.ravel())
    assert rc == 0 and rel(p.ravel(), ref) < 1e-8
    y = O.spmv(p)
    assert rel(y.ravel(), H @ p.ravel()) < 1e-13


def test_abd_only_block_jacobi_exact():
    # App. D: for scenes made only of affine bodies, block-Jacobi inverts H exactly
    s = scenes.mixed_scene(sphere_h=0.05, cloth_n=2, n_boxes=4)
    keep = s["vert_body"] >= 0
    # strip the soft sphere and cloth: a scene of 4 free-flying boxes
    sub = dict(s)
    idx = np.nonzero(keep)[0]
    remap = -np.ones(len(keep), int)
    remap[idx] = np.arange(len(idx))
    for k in ("rest_pos", "vel0", "vert_body"):
        sub[k] = s[k][idx]
    for k in ("tets", "tris", "hinges"):
        sub[k] = np.zeros((0, s[k].shape[1]), np.int32)
    for k in ("tet_E", "tet_nu", "tet_rho", "tri_E", "tri_nu", "tri_thick", "tri_rho", "hinge_kb"):
        sub[k] = np.zeros(0)
    st = remap[s["surf_tris"]]
    sub["surf_tris"] = st[(st >= 0).all(1)].astype(np.int32)
    sub["surf_edges"] = scenes.unique_edges(sub["surf_tris"]).astype(np.int32)
    sub["surf_verts"] = np.unique(sub["surf_tris"]).astype(np.int32)
    O = oracle.OracleSystem(sub)
    x, v = O.initial_state()
    x[O.nfree + 1::4] *= 1.05  # perturb A so the orthogonality term is active
    g = O.assemble(x, O.xtilde(x, v))
    p, it, rc = O.pcg(g, tol=1e-12)
    assert rc == 0 and it <= 1


def test_free_fall_closed_form():
    s = scenes.cubes_scene(n=2)
    s["rest_pos"] = s["rest_pos"] + np.array([0, 1.0, 0])  # far from the ground: no contact
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    v[:] = [0.3, -0.1, 0.2]
    x1, v1, rc, st = O.step(x, v)
    h = s["dt"]
    ref = x + h * v + h * h * s["gravity"]
    assert rc == 0
    assert np.abs(x1 - ref).max() < 1e-10 * s["bbox_diag"]


def test_affine_body_free_fall():
    s = scenes.mixed_scene(sphere_h=0.05, cloth_n=2, n_boxes=1)
    s["rest_pos"] = s["rest_pos"] + np.array([0, 2.0, 0])
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    x1, v1, rc, st = O.step(x, v)
    h = s["dt"]
    b0 = O.nfree
    assert np.allclose(x1[b0], x[b0] + h * h * s["gravity"], atol=1e-10)
    assert np.allclose(x1[b0 + 1:b0 + 4], np.eye(3), atol=1e-10)


def test_step_no_interpenetration_and_descent(cubes_contact):
    s, O, x, v = cubes_contact
    xt = O.xtilde(x, v)
    E0 = O.energy(x, xt)
    x1, v1, rc, st = O.step(x, v)
    assert rc == 0
    assert O.energy(x1, xt) <= E0
    P = O.positions(x1)
    assert P[:, 1].min() > 0
    # no crossing along the segment from x to x1: positions are linear in the
    # DOFs, so P(t) = P0 + t (P1 - P0); every pair found at the samples keeps a
    # positive distance (brute-force detection at each sample)
    P0 = O.positions(x)
    for t in np.linspace(0.0, 1.0, 33):
        Pt = P0 + t * (P - P0)
        xs = x + t * (x1 - x)
        assert np.allclose(O.positions(xs), Pt, rtol=0, atol=1e-15)
        pts, ees, pgs = O.pairs(xs, brute=True)
        for a, b, sub in pts:
            assert oracle.pt_classify(Pt[a], *Pt[s["surf_tris"][b]])[1] > 0
        for a, b, sub in ees:
            e, f = s["surf_edges"][a], s["surf_edges"][b]
            assert oracle.ee_classify(Pt[e[0]], Pt[e[1]], Pt[f[0]], Pt[f[1]])[1] > 0
        assert Pt[:, 1].min() > 0
    pt, ee, pg = O.pairs(x1)
    # every detected pair has a strictly positive distance
    for a, b, sub in pt:
        tv = s["surf_tris"][b]
        assert oracle.pt_classify(P[a], *P[tv])[1] > 0
    for a, b, sub in ee:
        e, f = s["surf_edges"][a], s["surf_edges"][b]
        assert oracle.ee_classify(P[e[0]], P[e[1]], P[f[0]], P[f[1]])[1] > 0


def test_pp_barrier_dof_sizes():
    g = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["pp_barrier_dof"]
    # a free cloth vertex a hair above a box corner region and two boxes touching:
    # node-space sizes of the pair contributions follow from the union Jacobians
    s = scenes.mixed_scene(sphere_h=0.05, cloth_n=2, n_boxes=2)
    O = oracle.OracleSystem(s)
    vnode, vr, vm = O.vertex_info()
    free_v = np.nonzero((s["vert_body"] < 0))[0][0]
    body_v = np.nonzero(s["vert_body"] == 0)[0][0]
    body_v2 = np.nonzero(s["vert_body"] == 1)[0][0]
    nodes = lambda v: {int(vnode[v])} if s["vert_body"][v] < 0 else {int(vnode[v]) + k for k in range(4)}
    assert 3 * len(nodes(free_v) | nodes(free_v + 1)) == g["free-free"]
    assert 3 * len(nodes(free_v) | nodes(body_v)) == g["free-abd"]
    assert 3 * len(nodes(body_v) | nodes(body_v2)) == g["abd-abd"]
    # the barrier Hessian is projected in the 6-dim position space of the two points
    p = np.array([-1.1e-4, -1.3e-4, 2.7e-4])  # nearest feature: triangle vertex a (PP)
    _, _, H, st = oracle.pair_local(0, np.array([p, [0, 0, 0], [1, 0, 0], [0, 1, 0]]), shat=1e-6, project=True)
    assert st == 0
    support = np.nonzero(np.abs(H).sum(0) > 0)[0]
    assert len(support) == g["projected"] and set(support) == set(range(6))


# ----------------------------------------------------------------- adjoint (differentiation form)
def _beam_rollout_setup(lift, T):
    s = scenes.beam_scene(nx=4, ny=1, nz=1, length=0.2, width=0.05, lift=lift, n_steps=T)
    O = oracle.OracleSystem(s, newton_tol=1e-10, pcg_tol=1e-12)
    x0, v0 = O.initial_state()
    return s, O, x0, v0


@pytest.mark.parametrize("lift", [0.0015, 0.05])  # with point-ground contact / free flight
def test_adjoint_matches_directional_fd(lift):
    """dL/dE and dL/dv0 of a 3-step rollout against central differences of the
    rollout itself (Richardson-extrapolated), along random directions: this pins
    the implicit-function adjoint to the forward steps it differentiates."""
    T = 3
    s, O, x0, v0 = _beam_rollout_setup(lift, T)
    E0 = np.array(s["tet_E"], float)
    r = np.random.default_rng(7)

    def run(E, v):
        # a step may stop on a line search that can no longer resolve the
        # energy decrease; accept that only once the Newton step is below 1e-9 m
        O.set_tet_young(E)
        states = [(x0, v)]
        for _ in range(T):
            x, vv, rc, st = O.step(*states[-1])
            assert rc == 0 or (rc == -6 and st["p_inf"] < 1e-9)
            states.append((x, vv))
        return states

    states = run(E0, v0)
    target = states[-1][0] + r.normal(0, 1e-2, size=x0.shape)
    loss = lambda st: 0.5 * np.sum((st[-1][0] - target) ** 2)
    _, vb, Eb = O.rollout_adjoint(states, states[-1][0] - target, np.zeros_like(v0))
    if lift < 0.01:
        assert len(O.pairs(states[-1][0])[2]) > 0  # the ground barrier is active
    for _ in range(2):
        d = r.normal(size=len(E0))
        dv = r.normal(size=v0.shape)

        def DE(eps):
            return (loss(run(E0 * (1 + eps * d), v0)) - loss(run(E0 * (1 - eps * d), v0))) / (2 * eps)

        def Dv(eps):
            return (loss(run(E0, v0 + eps * dv)) - loss(run(E0, v0 - eps * dv))) / (2 * eps)

        # relative steps in E are larger: the trajectory is far less sensitive
        # to E than to v0, and each forward step is exact only to ~1e-9 m
        fdE = (4 * DE(5e-3) - DE(1e-2)) / 3
        fdv = (4 * Dv(5e-4) - Dv(1e-3)) / 3
        assert abs(np.sum(Eb * E0 * d) - fdE) <= 2e-5 * abs(fdE)
        assert abs(np.sum(vb * dv) - fdv) <= 2e-5 * abs(fdv)


def test_adjoint_single_step_closed_form_free_fall():
    """No elastic or contact term active: a lone free vertex in free fall has
    x1 = x0 + h v0 + h^2 g, so dL/dv0 = h dL/dx1 and dL/dx0 = dL/dx1 exactly."""
    s = scenes.cubes_scene(n=1)
    s = dict(s)
    O = oracle.OracleSystem(s, newton_tol=1e-12, pcg_tol=1e-14)
    x0, v0 = O.initial_state()
    # make every tet modulus tiny so the elastic force vanishes to rounding
    O.set_tet_young(np.full(len(s["tets"]), 1e-12))
    x1, v1, rc, _ = O.step(x0, v0)
    assert rc == 0
    w = np.random.default_rng(3).normal(size=x0.shape)
    xp, vp, Eb, it, rc = O.adjoint_step(x0, v0, x1, w, np.zeros_like(w))
    assert rc == 0
    h = s["dt"]
    assert rel(vp, h * w) < 1e-9
    assert rel(xp, w) < 1e-9
