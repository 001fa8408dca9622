"""Full-size parity on sampled outputs.

The 64-tori pile (1,084,416 tets) after the benchmark's 14-step pre-roll, in
the benchmark's FP32-mixed configuration and in FP64, and the full mixed scene
(20k-tet sphere, 101x101 cloth, 16 affine boxes) after it has fallen into
contact.  The oracle cannot assemble these whole, so the checks sample outputs
it can compute one by one:

* every sampled pair the library reports is a real pair (oracle distance below
  dhat^2, same sub-type), and for sampled surface vertices / edges the pairs
  the library reports are exactly the pairs brute force over all primitives
  finds (bit-exact sets);
* sampled gradient rows and diagonal Hessian blocks equal the sum of the
  oracle's local contributions (inertia, elements, barrier pairs) at those
  nodes: 1e-10 of the contributions' magnitude in FP64, gradients also in the
  mixed form (they stay FP64), diagonal blocks 2e-5 in the mixed form;
* the PCG solution satisfies ||g - H p|| <= tol ||g|| (preconditioned norm
  checked in FP64 through the library's FP64 SpMV) at the full size.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

rng = np.random.default_rng(17)


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def yb():
    import paper_2605_23088_b300 as m
    return m


def prerolled(yb, scene, steps, precision=1):
    G = yb.System(scene, precision=precision, pcg_rel_tol=1e-4, newton_tol=1e-2 * scene["dt"])
    x, v = G.initial_state()
    for _ in range(steps):
        G.step(x, v, raise_on_error=False)
    return G, x, v


@pytest.fixture(scope="module")
def tori(yb):
    s = scenes.tori_scene()
    G, x, v = prerolled(yb, s, 14)
    O = oracle.OracleSystem(s)
    return s, O, G, x, v


@pytest.fixture(scope="module")
def mixed_full(yb):
    s = scenes.mixed_scene()
    G, x, v = prerolled(yb, s, 18, precision=0)
    O = oracle.OracleSystem(s)
    return s, O, G, x, v


# ---------------------------------------------------------------- pairs
def check_pairs(s, G, x, n_sample=1500):
    P = N(G.vertex_positions(x))
    dh = s["dhat"]
    sh = dh * dh
    pt, ee, pg = G.pairs(x)
    st, se = s["surf_tris"], s["surf_edges"]
    # every sampled reported pair is a pair
    for a, b, sub in pt[rng.choice(len(pt), min(n_sample, len(pt)), replace=False)] if len(pt) else []:
        r_sub, sd = oracle.pt_classify(P[a], *P[st[b]])
        assert sd < sh and r_sub == sub
    for a, b, sub in ee[rng.choice(len(ee), min(n_sample, len(ee)), replace=False)] if len(ee) else []:
        r_sub, sd = oracle.ee_classify(P[se[a, 0]], P[se[a, 1]], P[se[b, 0]], P[se[b, 1]])
        assert sd < sh and r_sub == sub
    # completeness around sampled surface vertices (PT) and surface edges (EE)
    body = s["vert_body"]
    tlo, thi = P[st].min(1), P[st].max(1)
    sv = s["surf_verts"]
    pt_by_v = {}
    for a, b, sub in pt:
        pt_by_v.setdefault(int(a), set()).add((int(b), int(sub)))
    hot = np.unique(pt[:, 0]) if len(pt) else np.zeros(0, int)
    cand_v = np.concatenate([rng.choice(sv, min(300, len(sv)), replace=False), hot[:300]])
    for v in cand_v:
        p = P[v]
        near = np.nonzero(np.all((tlo - dh <= p) & (p <= thi + dh), axis=1))[0]
        want = set()
        for b in near:
            tri = st[b]
            if v in tri or (body[v] >= 0 and body[v] == body[tri[0]]):
                continue
            sub, sd = oracle.pt_classify(p, *P[tri])
            if sd < sh:
                want.add((int(b), int(sub)))
        assert pt_by_v.get(int(v), set()) == want, v
    elo, ehi = P[se].min(1), P[se].max(1)
    ee_by_e = {}
    for a, b, sub in ee:
        ee_by_e.setdefault(int(a), set()).add((int(b), int(sub)))
        ee_by_e.setdefault(int(b), set()).add((int(a), int(sub)))
    hot_e = np.unique(ee[:, :2]) if len(ee) else np.zeros(0, int)
    cand_e = np.concatenate([rng.choice(len(se), min(300, len(se)), replace=False), hot_e[:300]])
    for i in cand_e:
        e = se[i]
        near = np.nonzero(np.all((elo - dh <= ehi[i]) & (elo[i] <= ehi + dh), axis=1))[0]
        want = set()
        for j in near:
            f = se[j]
            if j == i or len({*e, *f}) < 4 or (body[e[0]] >= 0 and body[e[0]] == body[f[0]]):
                continue
            # pairs are stored (smaller edge, larger edge); sub-types depend on that order
            lo_e, hi_e = (e, f) if i < j else (f, e)
            sub, sd = oracle.ee_classify(P[lo_e[0]], P[lo_e[1]], P[hi_e[0]], P[hi_e[1]])
            if sd < sh:
                want.add((int(j), int(sub)))
        assert ee_by_e.get(int(i), set()) == want, i
    return len(pt), len(ee), len(pg)


def test_tori_pairs_sampled(tori):
    s, O, G, x, v = tori
    npt, nee, npg = check_pairs(s, G, x)
    assert npt + nee > 0 and npg > 0


def test_mixed_full_pairs_sampled(mixed_full):
    s, O, G, x, v = mixed_full
    npt, nee, npg = check_pairs(s, G, x)
    assert npt + nee > 0


# ---------------------------------------------------------------- sampled rows
def local_rows(s, O, P, xs, xtil, pairs, nodes, vnode, vmass, project=True):
    """Gradient rows and diagonal blocks of the free nodes `nodes`, summed from
    the oracle's local contributions; also the magnitude of the contributions."""
    h2 = s["dt"] ** 2
    dh2 = s["dhat"] ** 2
    kappa = s["kappa"]
    want = set(int(n) for n in nodes)
    node_of = {int(n): None for n in nodes}
    g = {n: np.zeros(3) for n in want}
    H = {n: np.zeros((3, 3)) for n in want}
    mag = {n: 0.0 for n in want}
    vert_of_node = {}
    for vv in np.nonzero(np.isin(vnode, list(want)) & (s["vert_body"] < 0))[0]:
        vert_of_node[int(vnode[vv])] = int(vv)
    # inertia
    for n in want:
        vv = vert_of_node[n]
        m = vmass[vv]
        g[n] += m * (xs[n] - xtil[n])
        H[n] += m * np.eye(3)
        mag[n] = max(mag[n], np.abs(m * (xs[n] - xtil[n])).max(), m)
    verts = set(vert_of_node.values())

    def add(ids, gl, Hl, scale):
        for a, vv in enumerate(ids):
            if vv in verts:
                n = int(vnode[vv])
                g[n] += scale * gl[3 * a:3 * a + 3]
                H[n] += scale * Hl[3 * a:3 * a + 3, 3 * a:3 * a + 3]
                mag[n] = max(mag[n], np.abs(scale * gl[3 * a:3 * a + 3]).max(),
                             np.abs(scale * Hl[3 * a:3 * a + 3, 3 * a:3 * a + 3]).max())

    R = s["rest_pos"]
    for e in np.nonzero(np.isin(s["tets"], list(verts)).any(1))[0]:
        ids = s["tets"][e]
        mu, lam = oracle.lame(s["tet_E"][e], s["tet_nu"][e])
        _, gl, Hl = oracle.snh_local(P[ids], R[ids], mu, lam, project=project)
        add(ids, gl, Hl, h2)
    for e in np.nonzero(np.isin(s["tris"], list(verts)).any(1))[0] if len(s["tris"]) else []:
        ids = s["tris"][e]
        mu, lam = oracle.lame_plane_stress(s["tri_E"][e], s["tri_nu"][e])
        _, gl, Hl = oracle.stvk_local(P[ids], R[ids], mu, lam, s["tri_thick"][e], project=project)
        add(ids, gl, Hl, h2)
    for e in np.nonzero(np.isin(s["hinges"], list(verts)).any(1))[0] if len(s["hinges"]) else []:
        ids = s["hinges"][e]
        _, gl, Hl = oracle.bend_local(P[ids], R[ids], s["hinge_kb"][e], project=project)
        add(ids, gl, Hl, h2)
    pt, ee, pg = pairs
    st, se = s["surf_tris"], s["surf_edges"]
    for a, b, _ in pt:
        ids = [int(a), *map(int, st[b])]
        if verts.isdisjoint(ids):
            continue
        _, gl, Hl, _ = oracle.pair_local(0, P[ids], kappa=kappa, shat=dh2, project=project)
        add(ids, gl, Hl, 1.0)
    for a, b, _ in ee:
        ids = [*map(int, se[a]), *map(int, se[b])]
        if verts.isdisjoint(ids):
            continue
        _, gl, Hl, _ = oracle.pair_local(1, P[ids], kappa=kappa, shat=dh2, project=project)
        add(ids, gl, Hl, 1.0)
    for a, k, _ in pg:
        if int(a) not in verts:
            continue
        _, gl, Hl, _ = oracle.pair_local(2, P[[int(a)]], plane=s["planes"][k], kappa=kappa, shat=dh2, project=project)
        add([int(a)], gl, Hl, 1.0)
    return g, H, mag


def check_rows(s, O, G, x, v, tol_g, tol_h, n_nodes=120):
    xt = G.xtilde(x, v)
    pairs = G.pairs(x)
    G.eval_local(x, xt)
    gg = N(G.export_gradient())
    diag = G.export_bsr(0)[3]
    vnode, vr, vmass = O.vertex_info()
    P = N(G.vertex_positions(x))
    free_nodes = vnode[(vnode >= 0) & (s["vert_body"] < 0)]
    # half random, half where contact acts
    contact_v = np.unique(np.concatenate([pairs[0][:, 0], pairs[2][:, 0]])) if len(pairs[0]) + len(pairs[2]) else []
    contact_nodes = [vnode[c] for c in contact_v if vnode[c] >= 0 and s["vert_body"][c] < 0]
    nodes = np.unique(np.concatenate([rng.choice(free_nodes, n_nodes // 2, replace=False),
                                      np.asarray(contact_nodes[:n_nodes // 2], dtype=free_nodes.dtype)]))
    g_ref, H_ref, mag = local_rows(s, O, P, N(x), N(xt), pairs, nodes, vnode, vmass)
    for n in nodes:
        n = int(n)
        assert np.abs(gg[n] - g_ref[n]).max() <= tol_g * mag[n], (n, gg[n], g_ref[n])
        assert np.abs(diag[n] - H_ref[n]).max() <= tol_h * mag[n], (n, diag[n], H_ref[n])


def test_tori_rows_sampled_mixed_precision(tori):
    s, O, G, x, v = tori
    check_rows(s, O, G, x, v, tol_g=1e-10, tol_h=2e-5)


def test_tori_rows_sampled_fp64(yb, tori):
    s, O, G, x, v = tori
    G64 = yb.System(s, precision=0)
    check_rows(s, O, G64, x, v, tol_g=1e-10, tol_h=1e-10)
    G64.close()


def test_mixed_full_rows_sampled(mixed_full):
    s, O, G, x, v = mixed_full
    check_rows(s, O, G, x, v, tol_g=1e-10, tol_h=1e-10)


# ---------------------------------------------------------------- PCG property
@pytest.mark.parametrize("precision", [0, 1])
def test_tori_pcg_residual(yb, tori, precision):
    s, O, G, x, v = tori
    Gp = G if precision == 1 else yb.System(s, precision=0)
    xt = Gp.xtilde(x, v)
    Gp.detect_pairs(x)
    Gp.eval_local(x, xt)
    g = Gp.export_gradient()
    p, it, rr = Gp.pcg_solve(g, rel_tol=1e-8)
    r = g - Gp.spmv(p)  # FP64 SpMV of the stored (FP32 or FP64) Hessian
    # the stopping test is in the M^-1 norm; in the 2-norm allow the block-Jacobi
    # conditioning (1e3) on top of the tolerance
    assert float(torch.linalg.norm(r) / torch.linalg.norm(g)) <= 1e-5
    assert it > 0 and rr <= 1e-8
