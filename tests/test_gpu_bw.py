"""GPU parity of the Baraff-Witkin cloth (cloth_model 1) with the oracle.

Scene: the cloth-on-blob scene of the paper's first benchmark shape at a small
size (a 9 x 9 sheet pinned at its corners, a coarse soft blob lowered to
0.3 mm above it, so that cloth-blob contact pairs are active).  Checked: the
assembled gradient and BSR (projected and exact) against the oracle, the
membrane term alone against a sum of the oracle's per-triangle Baraff-Witkin
functions, and teacher-forced steps in FP64 and FP32-mixed.  Tolerances as in
test_gpu_parity (1e-10 per entry; positions 1e-6 of the bounding-box
diagonal).
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def bw():
    import paper_2605_23088_b300 as yb

    s = scenes.bw_cloth_scene(cloth_n=9, cloth_size=0.3, blob_h=0.02, blob_radius=0.05)
    blob = np.unique(s["tets"])
    cloth = np.unique(s["tris"])
    P = s["rest_pos"].copy()
    P[blob, 1] -= P[blob, 1].min() - (P[cloth, 1].max() + 3e-4)
    s["rest_pos"] = P
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    assert sum(len(a) for a in O.pairs(x)[:2]) > 0  # cloth-blob pairs
    return yb, s, O, x, v


@pytest.mark.parametrize("project", [True, False])
def test_bw_assembly(bw, project):
    from test_gpu_parity import compare_assembly

    yb, s, O, x, v = bw
    G = yb.System(s, pcg_rel_tol=1e-12)
    compare_assembly(G, O, x, v, project=project)


def test_bw_membrane_term(bw):
    from test_gpu_parity import RTOL, rel

    yb, s, O, x, v = bw
    G = yb.System(s, pcg_rel_tol=1e-12)
    rng = np.random.default_rng(2)
    xs = x + 2e-3 * rng.normal(size=x.shape)  # stretch and shear every triangle
    xt = O.xtilde(xs, v)
    G.detect_pairs(T(xs))
    G.eval_local(T(xs), T(xt), term_mask=yb.TERM_MEMBRANE, project=False)
    P = O.positions(xs)
    R = s["rest_pos"]
    vnode, _, _ = O.vertex_info()
    h2 = s["dt"] ** 2
    gref = np.zeros((O.nn, 3))
    for k, e in enumerate(s["tris"]):
        _, ge, _ = oracle.bw_local(P[e], R[e], s["tri_E"][k], s["tri_shear"][k], s["tri_thick"][k], project=False)
        for a in range(3):
            if vnode[e[a]] >= 0:
                gref[vnode[e[a]]] += h2 * ge[3 * a:3 * a + 3]
    assert np.abs(gref).max() > 0
    assert rel(N(G.export_gradient()), gref) <= RTOL


@pytest.mark.parametrize("precision", [0, 1])
def test_bw_teacher_forced_steps(bw, precision):
    yb, s, O, x, v = bw
    states = [(x, v)]
    for _ in range(2):
        x, v, rc, _ = O.step(x, v)
        assert rc == 0
        states.append((x, v))
    G = yb.System(s, precision=precision, pcg_rel_tol=1e-12 if precision == 0 else 1e-10)
    for k in range(2):
        xg, vg = T(states[k][0]), T(states[k][1])
        st = G.step(xg, vg)
        assert st["rc"] == 0
        assert np.abs(N(xg) - states[k + 1][0]).max() <= 1e-6 * s["bbox_diag"]
