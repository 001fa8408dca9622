"""GPU parity of the cage parameterisation (Sec. "Caged Bunny") with the oracle.

Embedded surface vertices sit at p = sum_k w_k c_k over the 8 corners of their
cage cell; contact pairs of such vertices couple the union of their cage
nodes (up to 32).  Checked through the C ABI against the oracle: vertex
positions (bit-exact up to the order of the 8-term weighted sum), contact
pairs (bit-exact), the assembled gradient and BSR (projected and exact,
1e-10 per entry as in test_gpu_parity), the support of the barrier term's
Hessian (evaluated alone) for a
point-point pair whose cells share 8, 4, 2, 1 or 0 cage vertices (the
paper's compressed sizes, pinned on the oracle side), and teacher-forced
steps in FP64 and FP32-mixed (positions within 1e-6 of the bounding-box
diagonal).
"""
import json
import os

import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def caged():
    import paper_2605_23088_b300 as yb

    s = scenes.caged_blob_scene(blob_h=0.02, cage_h=0.04)
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    rng = np.random.default_rng(9)
    x = x + 2e-5 * rng.normal(size=x.shape)
    pt, ee, pg = O.pairs(x)
    assert len(pg) > 0 and len(pt) + len(ee) > 0  # ground and box contact
    return yb, s, O, x, v


def test_caged_positions_and_pairs(caged):
    yb, s, O, x, v = caged
    G = yb.System(s)
    xg, vg = G.initial_state()
    xr, vr = O.initial_state()
    assert np.array_equal(N(xg), xr) and np.array_equal(N(vg), vr)
    P = N(G.vertex_positions(T(x)))
    Pr = O.positions(x)
    assert np.abs(P - Pr).max() <= 1e-15 * max(np.abs(Pr).max(), 1.0)
    for a, b in zip(G.pairs(T(x)), O.pairs(x)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("project", [True, False])
def test_caged_assembly(caged, project):
    from test_gpu_parity import compare_assembly

    yb, s, O, x, v = caged
    G = yb.System(s, pcg_rel_tol=1e-12)
    compare_assembly(G, O, x, v, project=project)


def _dense(G, nn):
    """Dense 3nn x 3nn matrix of the exported BSR (static + dynamic + diag)."""
    H = np.zeros((3 * nn, 3 * nn))
    for which in (0, 1):
        rp, col, vals, diag = G.export_bsr(which)
        for r in range(nn):
            for k in range(rp[r], rp[r + 1]):
                c = col[k]
                H[3 * r:3 * r + 3, 3 * c:3 * c + 3] += vals[k]
                if c != r:
                    H[3 * c:3 * c + 3, 3 * r:3 * r + 3] += vals[k].T
        if which == 0:
            for r in range(nn):
                H[3 * r:3 * r + 3, 3 * r:3 * r + 3] += diag[r]
    return H


@pytest.mark.parametrize("shared", [8, 4, 2, 1, 0])
def test_caged_pair_support_and_assembly(shared):
    import paper_2605_23088_b300 as yb
    from test_gpu_parity import compare_assembly
    from test_oracle_cage import cage_pair_scene

    sizes = json.load(open(os.path.join(GOLDEN, "paper_sizes.json")))["caged_pp_compressed"]
    s, O, x, v = cage_pair_scene(shared)
    G = yb.System(s, pcg_rel_tol=1e-12)
    compare_assembly(G, O, x, v, project=False)
    # the barrier term alone: every stored entry is a barrier contribution
    xt = O.xtilde(x, v)
    G.detect_pairs(T(x))
    G.eval_local(T(x), T(xt), term_mask=yb.TERM_BARRIER, project=False)
    H = _dense(G, O.nn)
    support = np.nonzero(np.abs(H).sum(0) > 0)[0]
    assert len(support) == sizes[str(shared)], (shared, len(support))


@pytest.mark.parametrize("precision", [0, 1])
def test_caged_teacher_forced_steps(caged, precision):
    yb, s, O, x, v = caged
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
