"""The single-precision prefilters of the contact kernels change no result.

The candidate and detection kernels reject far pairs first with conservative
FP32 bounds (box and separating-axis distance bounds, the relative-motion
bound of the CCD) on single-precision copies of the positions; a pair they
reject must be one the FP64 tests reject too.  Stress input: 2000 pairs of
small triangles placed up to 1 m from the origin (where FP32 rounds the
most), their point-triangle and edge-edge distances spread from 0.5 to 2.5
dhat, with random relative velocities (a 150-pair copy with kappa 1e2 for
the step, so that the oracle converges in seconds).  Checked against the oracle:
contact pairs bit-exact, barrier energy (1e-12 relative), the CCD bound for
displacements of several sizes (1e-14), and a teacher-forced step (its
swept candidates, line-search energies and detection all go through the
prefilters; positions within 1e-6 of the bounding-box diagonal).
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
def near():
    import paper_2605_23088_b300 as yb

    s = scenes.near_pairs_scene(n_pairs=2000)
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    return yb, s, O, x, v


def test_pairs_and_energy(near):
    yb, s, O, x, v = near
    G = yb.System(s)
    ref = O.pairs(x)
    assert len(ref[0]) > 1000 and len(ref[1]) > 1000
    for a, b in zip(G.pairs(T(x)), ref):
        assert np.array_equal(a, b)
    xt = O.xtilde(x, v)
    E, t = G.energy(T(x), T(xt), terms=True)
    Er, tr = O.energy(x, xt, terms=True)
    assert E == pytest.approx(Er, rel=1e-12)
    assert t[-1] == pytest.approx(tr[-1], rel=1e-12)


def test_ccd_bound(near):
    yb, s, O, x, v = near
    G = yb.System(s)
    rng = np.random.default_rng(4)
    p = rng.normal(size=x.shape) * s["dhat"]
    for scale in (0.3, 1.0, 3.0):
        a = G.ccd_bound(T(x), T(scale * p))
        ar = O.ccd_bound(x, scale * p)
        assert a == pytest.approx(ar, rel=1e-14, abs=0.0)
        assert ar < 1.0 or scale < 1.0


@pytest.fixture(scope="module")
def near_step():
    # a smaller, softer copy for a converged step (the oracle's PCG at 1e-12)
    s = scenes.near_pairs_scene(n_pairs=150, kappa=1e2)
    tol = 1e-2 * s["dt"]
    O = oracle.OracleSystem(s, pcg_tol=1e-12, newton_tol=tol)
    x, v = O.initial_state()
    x1, v1, rc, _ = O.step(x, v)
    assert rc == 0
    return s, tol, x, v, x1


def test_teacher_forced_step(near_step):
    # FP64: the prefilters see the same FP64 positions in both forms, and the
    # milligram triangles against a stiff barrier are beyond an FP32 inner solve
    import paper_2605_23088_b300 as yb

    s, tol, x, v, x1 = near_step
    G = yb.System(s, precision=0, newton_tol=tol, pcg_rel_tol=1e-12)
    xg, vg = T(x), T(v)
    st = G.step(xg, vg)
    assert st["rc"] == 0
    assert np.abs(N(xg) - x1).max() <= 1e-6 * s["bbox_diag"]
