"""Batching form: independent scenes in one system must behave exactly as each
scene alone.

The batch holds three scenes: two identical pairs of soft cubes lowered into
ground contact, which occupy the same region of space (so any pair across
scenes would be detected), and one soft two-finger gripper closing on a
deformable object.  The oracle has no batch mode: the reference for every
scene is the oracle (or the library) run on that scene alone.

Tolerances: pair sets bit-exact; per-scene PCG solutions 1e-8 relative (PCG
to 1e-12 on both sides); per-step positions within 1e-6 of each scene's
bounding-box diagonal (FP64 and FP32-mixed).
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def yb():
    import paper_2605_23088_b300 as m
    return m


def lowered_cubes():
    s = scenes.cubes_scene(n=2)
    s["rest_pos"] = s["rest_pos"] - np.array([0.0, 1.5e-3, 0.0])  # bottom 0.5 mm above the ground
    return s


@pytest.fixture(scope="module")
def batch():
    parts = [lowered_cubes(), scenes.gripper_scene(1200, np.random.default_rng(3)), lowered_cubes()]
    return parts, scenes.concat_scenes(parts, newton_tol=1e-9)


def node_ranges(parts):
    """[start, end) of each scene's nodes in the batch (no affine bodies: nodes
    are the non-fixed vertices in vertex order)."""
    out, at = [], 0
    for sc in parts:
        n = len(sc["rest_pos"]) - len(sc["fixed"])
        out.append((at, at + n))
        at += n
    return out


def test_batch_pairs_stay_inside_scenes(yb, batch):
    parts, b = batch
    G = yb.System(b)
    x, _ = G.initial_state()
    got = G.pairs(x)
    ref = [[], [], []]
    voff = toff = eoff = 0
    for sc in parts:
        O = oracle.OracleSystem(sc)
        xs, _ = O.initial_state()
        pt, ee, pg = O.pairs(xs)
        ref[0].append(pt + np.array([voff, toff, 0], np.int32))
        ref[1].append(ee + np.array([eoff, eoff, 0], np.int32))
        ref[2].append(pg + np.array([voff, 0, 0], np.int32))
        voff += len(sc["rest_pos"])
        toff += len(sc["surf_tris"])
        eoff += len(sc["surf_edges"])
    total = 0
    for a, r in zip(got, ref):
        r = np.concatenate(r, axis=0)
        assert np.array_equal(a, r)
        total += len(r)
    assert total > 0 and len(got[2]) > 0


def test_batch_pcg_is_per_scene_pcg(yb, batch):
    parts, b = batch
    G = yb.System(b, pcg_rel_tol=1e-12)
    x, v = G.initial_state()
    G.detect_pairs(x)
    G.eval_local(x, G.xtilde(x, v))
    p, it, rr = G.pcg_solve(G.export_gradient(), rel_tol=1e-12)
    assert it > 0
    for (lo, hi), sc in zip(node_ranges(parts), parts):
        Gk = yb.System(sc, pcg_rel_tol=1e-12)
        xk, vk = Gk.initial_state()
        Gk.detect_pairs(xk)
        Gk.eval_local(xk, Gk.xtilde(xk, vk))
        pk, itk, _ = Gk.pcg_solve(Gk.export_gradient(), rel_tol=1e-12)
        assert rel(N(p)[lo:hi], N(pk)) <= 1e-8, rel(N(p)[lo:hi], N(pk))


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_step_matches_each_scene_alone(yb, batch, precision):
    """FP64: two steps.  In the second, the lowered cubes' Newton iteration
    stalls (its step length halves to 2^-9 every iteration, in the oracle as
    well) and runs into the iteration cap while the gripper converges; the
    batch must reproduce both outcomes scene by scene.  FP32-mixed: the first
    step (the stall depends on the last bits of the Hessian, so the FP32
    Hessian may or may not run into it)."""
    parts, b = batch
    G = yb.System(b, precision=precision, pcg_rel_tol=1e-10, newton_tol=1e-9)
    x, v = G.initial_state()
    st = G.step(x, v)
    assert st["rc"] == 0
    newton, pcg, status = G.scene_stats()
    assert np.all(status == 0) and np.all(newton > 0) and np.all(pcg > 0)
    nsteps = 2 if precision == 0 else 1
    if nsteps == 2:
        G.step(x, v, raise_on_error=False)
        newton2, _, status2 = G.scene_stats()
    P = N(G.vertex_positions(x))
    offs = b["scene_vert_offsets"]
    for k, sc in enumerate(parts):
        O = oracle.OracleSystem(sc, pcg_tol=1e-10, newton_tol=1e-9)
        xs, vs = O.initial_state()
        xs, vs, rc, _ = O.step(xs, vs)
        assert rc == 0
        if nsteps == 2:
            xs, vs, rc, ost = O.step(xs, vs)
            assert rc == status2[k]  # the same scenes converge / hit the cap
            if rc == 0:
                assert abs(ost["newton_iters"] - newton2[k]) <= 1
        err = np.abs(P[offs[k]:offs[k + 1]] - O.positions(xs)).max()
        assert err <= 1e-6 * sc["bbox_diag"], (k, err)


def test_batch_rejects_elements_across_scenes(yb, batch):
    parts, b = batch
    bad = dict(b)
    tets = b["tets"].copy()
    tets[0, 0] = b["scene_vert_offsets"][1]  # first tet of scene 0 borrows a vertex of scene 1
    bad["tets"] = tets
    with pytest.raises(yb.YaspsError):
        yb.System(bad)


@pytest.mark.parametrize("which", ["single", "batch"])
@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_launch_configurations_agree_and_autotune(yb, batch, which, precision):
    """Every PCG launch configuration the autotuner chooses from solves the same
    system to the same answer; the autotuner returns one of them."""
    parts, b = batch
    G = yb.System(b if which == "batch" else parts[1], precision=precision, pcg_rel_tol=1e-10)
    x, v = G.initial_state()
    G.detect_pairs(x)
    G.eval_local(x, G.xtilde(x, v))
    g = G.export_gradient()
    sols = []
    for var in range(yb.PCG_VARIANTS):
        G.set_pcg_variant(var)
        p, it, rr = G.pcg_solve(g, rel_tol=1e-10)
        sols.append(N(p))
    for p in sols[1:]:
        assert rel(p, sols[0]) <= (1e-8 if precision == 0 else 1e-5)
    var, us = G.autotune_pcg(20)
    assert 0 <= var < yb.PCG_VARIANTS and np.all(us > 0) and us[var] == us.min()
