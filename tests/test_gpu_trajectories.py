"""Multi-step trajectories of the CUDA path against the FP64 oracle.

The first configuration (two stacked soft cubes falling onto the ground, 50
steps, kappa adaptive) is run by the oracle; the library then
  * steps from every oracle state (teacher forcing): the barrier stiffness it
    picks (reading c5) and the positions after each step must match, FP64 and
    FP32-mixed;
  * runs the whole rollout on its own from the initial state: its positions
    are compared with the oracle's every step and the largest deviation, with
    the step it occurs at, is reported.
The small mixed scene (soft sphere, cloth, affine boxes in contact) is stepped
teacher-forced for several steps in FP32-mixed.

Tolerance: positions within 1e-6 of the scene's bounding-box diagonal;
kappa within 1e-9 relative (the gradient-balance ratio of two FP64 dot
products summed in different orders).
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_STEPS = 50


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def yb():
    import paper_2605_23088_b300 as m
    return m


@pytest.fixture(scope="module")
def c1_rollout():
    """The oracle's 50-step rollout of the first configuration, kappa adaptive."""
    s = scenes.cubes_scene()
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    O.set_kappa_adaptive(True)
    x, v = O.initial_state()
    states, kappas = [(x, v)], []
    for _ in range(N_STEPS):
        x, v, rc, st = O.step(x, v)
        assert rc == 0
        states.append((x, v))
        kappas.append(st["kappa"])
    return s, O, states, kappas


def adaptive_system(yb, s, precision=0):
    # FP32-mixed: the FP64 refinement reaches 1e-10 within its sweeps
    G = yb.System(s, precision=precision, pcg_rel_tol=1e-12 if precision == 0 else 1e-10)
    G.set_params(kappa_adaptive=1)
    return G


def test_kappa_bounds_match_oracle(yb, c1_rollout):
    s, O, _, _ = c1_rollout
    G = adaptive_system(yb, s)
    lo, hi = O.kappa_bounds()
    _, _, _, glo, ghi = G.kappa_state()
    assert glo == pytest.approx(lo, rel=1e-12) and ghi == pytest.approx(hi, rel=1e-12)


@pytest.mark.parametrize("precision", [0, 1])
def test_c1_teacher_forced_adaptive_kappa(yb, c1_rollout, precision):
    s, O, states, kappas = c1_rollout
    G = adaptive_system(yb, s, precision)
    tol = 1e-6 * s["bbox_diag"]
    worst = 0.0
    for k in range(N_STEPS):
        x0, v0 = states[k]
        xg, vg = T(x0), T(v0)
        st = G.step(xg, vg)
        assert st["rc"] == 0, k
        assert st["kappa"] == pytest.approx(kappas[k], rel=1e-9), k
        err = np.abs(N(xg) - states[k + 1][0]).max()
        worst = max(worst, err)
        assert err <= tol, (k, err)
    assert len(set(kappas)) > 2  # kappa did adapt along the rollout
    print(f"teacher-forced c1 precision {precision}: max position error {worst:.3e} m ({worst / s['bbox_diag']:.2e} bbox)")


def test_c1_free_running_rollout(yb, c1_rollout):
    s, O, states, kappas = c1_rollout
    G = adaptive_system(yb, s)
    x, v = G.initial_state()
    errs = []
    for k in range(N_STEPS):
        st = G.step(x, v)
        assert st["rc"] == 0, k
        errs.append(np.abs(N(x) - states[k + 1][0]).max() / s["bbox_diag"])
    errs = np.array(errs)
    first = int(np.argmax(errs > 1e-6)) if (errs > 1e-6).any() else None
    print(f"free-running c1: max deviation {errs.max():.2e} bbox at step {int(errs.argmax())}, "
          f"first step above 1e-6 bbox: {first}")
    assert errs.max() <= 1e-6, (errs.max(), first)


def test_mixed_scene_fp32_mixed_teacher_forced(yb):
    from test_gpu_parity import mixed_contact_state

    s = scenes.mixed_scene(sphere_h=0.04, cloth_n=9, cloth_size=0.3, n_boxes=4)
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = mixed_contact_state(O, s)
    states = [(x, v)]
    for _ in range(4):
        x, v, rc, _ = O.step(x, v)
        assert rc == 0
        states.append((x, v))
    G = yb.System(s, precision=1, pcg_rel_tol=1e-10)
    tol = 1e-6 * s["bbox_diag"]
    for k in range(4):
        xg, vg = T(states[k][0]), T(states[k][1])
        st = G.step(xg, vg)
        assert st["rc"] == 0, k
        err = np.abs(N(xg) - states[k + 1][0]).max()
        assert err <= tol, (k, err)
