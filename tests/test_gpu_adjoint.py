"""Parity of the implicit-step adjoint (differentiation form) on the GPU.

* One reverse step, teacher-forced: the oracle's rollout states go to both the
  oracle's and the library's adjoint step; dL/dx_t, dL/dv_t and dL/dE must
  agree to 1e-8 relative (FP64, PCG to 1e-12 on both sides, so only summation
  order and the iterates' rounding differ).
* A whole rollout through ``paper_2605_23088_b300.adjoint.rollout`` (autograd)
  against the oracle's own rollout + reverse pass: 1e-5 relative (the two
  forward trajectories agree only to the Newton tolerance).
* The full-size clamped beam (52x8x8 hexes, 19,968 tets, 20 steps, loss =
  squared distance of the final state to the final state of a seed-1 rollout):
  autograd gradients along random directions against Richardson-extrapolated
  central differences of the library's own rollouts, 1e-5 relative; the
  FP32-mixed forward gives the FP64 gradient to 1e-4.
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


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def N(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def yb():
    import paper_2605_23088_b300 as m
    return m


def small_beam(lift=0.0015, steps=3):
    return scenes.beam_scene(nx=4, ny=1, nz=1, length=0.2, width=0.05, lift=lift, n_steps=steps)


def test_adjoint_step_teacher_forced(yb):
    s = small_beam()
    O = oracle.OracleSystem(s, newton_tol=1e-10, pcg_tol=1e-12)
    x0, v0 = O.initial_state()
    states, rcs = O.rollout(x0, v0, 3)
    assert len(O.pairs(states[-1][0])[2]) > 0  # point-ground barrier active
    G = yb.System(s, precision=0, pcg_rel_tol=1e-12)
    r = np.random.default_rng(11)
    xbar = r.normal(size=x0.shape)
    vbar = r.normal(size=x0.shape)
    for t in range(2, -1, -1):
        xt, vt = states[t]
        xn = states[t + 1][0]
        xp_r, vp_r, Eb_r, _, rc = O.adjoint_step(xt, vt, xn, xbar, vbar, tol=1e-12)
        assert rc == 0
        Eb = G.zeros(len(s["tets"]))
        xp, vp, it, rres = G.adjoint_step(T(xt), T(vt), T(xn), T(xbar), T(vbar), Eb, tol=1e-12)
        assert it > 0
        assert rel(N(xp), xp_r) <= 1e-8, rel(N(xp), xp_r)
        assert rel(N(vp), vp_r) <= 1e-8, rel(N(vp), vp_r)
        assert rel(N(Eb), Eb_r) <= 1e-8, rel(N(Eb), Eb_r)
        xbar, vbar = xp_r, vp_r


def test_rollout_gradient_matches_oracle(yb):
    from paper_2605_23088_b300.adjoint import rollout
    s = small_beam(steps=4)
    O = oracle.OracleSystem(s, newton_tol=1e-10, pcg_tol=1e-12)
    x0, v0 = O.initial_state()
    E0 = np.array(s["tet_E"], float)
    states, rcs = O.rollout(x0, v0, 4)
    target = states[-1][0] + np.random.default_rng(5).normal(0, 1e-2, size=x0.shape)
    _, vb_r, Eb_r = O.rollout_adjoint(states, states[-1][0] - target, np.zeros_like(v0), tol=1e-12)

    G = yb.System(s, precision=0, pcg_rel_tol=1e-12, newton_tol=1e-9)
    E = T(E0).requires_grad_(True)
    v = T(v0).requires_grad_(True)
    xT, vT = rollout(G, E, T(x0), v, 4, tol=1e-12)
    loss = 0.5 * ((xT - T(target)) ** 2).sum()
    loss.backward()
    assert rel(N(E.grad), Eb_r) <= 1e-5, rel(N(E.grad), Eb_r)
    assert rel(N(v.grad), vb_r) <= 1e-5, rel(N(v.grad), vb_r)


# Newton tolerance of the full-beam rollouts (m); the line search accepts
# energy changes within the FP64 rounding of the sums, so Newton gets there.
BEAM_NEWTON_TOL = 1e-10


@pytest.fixture(scope="module")
def full_beam(yb):
    """The 19,968-tet beam; target = final state of the seed-1 beam's rollout."""
    s = scenes.beam_scene()
    s1 = scenes.beam_scene(seed=1)
    G1 = yb.System(s1, precision=0, pcg_rel_tol=1e-10, newton_tol=BEAM_NEWTON_TOL)
    x1, v1 = G1.initial_state()
    for _ in range(s1["n_steps"]):
        G1.step(x1, v1)
    assert G1.detect_pairs(x1)[2] > 0  # the beam strikes the ground
    G1.close()
    G = yb.System(s, precision=0, pcg_rel_tol=1e-10, newton_tol=BEAM_NEWTON_TOL)
    x0, v0 = G.initial_state()
    return s, G, x0, v0, x1


def _beam_loss(yb, G, s, E, x0, v0, target):
    from paper_2605_23088_b300.adjoint import rollout
    xT, _ = rollout(G, E, x0, v0, s["n_steps"], tol=1e-10)
    return 0.5 * ((xT - target) ** 2).sum()


def test_full_beam_gradient_vs_fd(yb, full_beam):
    s, G, x0, v0, target = full_beam
    E0 = T(s["tet_E"])
    E = E0.clone().requires_grad_(True)
    v = v0.clone().requires_grad_(True)
    loss = _beam_loss(yb, G, s, E, x0, v, target)
    loss.backward()
    gE, gv = E.grad.clone(), v.grad.clone()
    r = np.random.default_rng(2)
    with torch.no_grad():
        for _ in range(2):
            d = T(r.normal(size=len(s["tet_E"])))
            dv = T(r.normal(size=tuple(v0.shape)))

            def DE(eps):
                lp = _beam_loss(yb, G, s, E0 * (1 + eps * d), x0, v0, target)
                lm = _beam_loss(yb, G, s, E0 * (1 - eps * d), x0, v0, target)
                return float(lp - lm) / (2 * eps)

            def Dv(eps):
                lp = _beam_loss(yb, G, s, E0, x0, v0 + eps * dv, target)
                lm = _beam_loss(yb, G, s, E0, x0, v0 - eps * dv, target)
                return float(lp - lm) / (2 * eps)

            fdE = (4 * DE(1e-3) - DE(2e-3)) / 3
            fdv = (4 * Dv(5e-4) - Dv(1e-3)) / 3
            adE = float((gE * E0 * d).sum())
            adv = float((gv * dv).sum())
            assert abs(adE - fdE) <= 1e-5 * abs(fdE), (adE, fdE)
            assert abs(adv - fdv) <= 1e-5 * abs(fdv), (adv, fdv)


def test_full_beam_mixed_precision_gradient(yb, full_beam):
    s, G, x0, v0, target = full_beam
    E0 = T(s["tet_E"])
    E = E0.clone().requires_grad_(True)
    _beam_loss(yb, G, s, E, x0, v0, target).backward()
    g64 = N(E.grad)
    Gm = yb.System(s, precision=1, pcg_rel_tol=1e-10, newton_tol=BEAM_NEWTON_TOL)
    Em = E0.clone().requires_grad_(True)
    _beam_loss(yb, Gm, s, Em, x0, v0, target).backward()
    g32 = N(Em.grad)
    assert np.linalg.norm(g32 - g64) <= 1e-4 * np.linalg.norm(g64)


def test_checkpointing_recomputes_the_same_gradient(yb):
    """Keeping every 3rd state and recomputing the others in the backward pass
    gives the gradient of keeping them all."""
    from paper_2605_23088_b300.adjoint import rollout
    s = small_beam(steps=5)
    G = yb.System(s, precision=0, pcg_rel_tol=1e-12, newton_tol=1e-10)
    x0, v0 = G.initial_state()
    E0 = T(s["tet_E"])
    target = T(np.random.default_rng(9).normal(0, 1e-2, size=tuple(x0.shape))) + x0
    grads = []
    for every in (1, 3):
        E = E0.clone().requires_grad_(True)
        v = v0.clone().requires_grad_(True)
        xT, vT = rollout(G, E, x0, v, 5, checkpoint_every=every, tol=1e-12)
        (0.5 * ((xT - target) ** 2).sum() + 0.1 * (vT ** 2).sum()).backward()
        grads.append((N(E.grad), N(v.grad)))
    assert rel(grads[1][0], grads[0][0]) <= 1e-9
    assert rel(grads[1][1], grads[0][1]) <= 1e-9
