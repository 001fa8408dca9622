"""Oracle pins for the adaptive barrier stiffness (reading c5; CPU).

kappa is chosen at the start of each step and frozen for it: the first step
that starts with contact pairs takes the kappa that best balances the barrier
gradient against the rest of the potential, argmin_k |g_E + k g_B|, clamped
to [kappa_min, kappa_max]; later steps double it (up to kappa_max) when the
smallest pair distance is below a threshold and smaller than at the previous
step's start.  The pins check the argmin property with gradients taken from
separate systems assembled at kappa = 0 and kappa = 1, the clamps, and the
doubling rule against distances recomputed from the pair lists.  The default
lower bound (the stiffness that holds an average vertex's weight at dhat / 2)
is pinned by the static equilibrium of such a vertex and by its scaling.
"""
import numpy as np
import pytest

import oracle
import scenes


def lowered_cubes():
    s = scenes.cubes_scene(n=2)
    s["rest_pos"] = s["rest_pos"] - np.array([0.0, 1.5e-3, 0.0])  # bottom 0.5 mm above the ground (dhat 1 mm)
    return s


def gradients(s, x, v):
    O0 = oracle.OracleSystem(s, kappa=0.0)
    O1 = oracle.OracleSystem(s, kappa=1.0)
    xt = O0.xtilde(x, v)
    gE = O0.assemble(x, xt).ravel()
    gB = O1.assemble(x, xt).ravel() - gE
    return gE, gB


def min_distance(s, O, x):
    P = O.positions(x)
    pt, ee, pg = O.pairs(x)
    d2 = [np.inf]
    for a, b, _ in pt:
        d2.append(oracle.pt_classify(P[a], *P[s["surf_tris"][b]])[1])
    for a, b, _ in ee:
        e, f = s["surf_edges"][a], s["surf_edges"][b]
        d2.append(oracle.ee_classify(P[e[0]], P[e[1]], P[f[0]], P[f[1]])[1])
    for v, k, _ in pg:
        pl = s["planes"][k]
        d2.append((pl[:3] @ P[v] - pl[3]) ** 2)
    return float(np.sqrt(min(d2)))


def test_first_contact_balances_the_gradients():
    s = lowered_cubes()
    O = oracle.OracleSystem(s, pcg_tol=1e-10)
    x, v = O.initial_state()
    assert len(O.pairs(x)[2]) > 0  # contact from the start
    gE, gB = gradients(s, x, v)
    kstar = -(gE @ gB) / (gB @ gB)
    assert kstar > 0  # the barrier pushes against gravity
    f = lambda k: np.linalg.norm(gE + k * gB)
    assert f(kstar) < f(1.001 * kstar) and f(kstar) < f(0.999 * kstar)
    O.set_kappa_adaptive(True, kappa_min=1e-6, kappa_max=1e15)
    _, _, rc, st = O.step(x, v)
    assert rc == 0
    assert st["kappa"] == pytest.approx(kstar, rel=1e-9)
    assert O.kappa == st["kappa"]


def test_clamps():
    s = lowered_cubes()
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    gE, gB = gradients(s, x, v)
    kstar = -(gE @ gB) / (gB @ gB)
    O.set_kappa_adaptive(True, kappa_min=10.0 * kstar, kappa_max=100.0 * kstar)
    assert O.step(x, v)[3]["kappa"] == pytest.approx(10.0 * kstar, rel=1e-12)
    O2 = oracle.OracleSystem(s)
    O2.set_kappa_adaptive(True, kappa_min=1e-6, kappa_max=0.1 * kstar)
    assert O2.step(x, v)[3]["kappa"] == pytest.approx(0.1 * kstar, rel=1e-12)


def test_no_contact_keeps_the_lower_bound():
    s = scenes.cubes_scene(n=1)
    s["rest_pos"] = s["rest_pos"] + np.array([0.0, 0.05, 0.0])  # 5 cm above the ground
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    O.set_kappa_adaptive(True, kappa_min=123.0, kappa_max=1e9)
    x, v, rc, st = O.step(x, v)
    assert rc == 0 and st["kappa"] == 123.0


def test_doubling_rule_follows_the_smallest_distance():
    s = lowered_cubes()
    O = oracle.OracleSystem(s, pcg_tol=1e-10)
    x, v = O.initial_state()
    kmax = 1e12
    dthr = 1e-3  # every contact distance is below it
    O.set_kappa_adaptive(True, kappa_min=1e-6, kappa_max=kmax, dmin=dthr)
    kappas, dmins = [], []
    for _ in range(6):
        dmins.append(min_distance(s, O, x))
        x, v, rc, st = O.step(x, v)
        # the cubes' second step runs into the Newton iteration cap (a stall of
        # this scene without adaptive kappa too); kappa is chosen before Newton
        assert rc in (0, -5)
        kappas.append(st["kappa"])
    doubled = 0
    for t in range(1, len(kappas)):
        shrink = dmins[t] < dthr and dmins[t] < dmins[t - 1]
        expect = min(2.0 * kappas[t - 1], kmax) if shrink else kappas[t - 1]
        assert kappas[t] == pytest.approx(expect, rel=1e-15), (t, dmins, kappas)
        doubled += shrink
    assert doubled > 0  # the cubes settle onto the ground: distances shrink at first


def test_off_by_default():
    s = lowered_cubes()
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    assert O.step(x, v)[3]["kappa"] == s["kappa"]


def hanging_vertex_scene(dhat=1e-3, dt=0.01, rho=1000.0):
    """One tet at rest with three vertices fixed 5 cm up and the fourth, free,
    dhat / 2 above the ground: the free vertex's only contact is its
    point-ground pair, and every vertex carries the same lumped mass."""
    h = 0.05
    verts = np.array([[0.0, dhat / 2, 0.0], [0.0, h, 0.0], [0.02, h, 0.0], [0.0, h, 0.02]])
    tets = np.array([[0, 2, 1, 3]])
    parts = scenes._empty_parts()
    scenes._add_soft(parts, verts, tets, 1e5, 0.3, rho)
    parts["fixed"].append([1, 2, 3])
    parts["fixed_vel"].append(np.zeros((3, 3)))
    s = scenes.finalize_scene(parts, "hanging", dt, dhat, 1e4, 1, planes=[[0, 1, 0, 0]])
    return s


@pytest.mark.parametrize("form", [0, 1])
def test_derived_lower_bound_is_the_resting_equilibrium(form):
    """kappa_min by default: the stiffness at which the barrier alone holds an
    average vertex's weight at dhat / 2.  A free vertex of that mass resting at
    dhat / 2 with zero velocity is then in static equilibrium: the first step
    (contact at its start) balances the gradients to exactly kappa_min, the
    incremental potential's gradient vanishes there, and the step leaves the
    vertex where it is."""
    s = hanging_vertex_scene()
    vol = abs(np.linalg.det(np.array([[0.02, 0, 0], [0, 0, 0.02], [0, 0.05 - 5e-4, 0]]))) / 6.0
    O = oracle.OracleSystem(s, pcg_tol=1e-12, barrier_form=form)
    x, v = O.initial_state()
    assert O.nn == 1 and len(O.pairs(x)[2]) == 1
    O.set_kappa_adaptive(True)
    kmin, kmax = O.kappa_bounds()
    assert kmax == pytest.approx(1e4 * kmin, rel=1e-15)
    # with kappa = kmin the assembled gradient at rest vanishes (equilibrium)
    Ok = oracle.OracleSystem(s, kappa=kmin, barrier_form=form)
    g = Ok.assemble(x, Ok.xtilde(x, v))
    m = 1000.0 * vol / 4.0
    assert np.abs(g).max() <= 1e-9 * m * s["dt"] ** 2 * 9.81
    x1, v1, rc, st = O.step(x, v)
    assert rc == 0 and st["kappa"] == pytest.approx(kmin, rel=1e-12)
    assert np.abs(x1 - x).max() <= 1e-12 and np.abs(v1).max() <= 1e-10


def test_derived_lower_bound_scales_with_mass_and_step():
    """m h^2 |g| scaling: doubling the density doubles kappa_min, doubling dt
    quadruples it."""
    def kmin(**kw):
        O = oracle.OracleSystem(hanging_vertex_scene(**kw))
        O.set_kappa_adaptive(True)
        return O.kappa_bounds()[0]
    k0 = kmin()
    assert kmin(rho=2000.0) == pytest.approx(2.0 * k0, rel=1e-12)
    assert kmin(dt=0.02) == pytest.approx(4.0 * k0, rel=1e-12)


def test_config1_rollout_with_derived_bounds():
    """The first configuration (two cubes, kappa adaptive) runs its first steps
    with every Newton solve converged, kappa non-decreasing from the lower bound."""
    s = scenes.cubes_scene()
    O = oracle.OracleSystem(s, pcg_tol=1e-8)
    O.set_kappa_adaptive(True)
    kmin, _ = O.kappa_bounds()
    x, v = O.initial_state()
    ks = []
    for _ in range(4):
        x, v, rc, st = O.step(x, v)
        assert rc == 0
        ks.append(st["kappa"])
    assert ks[0] == kmin and all(b >= a for a, b in zip(ks, ks[1:])) and ks[-1] > kmin
    assert O.positions(x)[:, 1].min() > 0
