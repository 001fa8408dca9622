"""Oracle pins for the adaptive barrier stiffness (reading c5; CPU).

kappa is chosen at the start of each step and frozen for it: the first step
that starts with contact pairs takes the kappa that best balances the barrier
gradient against the rest of the potential, argmin_k |g_E + k g_B|, clamped
to [kappa_min, kappa_max]; later steps double it (up to kappa_max) when the
smallest pair distance is below a threshold and smaller than at the previous
step's start.  The pins check the argmin property with gradients taken from
separate systems assembled at kappa = 0 and kappa = 1, the clamps, and the
doubling rule against distances recomputed from the pair lists.
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
