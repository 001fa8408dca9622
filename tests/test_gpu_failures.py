"""Failure paths of the library, exercised without faulting the GPU.

Every device-side wait of the PCG kernel is bounded; a test shrinks the bound
so that the grid barrier gives up before the other blocks arrive, and checks
that the solve reports YASPS_E_TIMEOUT and that the system still solves
afterwards.  The iteration caps, the line-search budget, the scene-count
capacity and a non-finite state are injected from the host and must come back
as their status codes.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.fixture(scope="module")
def yb():
    import paper_2605_23088_b300 as m
    return m


@pytest.fixture(scope="module")
def contact_state():
    s = scenes.cubes_scene()
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    for _ in range(2):
        x, v, rc, _ = O.step(x, v)
        assert rc == 0
    return s, x, v, O.xtilde(x, v)


def assembled(yb, contact_state, **kw):
    s, x, v, xt = contact_state
    G = yb.System(s, **kw)
    assert sum(G.detect_pairs(T(x))) > 0
    G.eval_local(T(x), T(xt))
    return G


@pytest.mark.parametrize("precision", [0, 1])
def test_pcg_wait_timeout_is_reported_and_recoverable(yb, contact_state, precision):
    G = assembled(yb, contact_state, precision=precision)
    g = G.export_gradient()
    p_ref, it_ref, _ = G.pcg_solve(g, rel_tol=1e-8)
    # a barrier count that no grid reaches, bounded to a few thousand polls
    G.set_wait_limit(4096, unmet_next=True)
    with pytest.raises(yb.YaspsError) as e:
        G.pcg_solve(g, rel_tol=1e-8)
    assert e.value.code == -7
    G.set_wait_limit(0)
    p, it, rr = G.pcg_solve(g, rel_tol=1e-8)
    assert rr <= 1e-8
    assert float((p - p_ref).abs().max()) <= 1e-6 * float(p_ref.abs().max())


def test_iteration_caps(yb, contact_state):
    s, x, v, xt = contact_state
    G = assembled(yb, contact_state, pcg_max_iter=2)
    with pytest.raises(yb.YaspsError) as e:
        G.pcg_solve(G.export_gradient(), rel_tol=1e-12)
    assert e.value.code == -5
    G = yb.System(s, newton_max_iter=1)
    st = G.step(T(x), T(v), raise_on_error=False)
    assert st["rc"] == -5 and st["newton_iters"] == 1


def test_line_search_budget(yb, contact_state):
    s, x, v, xt = contact_state
    G = yb.System(s, ls_max_iter=0)
    st = G.step(T(x), T(v), raise_on_error=False)
    assert st["rc"] == -6


def test_non_finite_state(yb, contact_state):
    s, x, v, xt = contact_state
    G = yb.System(s)
    xb = x.copy()
    xb[3, 1] = np.nan
    st = G.step(T(xb), T(v), raise_on_error=False)
    assert st["rc"] == -8


def test_scene_count_capacity(yb):
    parts = [scenes.cubes_scene(n=1) for _ in range(1025)]
    with pytest.raises(yb.YaspsError) as e:
        yb.System(scenes.concat_scenes(parts))
    assert e.value.code == -4
