"""Both projection paths of the PT / EE barrier Hessians against the oracle.

The barrier kernel projects the reduced Hessian K either inside the
warp-per-pair kernel (warp-parallel Jacobi; below 8,192 pairs in FP32 and
16,384 in FP64) or in a separate pass with one pair per thread (above).
Scenes: 600 and 6000 near-contact triangle pairs (about 4k and 40k PT + EE
pairs), so that each precision takes each path once.  The assembled gradient
and BSR (projected) match the oracle within 1e-10 per entry in FP64, as in
test_gpu_parity; the FP32-mixed blocks within 2e-5 of the largest.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n_pairs", [600, 6000])
def test_projected_barrier_assembly(n_pairs):
    import paper_2605_23088_b300 as yb
    from test_gpu_parity import compare_assembly, rel

    s = scenes.near_pairs_scene(n_pairs=n_pairs)
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    pt, ee, _ = O.pairs(x)
    npairs = len(pt) + len(ee)
    assert (npairs >= 16384) == (n_pairs == 6000) and (npairs >= 8192) == (n_pairs == 6000), npairs
    G = yb.System(s)
    compare_assembly(G, O, x, v, project=True)
    # FP32-mixed: the same blocks in single precision
    Gm = yb.System(s, precision=1)
    xt = O.xtilde(x, v)
    O.assemble(x, xt, project=True)
    Gm.detect_pairs(T(x))
    Gm.eval_local(T(x), T(xt), project=True)
    for which in (0, 1):
        _, _, vals, diag = Gm.export_bsr(which)
        _, _, vals_r, diag_r = O.bsr(which)
        if len(vals_r):
            assert rel(vals, vals_r) <= 2e-5, which
