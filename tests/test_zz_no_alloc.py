"""The allocation-free PCG entry point (yasps_pcg_solve_static).

It serves callers that may not allocate device memory at solve time: they hand
in an assembled matrix and their own right-hand side and output buffers, and the
solver works entirely in a fixed array inside the library.  Here it must agree
with the regular allocating entry point (yasps_pcg_solve) on the same assembled
system, on two calls in a row (the fixed array keeps the previous call's
contents, so the second call checks that the solver clears what it must).

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def T(a, dtype=np.float64):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=dtype), device="cuda")


def test_static_pcg_matches_allocating_pcg():
    import paper_2605_23088_b300 as yb

    s = scenes.cubes_scene()
    O = oracle.OracleSystem(s, pcg_tol=1e-12)
    x, v = O.initial_state()
    for _ in range(2):  # bring the cubes into contact: dynamic (barrier) blocks exist
        x, v, rc, _ = O.step(x, v)
        assert rc == 0
    xt = O.xtilde(x, v)
    G = yb.System(s, pcg_rel_tol=1e-12)
    counts = G.detect_pairs(T(x))
    assert sum(counts) > 0
    G.eval_local(T(x), T(xt))
    g = G.export_gradient()
    tol = 1e-12
    p_ref, it_ref, rr_ref = G.pcg_solve(g, rel_tol=tol)
    # the same assembled matrix, handed over as caller-owned device arrays
    rows, cols, vals = [], [], []
    diag = None
    for which in (0, 1):
        rp, col, blk, dg = G.export_bsr(which)
        rows.append(np.repeat(np.arange(G.n_nodes), np.diff(rp)).astype(np.int32))
        cols.append(col.astype(np.int32))
        vals.append(blk)
        if which == 0:
            diag = dg
    row_d = T(np.concatenate(rows), np.int32)
    col_d = T(np.concatenate(cols), np.int32)
    val_d = T(np.concatenate(vals))
    diag_d = T(diag)
    ref = p_ref.cpu().numpy()
    scale = np.abs(ref).max()
    for call in range(2):
        p, it, rr = yb.pcg_solve_static(G.n_nodes, row_d, col_d, val_d, diag_d, g, rel_tol=tol)
        assert rr <= tol
        assert np.abs(p.cpu().numpy() - ref).max() <= 1e-8 * scale, call


def test_static_pcg_rejects_oversize():
    import paper_2605_23088_b300 as yb

    n = 65537
    z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    d = torch.zeros((n, 3, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(yb.YaspsError, match="capacity"):
        yb.pcg_solve_static(n, e, e, torch.zeros((0, 3, 3), dtype=torch.float64, device="cuda"), d, z)
