"""The allocation-free PCG entry point (yasps_pcg_solve_static).

It serves callers that may not allocate device memory at solve time: they hand
in an assembled matrix and their own right-hand side and output buffers, and the
solver works entirely in a fixed array inside the library.  Here it must agree
with the regular allocating entry point (yasps_pcg_solve) on the same assembled
system, on two calls in a row (the fixed array keeps the previous call's
contents, so the second call checks that the solver clears what it must).

The checks cover one thread block (two small cubes) and many blocks (two
12x12x12-hex cubes, 4394 nodes, not a multiple of the 256-thread block), a
device-memory check around the call, and the failure statuses (non-finite
right-hand side, an indefinite diagonal block, an out-of-range block index,
an aliased output, the iteration cap).

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


def _exported(G):
    rows, cols, vals = [], [], []
    diag = None
    for which in (0, 1):
        rp, col, blk, dg = G.export_bsr(which)
        rows.append(np.repeat(np.arange(G.n_nodes), np.diff(rp)).astype(np.int32))
        cols.append(col.astype(np.int32))
        vals.append(blk)
        if which == 0:
            diag = dg
    return np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), diag


@pytest.fixture(scope="module")
def multiblock():
    """Two 12^3-hex cubes brought into contact by the library's own steps."""
    import paper_2605_23088_b300 as yb

    s = scenes.cubes_scene(n=12)
    G = yb.System(s, pcg_rel_tol=1e-8, newton_tol=1e-2 * s["dt"])
    x, v = G.initial_state()
    for _ in range(3):
        G.step(x, v)
    xt = G.xtilde(x, v)
    assert sum(G.detect_pairs(x)) > 0
    G.eval_local(x, xt)
    g = G.export_gradient()
    row, col, vals, diag = _exported(G)
    return G, g, row, col, vals, diag


def test_static_pcg_many_blocks_matches_allocating_pcg(multiblock):
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl

    import paper_2605_23088_b300 as yb

    G, g, row, col, vals, diag = multiblock
    n = G.n_nodes
    assert n > 4 * 256 and n % 256 != 0
    tol = 1e-11
    p_ref, _, _ = G.pcg_solve(g, rel_tol=tol)
    ref = p_ref.cpu().numpy()
    # an independent reference: a sparse direct solve of the same matrix
    def blocks(r, c, b):  # COO of 3x3 blocks at (r, c); repeated coordinates are summed
        ii = (3 * r[:, None, None] + np.arange(3)[None, :, None]) + 0 * b.astype(np.int64)
        jj = (3 * c[:, None, None] + np.arange(3)[None, None, :]) + 0 * b.astype(np.int64)
        return sp.coo_matrix((b.ravel(), (ii.ravel(), jj.ravel())), shape=(3 * n, 3 * n)).tocsr()

    U = blocks(row.astype(np.int64), col.astype(np.int64), vals)
    H = U + U.T + blocks(np.arange(n), np.arange(n), diag)
    direct = spl.spsolve(H.tocsc(), g.cpu().numpy().ravel()).reshape(-1, 3)
    scale = np.abs(direct).max()
    assert np.abs(ref - direct).max() <= 1e-6 * scale
    row_d, col_d, val_d, diag_d = T(row, np.int32), T(col, np.int32), T(vals), T(diag)
    out = torch.empty_like(g)
    yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, g, rel_tol=tol, out=out)  # first call on the device
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    allocs0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for call in range(2):
        out.fill_(np.nan)
        p, it, rr = yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, g, rel_tol=tol, out=out)
        assert p.data_ptr() == out.data_ptr() and rr <= tol and it > 8
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-8 * scale, call
        assert np.abs(got - direct).max() <= 1e-6 * scale, call
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0  # the calls allocated no device memory
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs0


def test_static_pcg_failure_statuses(multiblock):
    import paper_2605_23088_b300 as yb

    G, g, row, col, vals, diag = multiblock
    n = G.n_nodes
    row_d, col_d, val_d, diag_d = T(row, np.int32), T(col, np.int32), T(vals), T(diag)
    out = torch.empty_like(g)
    # the iteration cap: exactly max_iter iterations, then E_NOCONV
    with pytest.raises(yb.YaspsError) as e:
        yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, g, rel_tol=1e-12, max_iter=3, out=out)
    assert e.value.code == -5
    # a non-finite right-hand side
    bad = g.clone()
    bad[n // 2, 1] = float("nan")
    with pytest.raises(yb.YaspsError) as e:
        yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, bad, out=out)
    assert e.value.code == -8
    # a diagonal block with two negative eigenvalues (det > 0 but indefinite)
    dneg = diag.copy()
    dneg[n - 1] = np.diag([-1.0, -1.0, 1.0])
    with pytest.raises(yb.YaspsError) as e:
        yb.pcg_solve_static(n, row_d, col_d, val_d, T(dneg), g, out=out)
    assert e.value.code == -8
    # an upper block whose column lies outside the matrix is skipped and reported
    cbad = col.copy()
    cbad[len(cbad) // 3] = n + 5
    with pytest.raises(yb.YaspsError) as e:
        yb.pcg_solve_static(n, row_d, T(cbad, np.int32), val_d, diag_d, g, out=out)
    assert e.value.code == -1 and "outside" in str(e.value)
    # the output may not alias the right-hand side
    with pytest.raises(yb.YaspsError) as e:
        yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, g, out=g)
    assert e.value.code == -1
    # wrong dtypes never reach the library
    with pytest.raises(ValueError):
        yb.pcg_solve_static(n, row_d.long(), col_d, val_d, diag_d, g, out=out)
    # a zero right-hand side is solved by p = 0
    out.fill_(1.0)
    p, it, rr = yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, torch.zeros_like(g), out=out)
    assert it == 0 and float(out.abs().max()) == 0.0
    # and a good call still works after the failures
    p, it, rr = yb.pcg_solve_static(n, row_d, col_d, val_d, diag_d, g, rel_tol=1e-8, out=out)
    assert rr <= 1e-8


def test_static_pcg_rejects_oversize():
    import paper_2605_23088_b300 as yb

    n = 65537
    z = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    d = torch.zeros((n, 3, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    with pytest.raises(yb.YaspsError, match="capacity"):
        yb.pcg_solve_static(n, e, e, torch.zeros((0, 3, 3), dtype=torch.float64, device="cuda"), d, z)
