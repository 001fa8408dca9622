"""The SpMV layout study's kernels (yasps_spmv_format) against the oracle.

The matrix is the oracle's own assembly of the two-cube scene in contact
(static and contact parts); each of the four layouts, in FP64 and FP32, in
the natural node order and after a seeded renumbering of the nodes, must give
the oracle's y = H x: FP64 within 1e-12 and FP32 within 1e-5 of max |y|
(products and sums of 3x3 blocks, rounding only).  A block outside its
layout is skipped and flagged.
"""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def matrix():
    s = scenes.cubes_scene()
    O = oracle.OracleSystem(s)
    x, v = O.initial_state()
    for _ in range(3):
        x, v, rc, _ = O.step(x, v)
        assert rc == 0
    O.assemble(x, O.xtilde(x, v))
    rows, cols, vals = [], [], []
    diag = None
    for which in (0, 1):
        rp, col, blk, dg = O.bsr(which)
        rows.append(np.repeat(np.arange(O.nn), np.diff(rp)))
        cols.append(col)
        vals.append(blk)
        diag = dg if diag is None else diag + dg
    assert len(rows[1]) > 0  # contact blocks present
    return O, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), diag


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("renumber", [False, True])
def test_layouts_match_oracle_spmv(matrix, precision, renumber):
    import bench
    import paper_2605_23088_b300 as yb

    O, row, col, vals, diag = matrix
    n = O.nn
    rng = np.random.default_rng(11)
    x = rng.normal(size=(n, 3))
    ref = O.spmv(x)
    perm = rng.permutation(n) if renumber else None
    d, lay = bench.spmv_layouts(row, col, vals, diag, perm)
    xo = x if perm is None else x[np.argsort(perm)]
    dt = torch.float64 if precision == 0 else torch.float32
    tol = 1e-12 if precision == 0 else 1e-5
    for name in yb.SPMV_FORMATS:
        r_, c_, v_ = lay[name]
        X = torch.as_tensor(xo, dtype=dt, device="cuda")
        Y = torch.full_like(X, float("nan"))
        flag = torch.zeros(1, dtype=torch.int32, device="cuda")
        yb.spmv_format(yb.SPMV_FORMATS.index(name), n, torch.as_tensor(r_, device="cuda"),
                       torch.as_tensor(c_, device="cuda"), torch.as_tensor(v_, dtype=dt, device="cuda"),
                       torch.as_tensor(d, dtype=dt, device="cuda"), X, Y, flag)
        y = Y.double().cpu().numpy()
        if perm is not None:
            y = y[perm]
        assert int(flag.item()) == 0
        assert np.abs(y - ref).max() <= tol * np.abs(ref).max(), name


def test_block_outside_layout_is_flagged(matrix):
    import bench
    import paper_2605_23088_b300 as yb

    O, row, col, vals, diag = matrix
    d, lay = bench.spmv_layouts(row, col, vals, diag)
    r_, c_, v_ = lay["upper_bsr"]
    r_ = r_.copy()
    r_[3] = c_[3]  # a diagonal coordinate in an upper layout
    X = torch.ones((O.nn, 3), dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    yb.spmv_format(yb.SPMV_UPPER_BSR, O.nn, torch.as_tensor(r_, device="cuda"), torch.as_tensor(c_, device="cuda"),
                   torch.as_tensor(v_, device="cuda"), torch.as_tensor(d, device="cuda"), X, Y, flag)
    torch.cuda.synchronize()
    assert int(flag.item()) == 1
