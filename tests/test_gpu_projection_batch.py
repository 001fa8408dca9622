"""The batched warp-Jacobi projection (yasps_project_batch) against numpy.

Project(A) = V max(Lambda, 0) V^T with numpy.linalg.eigh as the library
primitive, for every size the projection study uses (3, 6, 9, 12, 15, 24),
random symmetric matrices and the study's point-point barrier Hessians in node
and position space.  FP64 within 1e-10 and FP32 within 2e-5 of max |A|.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def project(A):
    lam, V = np.linalg.eigh(0.5 * (A + A.T))
    return (V * np.maximum(lam, 0.0)) @ V.T


@pytest.mark.parametrize("n", [3, 6, 9, 12, 15, 24])
@pytest.mark.parametrize("precision", [0, 1])
def test_random_symmetric(n, precision):
    import paper_2605_23088_b300 as yb

    rng = np.random.default_rng(n)
    B = rng.normal(size=(37, n, n))
    A = 0.5 * (B + B.transpose(0, 2, 1)) + rng.normal(size=(37, 1, 1)) * np.eye(n)
    dt = torch.float64 if precision == 0 else torch.float32
    out = yb.project_batch(torch.as_tensor(A, dtype=dt, device="cuda")).double().cpu().numpy()
    tol = 1e-10 if precision == 0 else 2e-5
    for k in range(len(A)):
        ref = project(A[k])
        assert np.abs(out[k] - ref).max() <= tol * np.abs(A[k]).max(), (n, k)


def test_study_inputs():
    import bench
    import paper_2605_23088_b300 as yb

    mats = bench.pp_barrier_hessians(16)
    for n, H in mats.items():
        out = yb.project_batch(torch.as_tensor(H, device="cuda")).cpu().numpy()
        for k in range(len(H)):
            ref = project(H[k])
            assert np.abs(out[k] - ref).max() <= 1e-10 * np.abs(H[k]).max(), (n, k)
