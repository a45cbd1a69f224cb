"""Dense-direct shifted solves (CARE_KRYLOV_DENSE_LU: M_p = (A + p I)^T formed densely,
LU with partial pivoting; the solvers of Section 5.1's stability study) against the
oracle's direct SMW solve and NumPy's LU solve, entry by entry: real and complex
shifts, with and without the feedback term, FP64 and FP32, matrices that need row
exchanges, a ragged size, a size spanning several columns per CTA, and an exactly
singular system (reported, finite output)."""
import numpy as np
import pytest
import scipy.sparse as sp

import care_inputs as ci
from oracle import lowrank as ol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


def _op(pb, A):
    A = sp.csr_matrix(A)
    return pb.Operator(pb.CSR.from_arrays(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32),
                                          A.data.astype(np.float64)))


def _dense_opts(pb):
    return pb.default_options(krylov=pb.KRYLOV_DENSE_LU)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("mixed", 2e-4)])
@pytest.mark.parametrize("shift", [-0.3, complex(-0.2, 0.7)])
@pytest.mark.parametrize("feedback", [False, True])
def test_dense_lu_smw_parity(pb, prec, tol, shift, feedback):
    prob = ci.config_dense_conditioning(3)
    As = prob.A.to_scipy()
    op = _op(pb, As)
    W = ci.random_block(prob.n, 4, 81)
    K = 0.05 * ci.random_block(prob.n, 2, 82) if feedback else None
    B = prob.B if feedback else None
    ref = ol.smw_solve(ol.ShiftedSolver(As), B, K, shift, W)
    V, it, st = pb.shifted_solve(op, W, shift, B=B, K=K, prec=prec, opts=_dense_opts(pb), with_status=True)
    V = V.cpu().numpy()
    assert st == 0 and it >= 1
    assert np.abs(V - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("n,shift", [(203, 0.0), (203, complex(0.5, -1.5)), (1000, -2.0)])
def test_dense_lu_pivoting_sizes(pb, n, shift):
    """Zero diagonal (every step exchanges rows), odd size; n = 1000 gives several
    columns per CTA of the factorisation."""
    rng = np.random.default_rng(n)
    Ad = rng.standard_normal((n, n))
    np.fill_diagonal(Ad, 0.0)
    op = _op(pb, Ad)
    W = ci.random_block(n, 3, 83)
    M = (Ad + shift * np.eye(n)).T
    ref = np.linalg.solve(M, W.astype(M.dtype))
    V, _, st = pb.shifted_solve(op, W, shift, prec="fp64", opts=_dense_opts(pb), with_status=True)
    V = V.cpu().numpy()
    cond = np.linalg.cond(M)
    assert st == 0
    assert np.abs(V - ref).max() <= 1e-13 * cond * np.abs(ref).max(), cond


def test_dense_lu_singular_is_reported(pb):
    """An exactly singular M_p (a zero column) is reported as an inner failure and
    leaves finite numbers behind."""
    n = 64
    Ad = np.diag(-1.0 - np.arange(n, dtype=float)) + np.triu(np.ones((n, n)), 1)
    Ad[5, :] = 0.0  # a zero row of A: M_p = A^T has a zero column, singular for p = 0
    op = _op(pb, Ad)
    W = ci.random_block(n, 2, 84)
    V, _, st = pb.shifted_solve(op, W, 0.0, prec="fp64", opts=_dense_opts(pb), with_status=True)
    assert st == 7
    assert torch.isfinite(V).all()
