"""Failure detection, injected on the host (no GPU fault, trap or hang): bad inputs,
an unstable operator, starved inner solves, too small a factor capacity, and an
expired bounded wait in the tensor-core pipeline (a test hook that withholds the
operand copies).  Each returns its status code and leaves the context usable."""
import ctypes as ct

import numpy as np
import pytest

import care_inputs as ci

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def small():
    return ci.config_small_fdm()


def dcsr(pb, prob, shift=0.0):
    val = prob.A.val.copy()
    if shift:
        rows = np.repeat(np.arange(prob.n), np.diff(prob.A.rowptr))
        val[rows == prob.A.colind] += shift
    return pb.CSR.from_arrays(prob.A.n, prob.A.rowptr, prob.A.colind, val)


def _status(pb, fn):
    with pytest.raises(pb.CareError) as e:
        fn()
    return pb.status_string(e.value.status)


def test_nonfinite_inputs(pb, small):
    B = small.B.copy()
    B[7, 0] = np.nan
    assert _status(pb, lambda: pb.care_solve(dcsr(pb, small), B, small.C, tol=1e-10, r_cap=64)) == "CARE_NONFINITE"
    C = small.C.copy()
    C[0, 3] = np.inf
    assert _status(pb, lambda: pb.care_solve(dcsr(pb, small), small.B, C, tol=1e-10, r_cap=64)) == "CARE_NONFINITE"
    # the next solve on the same context works
    Z, info = pb.care_solve(dcsr(pb, small), small.B, small.C, tol=1e-10, r_cap=256)
    assert info["status"] == "CARE_OK"


def test_unstable_operator(pb, small):
    """A + c I with c above the spectral radius has every eigenvalue in the right
    half-plane: K_0 = 0 is not stabilising and NLR-ADI cannot start."""
    A = small.A.to_dense()
    c = 2.0 * np.abs(np.linalg.eigvals(A)).max()
    for prec in ("mixed", "fp64"):
        st = _status(pb, lambda: pb.care_solve(dcsr(pb, small, c), small.B, small.C, tol=1e-10, prec=prec,
                                               r_cap=64))
        assert st == "CARE_UNSTABLE", (prec, st)


def test_starved_inner_solves_are_counted(pb, small):
    """One Krylov iteration per shifted solve: the shifted-solve entry point reports
    CARE_INNER_FAILED; inside care_solve inexact inner solves are allowed (as in the
    paper) but counted, and the refinement still ends with a valid status."""
    op = pb.Operator(dcsr(pb, small))
    o = pb.default_options(krylov_maxit_hi=1, krylov_maxit_lo=1)
    W = ci.random_block(small.n, 3, 91)
    L = pb.lib()
    # through the binding, which accepts status 7 and returns the iteration count
    V, it = pb.shifted_solve(op, W, -500.0, prec="fp64", opts=o)
    assert it == 1
    Z, info = pb.care_solve(dcsr(pb, small), small.B, small.C, tol=1e-10, prec="mixed", r_cap=256, opts=o,
                            allow=(5, 6, 7))
    assert info["krylov_unconverged"] > 0
    assert info["status"] in ("CARE_OK", "CARE_STAGNATED", "CARE_NOT_CONVERGED", "CARE_INNER_FAILED")


def test_rank_capacity(pb, small):
    st = _status(pb, lambda: pb.care_solve(dcsr(pb, small), small.B, small.C, tol=1e-10, r_cap=2))
    assert st == "CARE_ERR_RANK_CAPACITY"


def test_tensor_core_wait_expires_and_context_survives(pb):
    if not pb.tc_available():
        pytest.skip("tensor-core path needs sm_103")
    X = torch.randn(4096, 64, dtype=torch.float64, device="cuda")
    pb.lib().care_tc_test_starve(1)
    try:
        st = _status(pb, lambda: pb.gram_tc(X, X, "f64"))
    finally:
        pb.lib().care_tc_test_starve(0)
    assert st == "CARE_TIMEOUT"
    # the context is intact: the same product now succeeds and is right
    G = pb.gram_tc(X, X, "f64").cpu().numpy()
    Xh = X.cpu().numpy()
    assert np.allclose(G, Xh.T @ Xh, rtol=1e-13, atol=1e-10)
