"""ILU(0) of the shifted matrix M_p = (A + p I)^T on the device (Section 5.2's GMRES
preconditioner) against the oracle's IKJ elimination: the exact factor entry by
entry (FP64 and FP32, real and complex shifts, several hundred rows per wave of the
row-ticket schedule and a ragged tail), and the fixed-point sweep factor as an
approximation whose pattern residual the exact factor beats."""
import numpy as np
import pytest
import scipy.sparse as sp

import care_inputs as ci
from oracle.precond import ilu0, ilu0_split, shifted_transpose

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


def _problem(case):
    if case == "conv3d":
        q = ci.convection_diffusion(11, (10.0, 50.0, 100.0))  # n = 1331
        return sp.csr_matrix((q.val, q.colind, q.rowptr), shape=(q.n, q.n))
    if case == "fdm2d":
        return ci.config_fdm2d(43, 2, 2).A.to_scipy()  # n = 1849
    rng = np.random.default_rng(11)  # unstructured: random pattern plus the diagonal
    n = 1500
    R = sp.random(n, n, density=0.003, random_state=12, format="csr")
    return sp.csr_matrix(R - sp.diags(4.0 + rng.random(n)))


def _op(pb, A):
    A = sp.csr_matrix(A)
    return pb.Operator(pb.CSR.from_arrays(A.shape[0], A.indptr.astype(np.int32), A.indices.astype(np.int32),
                                          A.data.astype(np.float64)))


def _pattern_residual(M, F):
    L, U = ilu0_split(F)
    D = (L @ U - M).tocsr()
    mask = sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape)
    return abs(D.multiply(mask)).max() / abs(M).max()


@pytest.mark.parametrize("case", ["conv3d", "fdm2d", "random"])
@pytest.mark.parametrize("shift", [-3.0, -2.0 + 5.0j])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_ilu0_exact_matches_oracle(pb, case, shift, dtype):
    A = _problem(case)
    n = A.shape[0]
    op = _op(pb, A)
    F_dev = pb.ilu0(op, shift, exact=True, dtype=dtype).cpu().numpy()
    M = shifted_transpose(A, shift)
    F_ref = ilu0(M)
    assert np.array_equal(M.indptr, op_rowptr(pb, op)) and M.nnz == F_dev.shape[0]
    scale = np.abs(F_ref.data).max()
    err = np.abs(F_dev - F_ref.data).max() / scale
    tol = 1e-13 if dtype == torch.float64 else 2e-6
    assert err < tol, (case, shift, err)
    # the sweep factor (the default, fewer synchronisations) only approximates it
    F_sw = pb.ilu0(op, shift, exact=False, dtype=dtype).cpu().numpy()
    Fs = sp.csr_matrix((F_sw.astype(F_ref.dtype), F_ref.indices, F_ref.indptr), shape=(n, n))
    Fe = sp.csr_matrix((F_dev.astype(F_ref.dtype), F_ref.indices, F_ref.indptr), shape=(n, n))
    assert _pattern_residual(M, Fe) <= max(_pattern_residual(M, Fs), 10 * tol)


def op_rowptr(pb, op):
    base = op.mem.data_ptr()
    off = int(op.op.rowptr_t) - base
    return op.mem[off:off + 4 * (op.n + 1)].view(torch.int32).cpu().numpy()


def test_ilu0_exact_gmres_solve(pb):
    """GMRES preconditioned by the exact ILU(0) (the paper's configuration) on one
    shifted block solve, checked against a sparse direct solve; fewer iterations
    than with the sweep factor or none."""
    A = _problem("conv3d")
    n = A.shape[0]
    op = _op(pb, A)
    W = ci.random_block(n, 6, 5)
    p = -4.0 + 2.0j
    ref = sp.linalg.spsolve(sp.csc_matrix(shifted_transpose(A, p)), W.astype(complex))
    its = {}
    for name, pc in (("none", pb.PRECOND_NONE), ("ilu0", pb.PRECOND_ILU0), ("exact", pb.PRECOND_ILU0_EXACT)):
        o = pb.default_options(krylov=pb.KRYLOV_GMRES, precond=pc, krylov_maxit_hi=4000)
        V, its[name] = pb.shifted_solve(op, W, p, prec="fp64", opts=o)
        rel = np.abs(V.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert rel < 1e-8, (name, rel)
    assert its["exact"] <= its["ilu0"] < its["none"], its
