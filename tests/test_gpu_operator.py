"""Setup step (operator preparation): A in CSR (unsorted columns allowed) becomes A^T
in CSR with sorted rows, FP64 and FP32 values, the diagonal, FP32 row sums of A^T
(from FP64 sums), ||A||_F and the structure flags -- checked entry by entry against
SciPy's transpose on the CPU."""
import numpy as np
import pytest
import scipy.sparse as sp

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


def _view(op, ptr, count, dtype):
    """Device array inside the operator's buffer as a CPU numpy copy."""
    base = op.mem.data_ptr()
    off = int(ptr) - base
    es = torch.tensor([], dtype=dtype).element_size()
    return op.mem[off:off + count * es].view(dtype).cpu().numpy()


def _shuffled_csr(M, seed):
    """CSR of M with the column order inside every row permuted."""
    M = sp.csr_matrix(M)
    rng = np.random.default_rng(seed)
    ci_, v = M.indices.copy(), M.data.copy()
    for i in range(M.shape[0]):
        a, b = M.indptr[i], M.indptr[i + 1]
        p = rng.permutation(b - a)
        ci_[a:b], v[a:b] = ci_[a:b][p], v[a:b][p]
    return M.indptr.astype(np.int32), ci_.astype(np.int32), v


@pytest.mark.parametrize("case", ["fdm2d", "fdm3d", "random_missing_diag"])
def test_operator_prepare(pb, case):
    if case == "fdm2d":
        p = ci.config_fdm2d(37, 2, 2)
        A = p.A.to_scipy()
    elif case == "fdm3d":
        q = ci.convection_diffusion(13, (10.0, 50.0, 100.0))
        A = sp.csr_matrix((q.val, q.colind, q.rowptr), shape=(q.n, q.n))
    else:
        rng = np.random.default_rng(7)
        A = sp.random(1000, 1000, density=0.004, random_state=8, format="csr") - 3.0 * sp.eye(1000)
        A = sp.csr_matrix(A.toarray() * (rng.random(1000)[:, None] > 0.01))  # a few empty rows
    n = A.shape[0]
    rp, cidx, val = _shuffled_csr(A, 3)
    op = pb.Operator(pb.CSR.from_arrays(n, rp, cidx, val))
    o = op.op
    At = sp.csr_matrix(A.T)
    At.sort_indices()
    assert o.n == n and o.nnz == At.nnz
    assert np.array_equal(_view(op, o.rowptr_t, n + 1, torch.int32), At.indptr)
    assert np.array_equal(_view(op, o.colind_t, At.nnz, torch.int32), At.indices)
    v64 = _view(op, o.val64_t, At.nnz, torch.float64)
    assert np.array_equal(v64, At.data)
    assert np.array_equal(_view(op, o.val32_t, At.nnz, torch.float32), At.data.astype(np.float32))
    assert np.array_equal(_view(op, o.diag64, n, torch.float64), A.diagonal())
    rs = np.asarray(At.sum(axis=1)).ravel()
    r32 = _view(op, o.rowsum32_t, n, torch.float32).astype(np.float64)
    assert np.all(np.abs(r32 - rs) <= 2.0 ** -24 * np.abs(rs) + 1e-12 * np.abs(At).sum(axis=1).A.ravel())
    assert o.a_fro == pytest.approx(np.sqrt((A.data ** 2).sum()), rel=1e-13)
    assert o.max_row_nnz == int(np.diff(At.indptr).max())
    has_diag = np.all(A.diagonal() != 0) or all(
        (At.indices[At.indptr[i]:At.indptr[i + 1]] == i).any() for i in range(n))
    assert o.full_diag == (1 if has_diag else 0)
    d = A.diagonal()
    assert o.diag_const == (1 if np.all(d == d[0]) else 0)
