"""Pins of the oracle's ILU(0) (Section 5.2's GMRES preconditioner): the defining
pattern identity (L U)_ij = M_ij on the pattern, exactness where elimination
makes no fill (tridiagonal, full pattern) against SciPy's LU, and the dropped
fill on a 2-D Laplacian, where L U - M is nonzero exactly off the pattern."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

import care_inputs as ci
from oracle.precond import ilu0, ilu0_split, shifted_transpose


def _pattern_residual(M, F):
    L, U = ilu0_split(F)
    D = (L @ U - M).tocsr()
    mask = sp.csr_matrix((np.ones(M.nnz), M.indices, M.indptr), shape=M.shape)
    on = D.multiply(mask)
    off = D - on
    scale = abs(M).max()
    return (abs(on).max() if on.nnz else 0.0) / scale, (abs(off).max() if off.nnz else 0.0) / scale


@pytest.mark.parametrize("p", [-2.0, -1.5 + 3.0j])
def test_ilu0_pattern_identity_convection(p):
    q = ci.convection_diffusion(6, (10.0, 50.0, 100.0))
    A = sp.csr_matrix((q.val, q.colind, q.rowptr), shape=(q.n, q.n))
    M = shifted_transpose(A, p)
    F = ilu0(M)
    assert F.nnz == M.nnz and np.array_equal(F.indices, M.indices)
    on, off = _pattern_residual(M, F)
    assert on < 1e-13
    assert off > 1e-6  # a 3-D stencil creates fill, which ILU(0) drops


def test_ilu0_tridiagonal_is_exact_lu():
    rng = np.random.default_rng(3)
    n = 40
    T = sp.diags([rng.standard_normal(n - 1), 4.0 + rng.random(n), rng.standard_normal(n - 1)], [-1, 0, 1],
                 format="csr")
    F = ilu0(T)
    L, U = ilu0_split(F)
    P, Ld, Ud = sla.lu(T.toarray())
    assert np.array_equal(P, np.eye(n))  # diagonally dominant: no row exchanges
    assert np.abs(L.toarray() - Ld).max() < 1e-14
    assert np.abs(U.toarray() - Ud).max() < 1e-13


def test_ilu0_full_pattern_is_lu_complex():
    rng = np.random.default_rng(4)
    n = 12
    Md = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * n * np.eye(n)
    F = ilu0(sp.csr_matrix(Md))
    L, U = ilu0_split(F)
    P, Ld, Ud = sla.lu(Md)
    assert np.array_equal(P, np.eye(n))
    assert np.abs(L.toarray() - Ld).max() < 1e-13
    assert np.abs(U.toarray() - Ud).max() < 1e-12 * np.abs(Md).max()


def test_ilu0_laplacian_fill_dropped_only_off_pattern():
    p = ci.config_fdm2d(9, 1, 1)
    M = shifted_transpose(p.A.to_scipy(), -0.5)
    F = ilu0(M)
    L, U = ilu0_split(F)
    D = (L @ U - M).toarray()
    pat = M.toarray() != 0
    scale = np.abs(M.toarray()).max()
    assert np.abs(D[pat]).max() < 1e-14 * scale
    # classic 5-point fill (grid rows of N points): eliminating entry (N, 0) with row 0
    # of U would create (N, 1), and symmetrically (1, N); both lie off the pattern
    N = 9
    assert np.abs(D[N, 1]) > 1e-3 * scale and np.abs(D[1, N]) > 1e-3 * scale


def test_ilu0_missing_diagonal_rejected():
    M = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 2.0]]))
    M.eliminate_zeros()
    with pytest.raises(ValueError):
        ilu0(M)
