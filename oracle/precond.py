"""ILU(0) of a shifted operator: the preconditioner of the restarted GMRES that
Section 5.2 uses for every shifted solve of NLR-ADI / LR-ADI.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): nothing in the library
imports this module.

ILU(0) (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed., Sec. 10.3.2)
factors M ~ L U with L unit lower triangular and U upper triangular, both kept on
the sparsity pattern of M (no fill).  It is Gaussian elimination in the row-by-row
(IKJ) order in which every update that would land outside the pattern is dropped.
Its defining property, used as the pin: (L U)_ij = M_ij for every (i, j) in the
pattern.  Written as plain Python loops over a CSR with sorted column indices, for
small cases only.
"""
import numpy as np
import scipy.sparse as sp


def ilu0(M):
    """ILU(0) of the square sparse matrix M (real or complex).

    Returns a CSR matrix F with M's pattern (columns sorted in each row): its
    strictly lower part holds L below the unit diagonal, the rest holds U.
    Every diagonal entry of M must be stored and every pivot nonzero.
    """
    F = sp.csr_matrix(M, copy=True)
    F.sort_indices()
    n = F.shape[0]
    ptr, col = F.indptr, F.indices
    val = F.data.astype(np.complex128 if np.iscomplexobj(F.data) else np.float64)
    diag = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        for q in range(ptr[i], ptr[i + 1]):
            if col[q] == i:
                diag[i] = q
    if np.any(diag < 0):
        raise ValueError("ilu0: a diagonal entry is not stored")
    for i in range(n):
        where = {int(col[q]): q for q in range(ptr[i], ptr[i + 1])}
        for q in range(ptr[i], ptr[i + 1]):
            k = int(col[q])
            if k >= i:
                break
            # l_ik = a_ik / u_kk, then row i -= l_ik * (row k of U) on the pattern
            val[q] = val[q] / val[diag[k]]
            for r in range(diag[k] + 1, ptr[k + 1]):
                j = int(col[r])
                t = where.get(j)
                if t is not None:
                    val[t] -= val[q] * val[r]
        if val[diag[i]] == 0:
            raise ZeroDivisionError(f"ilu0: zero pivot in row {i}")
    return sp.csr_matrix((val, col.copy(), ptr.copy()), shape=F.shape)


def ilu0_split(F):
    """(L, U) from the packed factor of ``ilu0``: L unit lower, U upper (CSR)."""
    n = F.shape[0]
    L = sp.tril(F, k=-1, format="csr") + sp.eye(n, dtype=F.dtype, format="csr")
    U = sp.triu(F, k=0, format="csr")
    return L, U


def shifted_transpose(A, p):
    """M_p = (A + p I)^T as CSR with sorted columns: the base matrix of every
    shifted solve once the SMW formula of Section 4 has removed the low-rank
    feedback term."""
    n = A.shape[0]
    M = sp.csr_matrix((sp.csr_matrix(A) + p * sp.eye(n)).T)
    M.sort_indices()
    return M
