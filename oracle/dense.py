"""Dense FP64 oracle: the CARE, its residual, Newton's method, and independent solvers.

Test infrastructure only (see ``oracle/__init__.py``).

Notation follows Section 2 of the paper: the Riccati operator
    R(X) = A^T X + X A - X B B^T X + C^T C,
its Frechet derivative  R'_X[Y] = (A - B B^T X)^T Y + Y (A - B B^T X),
and Newton's method  X_{k+1} = X_k + Y_k  with  R'_{X_k}[Y_k] = -R(X_k)
(Eq. (2.2), the correction Lyapunov equation).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def riccati_residual(A, B, C, X):
    """R(X) = A^T X + X A - X B B^T X + C^T C  (Section 2, definition of the Riccati operator)."""
    XB = X @ B
    return A.T @ X + X @ A - XB @ XB.T + C.T @ C


def lyap_bartels_stewart(F, Q):
    """Solve F X + X F^T + Q = 0 for X (Q symmetric) by the Bartels-Stewart method.

    Complex Schur form F = U T U^*; with Y = U^* X U and Qt = U^* Q U the
    equation becomes T Y + Y T^* + Qt = 0.  Column j of Y T^* is
    sum_{k >= j} conj(T[j, k]) y_k, so the columns are found from the last to
    the first by the upper-triangular solves
        (T + conj(T[j, j]) I) y_j = -qt_j - sum_{k > j} conj(T[j, k]) y_k.
    """
    n = F.shape[0]
    T, U = sla.schur(F.astype(complex), output="complex")
    Qt = U.conj().T @ Q @ U
    Y = np.zeros((n, n), dtype=complex)
    d = np.arange(n)
    for j in range(n - 1, -1, -1):
        rhs = -Qt[:, j]
        if j + 1 < n:
            rhs = rhs - Y[:, j + 1:] @ np.conj(T[j, j + 1:])
        M = T.copy()
        M[d, d] += np.conj(T[j, j])
        Y[:, j] = sla.solve_triangular(M, rhs, lower=False, check_finite=False)
    X = (U @ Y @ U.conj().T).real
    return 0.5 * (X + X.T)


def newton_care(A, B, C, X0=None, tol=1e-14, maxit=60, stag=None, keep_iterates=False):
    """Newton's method for the CARE in the correction form of Section 2.

    X_0 = 0 requires A stable (the configurations here are).  Each step solves
    (A - B B^T X_k)^T Y_k + Y_k (A - B B^T X_k) = -R(X_k) and sets
    X_{k+1} = X_k + Y_k.  Stops when ||R(X_k)||_F <= tol ||C^T C||_F, when the
    residual ratio exceeds ``stag`` (the paper's stagnation test, Section 5;
    off by default because from X_0 = 0 the residual may grow in the first
    steps before the monotone phase), once it stops decreasing at rounding
    level, or after ``maxit`` steps.
    """
    n = A.shape[0]
    X = np.zeros((n, n)) if X0 is None else np.array(X0, dtype=float)
    ctc = np.linalg.norm(C @ C.T)
    hist, iters = [], [X.copy()] if keep_iterates else None
    prev = None
    for _ in range(maxit + 1):
        R = riccati_residual(A, B, C, X)
        r = np.linalg.norm(R)
        hist.append(r)
        if r <= tol * ctc:
            break
        if stag is not None and prev is not None and r / prev > stag:
            break
        if prev is not None and r < 1e-12 * ctc and r >= prev:
            break
        prev = r
        Ak = A - B @ (B.T @ X)
        Y = lyap_bartels_stewart(Ak.T, R)
        X = X + Y
        X = 0.5 * (X + X.T)
        if keep_iterates:
            iters.append(X.copy())
    out = dict(X=X, res_hist=np.array(hist), rel_res=hist[-1] / ctc)
    if keep_iterates:
        out["iterates"] = iters
    return out


def hamiltonian_care(A, B, C):
    """Stabilising CARE solution from the stable invariant subspace of the Hamiltonian
    [[A, -B B^T], [-C^T C, -A^T]]: ordered real Schur form, X = U2 U1^{-1}."""
    n = A.shape[0]
    H = np.block([[A, -B @ B.T], [-C.T @ C, -A.T]])
    T, U, sdim = sla.schur(H, output="real", sort="lhp")
    assert sdim == n, "Hamiltonian has eigenvalues on the imaginary axis"
    U1, U2 = U[:n, :n], U[n:, :n]
    X = np.linalg.solve(U1.T, U2.T).T
    return 0.5 * (X + X.T)


def scalar_care(a, b, c):
    """n = m = p = 1:  2 a x - b^2 x^2 + c^2 = 0, stabilising root x = (a + sqrt(a^2 + b^2 c^2)) / b^2,
    evaluated in the algebraically equal form c^2 / (sqrt(a^2 + b^2 c^2) - a), which has no
    cancellation for a < 0."""
    s = np.sqrt(a * a + b * b * c * c)
    return (c * c) / (s - a)


def lowrank_diff_fro(Z, Y):
    """||Z Z^T - Y Y^T||_F without forming n x n matrices: with [Z, Y] = Q [R1, R2]
    (thin QR), Z Z^T - Y Y^T = Q (R1 R1^T - R2 R2^T) Q^T."""
    r = Z.shape[1]
    _, R = np.linalg.qr(np.hstack([Z, Y]))
    R1, R2 = R[:, :r], R[:, r:]
    return np.linalg.norm(R1 @ R1.T - R2 @ R2.T)


def lowrank_fro(Z):
    """||Z Z^T||_F = ||Z^T Z||_F."""
    return np.linalg.norm(Z.T @ Z)
