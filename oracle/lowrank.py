"""Low-rank FP64 oracle: LR-ADI, NLR-ADI, Algorithms 1 and 2, Framework 1.

Test infrastructure only (see ``oracle/__init__.py``).

Everything is float64 (the paper's u_s = u = u_r = u_c = FP64 setting,
Section 5) unless an inner precision u_s = FP32 is asked for (``inner="fp32"``):
then NLR-ADI and the correction LR-ADI solves run in IEEE single precision
(float32 / complex64 arrays, so numpy and LAPACK compute in single precision),
as in the FP32 rows of Section 5.1, while Algorithms 1 and 2 stay in float64.
Shifted solves use a sparse (SuperLU) or dense (LAPACK) LU factorisation of
M_p = (A + p I)^T, complex when p is complex; the feedback term of the
closed-loop matrix A_k = A - B K^T is removed with the
Sherman-Morrison-Woodbury formula of Section 4.

Readings of points the paper leaves open (each is a named choice here):
  * LR-ADI (not printed; Section 4 cites the low-rank ADI literature): the
    residual-factor form with real arithmetic for complex-conjugate shift
    pairs (Benner, Kuerschner, Saak 2013); stop when
    ||W_j^T W_j||_2 <= tol ||W_0^T W_0||_2 or after jmax shifts.
  * Shifts (Section 5: "generated dynamically from Krylov subspaces"):
    projection shifts -- Ritz values of F = A_k^T on an orthonormal basis of
    the right-hand side (extended by Krylov blocks F W ... until it has at
    least ``hmin`` columns), later on the span of the newest ADI block;
    values in the closed right half-plane are mirrored, conjugate pairs are
    kept once (Im > 0) and used as a pair; ordered by decreasing modulus.
  * NLR-ADI (not printed; Section 4): Newton-Kleinman with K_0 = 0 (A stable),
    right-hand side [C^T, K_i], K_{i+1} = Z_{i+1} Z_{i+1}^T B, stopping on
    ||K_{i+1} - K_i||_F <= tol_newton ||K_{i+1}||_F.
  * Algorithm 1 keeps lambda >= eta_r and lambda <= -eta_r with
    eta_r = eta_r_rel * max|lambda(H)| (Section 5 parameter list); ||R||_F is
    taken from all eigenvalues before truncation (end of Section 2).
  * Algorithm 2 keeps sigma >= eta_s = eta_s_mult * u * max|sigma(P)|,
    u = 2^-53.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

U_FP64 = 2.0 ** -53
INNER_DTYPES = {"fp64": (np.float64, np.complex128), "fp32": (np.float32, np.complex64),
                "bf16": (np.float32, np.complex64), "fp16": (np.float32, np.complex64)}


def _round_bf16(x):
    """Round float32 values to the nearest bfloat16 (8 significant bits, ties to even),
    returned as float32: the IEEE bit pattern's low 16 bits are rounded away."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    r = ((b + np.uint32(0x7FFF) + ((b >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000))
    r = np.where(np.isfinite(x), r, b)  # inf / nan unchanged
    return r.view(np.float32)


def storage_rounding(inner: str):
    """Lower inner precisions (the paper's future work, Section 6) are modelled as
    FP32 arithmetic whose stored results -- shifted-solve solutions, ADI residual and
    factor blocks, K, and the operator's entries -- are rounded to ``inner`` (bf16:
    8, fp16: 11 significant bits).  Identity for fp32 / fp64."""
    if inner == "bf16":
        f = _round_bf16
    elif inner == "fp16":
        f = lambda x: np.asarray(x, np.float32).astype(np.float16).astype(np.float32)
    else:
        return lambda x: x

    def rnd(x):
        x = np.asarray(x)
        if np.iscomplexobj(x):
            return (f(x.real) + 1j * f(x.imag)).astype(np.complex64)
        return f(x)
    return rnd


class ShiftedSolver:
    """Applies M_p^{-1} with M_p = (A + p I)^T = A^T + p I (Section 4, SMW formula),
    in the inner precision ``inner`` ("fp64" or "fp32")."""

    def __init__(self, A, dense: bool = False, inner: str = "fp64"):
        self.dense = dense
        self.rdt, self.cdt = INNER_DTYPES[inner]
        self.rnd = storage_rounding(inner)
        if dense:
            self.At = self.rnd(np.asarray(A.T if not sp.issparse(A) else A.T.toarray(), dtype=float).astype(self.rdt))
        else:
            self.At = sp.csc_matrix(A.T).astype(self.rdt)
            self.At.data = self.rnd(self.At.data)
        self.n = self.At.shape[0]
        self._cache = {}
        self.nsolves = 0

    def _factor(self, p):
        key = (float(np.real(p)), float(np.imag(p)))
        if key in self._cache:
            return self._cache[key]
        self._cache.clear()
        dt = self.cdt if np.imag(p) != 0 else self.rdt
        if self.dense:
            M = (self.At + np.asarray(p, dtype=dt) * np.eye(self.n, dtype=dt)).astype(dt)
            f = sla.lu_factor(M)
            solve = lambda R, f=f: sla.lu_solve(f, R)
        else:
            M = (self.At.astype(dt) + np.asarray(p, dtype=dt) * sp.identity(self.n, format="csc", dtype=dt)).tocsc()
            f = spla.splu(M)
            solve = f.solve
        self._cache[key] = solve
        return solve

    def solve(self, p, R):
        self.nsolves += 1
        p = complex(p) if np.imag(p) != 0 else float(np.real(p))
        solve = self._factor(p)
        R = np.asarray(R, dtype=self.cdt if isinstance(p, complex) else self.rdt)
        return self.rnd(solve(R))


def smw_solve(solver: ShiftedSolver, B, K, p, W):
    """V = (A_k + p I)^{-T} W with A_k = A - B K^T, via the Sherman-Morrison-Woodbury
    formula of Section 4:
        (A_k + p I)^{-T} = M_p^{-1} + M_p^{-1} K (I_m - B^T M_p^{-1} K)^{-1} B^T M_p^{-1}.
    K = None means no feedback (A_k = A)."""
    V0 = solver.solve(p, W)
    if K is None or not np.any(K):
        return V0
    Y = solver.solve(p, K)
    Bt = np.asarray(B, dtype=Y.real.dtype).T
    m = Bt.shape[0]
    S = np.eye(m, dtype=Y.dtype) - Bt @ Y
    return solver.rnd(V0 + Y @ np.linalg.solve(S, Bt @ V0))


def _orth(X, rtol=1e-12):
    """Orthonormal basis of range(X) from an SVD, dropping directions below rtol * sigma_max."""
    if X.shape[1] == 0:
        return X
    Uu, s, _ = np.linalg.svd(X, full_matrices=False)
    if s.size == 0 or s[0] == 0:
        return X[:, :0]
    return Uu[:, s > rtol * s[0]]


def apply_F(A, B, K, X):
    """F X with F = A_k^T = A^T - K B^T."""
    Y = A.T @ X
    if K is not None and np.any(K):
        Y = Y - K @ (B.T @ X)
    return Y


def projection_shifts(A, B, K, U, hmin=4, maxblocks=4):
    """Ritz values of F = A^T - K B^T on range(U) extended by Krylov blocks until it
    has at least ``hmin`` columns; returns a list of shifts with Re < 0, one
    representative (Im > 0) per conjugate pair, ordered by decreasing modulus."""
    Q = _orth(U)
    blk = Q
    it = 0
    while Q.shape[1] < hmin and it < maxblocks and blk.shape[1] > 0:
        blk = apply_F(A, B, K, blk)
        blk = blk - Q @ (Q.T @ blk)
        blk = blk - Q @ (Q.T @ blk)
        blk = _orth(blk, 1e-8)
        Q = np.hstack([Q, blk])
        it += 1
    Hp = Q.T @ apply_F(A, B, K, Q)
    ev = np.linalg.eigvals(Hp)
    out = []
    for z in ev:
        if not np.isfinite(z) or abs(z) == 0:
            continue
        re, im = -abs(z.real), z.imag
        if abs(im) <= 1e-10 * abs(z):
            out.append(complex(re, 0.0))
        elif im > 0:
            out.append(complex(re, im))
    out.sort(key=lambda z: -abs(z))
    return out


def lradi(A, B, K, W, tol, jmax=50, solver=None, dense=False, split=None, hmin=4, inner="fp64"):
    """LR-ADI for  F X + X F^T + W W^T = 0  with F = A_k^T = A^T - K B^T, X ~ Z Z^T.

    Residual-factor form (Section 4 reading): W_0 = W and per shift p_j
      V_j = (F + p_j I)^{-1} W_{j-1}           (SMW, ``smw_solve``)
      real p:     W_j = W_{j-1} - 2 p V_j,   Z <- [Z, sqrt(-2 p) V_j]
      complex p (used with its conjugate as one double step),
                  gamma = 2 sqrt(-Re p), delta = Re p / Im p,
                  W_{j+1} = W_{j-1} + gamma^2 (Re V_j + delta Im V_j),
                  Z <- [Z, gamma (Re V_j + delta Im V_j), gamma sqrt(delta^2 + 1) Im V_j].
    Stops when ||W^T W||_2 <= tol ||W_0^T W_0||_2 or after jmax shifts.

    ``inner`` = "fp32" runs every step (solves, W update, Z blocks, the residual
    norm and the shift computation) in single precision.

    ``split`` = number of leading columns of W that belong to the first of two
    jointly solved equations (the +/- correction pair of Framework 1); the
    Z columns are then returned as (Z_first, Z_second).
    """
    if solver is None:
        solver = ShiftedSolver(A, dense=dense, inner=inner)
    rdt, rnd = solver.rdt, solver.rnd
    W = rnd(np.array(W, dtype=rdt))
    if rdt != np.float64:
        # the inner equation as u_s holds it: A_k's data rounded to u_s
        if sp.issparse(A):
            A = A.astype(rdt)
            A.data = rnd(A.data)
        else:
            A = rnd(np.asarray(A).astype(rdt))
        B = rnd(np.asarray(B).astype(rdt))
        K = None if K is None else rnd(np.asarray(K).astype(rdt))
    n, b = W.shape
    w0 = np.linalg.norm(W.T @ W, 2)
    blocks = []
    shifts = projection_shifts(A, B, K, W, hmin=hmin)
    j = 0
    used = []
    res_hist = [1.0]
    last_block = None
    while j < jmax and res_hist[-1] > tol:
        if not shifts:
            shifts = projection_shifts(A, B, K, last_block, hmin=hmin)
            if not shifts:
                break
        p = shifts.pop(0)
        used.append(p)
        V = smw_solve(solver, B, K, p, W)
        if p.imag == 0.0:
            pr = rdt(p.real)
            V = V.real if np.iscomplexobj(V) else V
            W = rnd(W - rdt(2.0) * pr * V)
            blk = rnd(rdt(math.sqrt(-2.0 * p.real)) * V)
            blocks.append([blk])
            last_block = blk
            j += 1
        else:
            gam = rdt(2.0 * math.sqrt(-p.real))
            dlt = rdt(p.real / p.imag)
            Vr, Vi = V.real, V.imag
            W = rnd(W + gam * gam * (Vr + dlt * Vi))
            b1 = rnd(gam * (Vr + dlt * Vi))
            b2 = rnd(gam * rdt(math.sqrt(float(dlt) * float(dlt) + 1.0)) * Vi)
            blocks.append([b1, b2])
            last_block = np.hstack([b1, b2])
            j += 2
        res_hist.append(np.linalg.norm(W.T @ W, 2) / w0 if w0 > 0 else 0.0)
    cols = [c for blk in blocks for c in blk]
    Z = np.hstack(cols) if cols else np.zeros((n, 0), dtype=rdt)
    info = dict(steps=j, shifts=used, res_hist=np.array(res_hist), nsolves=solver.nsolves)
    if split is None:
        return Z, info
    Zp = np.hstack([c[:, :split] for c in cols]) if cols else np.zeros((n, 0), dtype=rdt)
    Zm = np.hstack([c[:, split:] for c in cols]) if cols else np.zeros((n, 0), dtype=rdt)
    return (Zp, Zm), info


def nlradi(A, B, C, tol_lyap=1e-12, tol_newton=1e-12, kmax=20, jmax=50, dense=False, inner="fp64"):
    """NLR-ADI initial approximation (Section 4 reading): Newton-Kleinman whose
    step i solves A_i^T X + X A_i + C^T C + K_i K_i^T = 0, A_i = A - B K_i^T,
    by LR-ADI with right-hand side factor [C^T, K_i]; K_{i+1} = Z Z^T B.
    With inner="fp32" every step runs in single precision (Z, K included)."""
    n, m = B.shape
    solver = ShiftedSolver(A, dense=dense, inner=inner)
    rdt, rnd = solver.rdt, solver.rnd
    Bs, Cs = rnd(np.asarray(B).astype(rdt)), rnd(np.asarray(C).astype(rdt))
    K = np.zeros((n, m), dtype=rdt)
    inner_steps = 0
    Z = np.zeros((n, 0), dtype=rdt)
    steps = 0
    for i in range(kmax):
        W = Cs.T if not np.any(K) else np.hstack([Cs.T, K])
        Z, info = lradi(A, Bs, K, W, tol_lyap, jmax, solver=solver, inner=inner)
        inner_steps += info["steps"]
        steps = i + 1
        Knew = rnd(Z @ (Z.T @ Bs))
        dk = np.linalg.norm(Knew - K)
        K = Knew
        if dk <= tol_newton * np.linalg.norm(Knew):
            break
    return Z, dict(newton_steps=steps, adi_steps=inner_steps)


def residual_factor(A, B, C, Z, eta_r_rel=1e-4):
    """Algorithm 1 (Residual Factor Decomposition), Section 2.

    F = [Z, A^T Z, Z Z^T B, C^T] = U T (thin Householder QR);
    M = [[0, I_r, 0, 0], [I_r, 0, 0, 0], [0, 0, -I_m, 0], [0, 0, 0, I_p]];
    H = T M T^T = Q Lambda Q^T; ||R(Z)||_F = ||H||_F (before truncation);
    J+ = {lambda >= eta_r}, J- = {lambda <= -eta_r}, eta_r = eta_r_rel max|lambda|;
    C+ = U Q+ Lambda+^{1/2}, C- = U Q- (-Lambda-)^{1/2}.
    """
    n, r = Z.shape
    m, p = B.shape[1], C.shape[0]
    F = np.hstack([Z, A.T @ Z, Z @ (Z.T @ B), C.T])
    U, T = np.linalg.qr(F)
    q = 2 * r + m + p
    M = np.zeros((q, q))
    M[:r, r:2 * r] = np.eye(r)
    M[r:2 * r, :r] = np.eye(r)
    M[2 * r:2 * r + m, 2 * r:2 * r + m] = -np.eye(m)
    M[2 * r + m:, 2 * r + m:] = np.eye(p)
    H = T @ M @ T.T
    H = 0.5 * (H + H.T)
    lam, Q = np.linalg.eigh(H)
    res = math.sqrt(float(np.sum(lam * lam)))
    eta = eta_r_rel * (np.max(np.abs(lam)) if lam.size else 0.0)
    jp = lam >= eta
    jm = lam <= -eta
    if eta == 0.0:
        jp = lam > 0
        jm = lam < 0
    Cp = U @ (Q[:, jp] * np.sqrt(lam[jp]))
    Cm = U @ (Q[:, jm] * np.sqrt(-lam[jm]))
    return Cp, Cm, res, dict(H=H, lam=lam, q=q)


def solution_factor(Z, Zp, Zm, eta_s_mult=10.0):
    """Algorithm 2 (Solution Factor Decomposition), Section 2.

    G = [Z, Z+, Z-] = V Gamma (thin QR); N = diag(I, I, -I);
    P = Gamma N Gamma^T = Theta Sigma Theta^T; keep sigma >= eta_s
    (eta_s = eta_s_mult * u * max|sigma|); Z_new = V Theta+ Sigma+^{1/2}.
    """
    G = np.hstack([Z, Zp, Zm])
    V, Gam = np.linalg.qr(G)
    d = np.concatenate([np.ones(Z.shape[1] + Zp.shape[1]), -np.ones(Zm.shape[1])])
    P = (Gam * d) @ Gam.T
    P = 0.5 * (P + P.T)
    sig, Th = np.linalg.eigh(P)
    eta = eta_s_mult * U_FP64 * (np.max(np.abs(sig)) if sig.size else 0.0)
    keep = sig >= eta
    if eta == 0.0:
        keep = sig > 0
    return V @ (Th[:, keep] * np.sqrt(sig[keep])), dict(sig=sig, P=P)


def res_paper(A, B, C, Z, res_fro):
    """Res = ||R||_F / (2 ||A||_F ||Z^T Z||_F + ||B^T B||_F ||Z^T Z||_F^2 + ||C C^T||_F) (Section 5)."""
    ztz = np.linalg.norm(Z.T @ Z)
    a_f = np.linalg.norm(A.data) if sp.issparse(A) else np.linalg.norm(A)
    den = 2 * a_f * ztz + np.linalg.norm(B.T @ B) * ztz * ztz + np.linalg.norm(C @ C.T)
    return res_fro / den


def framework1(A, B, C, tau_R=1e-12, kmax=20, jmax=50, tol_lyap=1e-12, tol_newton=1e-12,
               eta_r_rel=1e-4, eta_s_mult=10.0, stag=0.999, dense=False, Z1=None, inner="fp64"):
    """Framework 1 (Factorization-based Newton iterative refinement), Section 2, with
    the inner solves (NLR-ADI and the correction LR-ADI) in ``inner`` precision and
    Algorithms 1-2 in FP64.

    1. Z_1 from NLR-ADI (unless given).
    2. For k = 1..kmax: Algorithm 1 -> C+, C-, ||R(Z_k)||_F; stop if
       ||R||_F <= tau_R ||C^T C||_F or the ratio to the previous residual
       exceeds ``stag``; solve the +/- Lyapunov pair with A_k = A - B K_k^T,
       K_k = Z_k Z_k^T B, as one LR-ADI run on [C+, C-]; Algorithm 2 -> Z_{k+1}.
    """
    if Z1 is None:
        Z, init = nlradi(A, B, C, tol_lyap, tol_newton, kmax, jmax, dense=dense, inner=inner)
        Z = np.asarray(Z, dtype=float)  # stored in u = FP64
    else:
        Z, init = np.array(Z1, float), dict(newton_steps=0, adi_steps=0)
    ctc = np.linalg.norm(C @ C.T)
    solver = ShiftedSolver(A, dense=dense, inner=inner)
    hist = []
    inner_steps = 0
    status = "not_converged"
    outer = 0
    for k in range(1, kmax + 1):
        outer = k
        Cp, Cm, res, _ = residual_factor(A, B, C, Z, eta_r_rel)
        hist.append(res)
        if res <= tau_R * ctc:
            status = "ok"
            break
        if len(hist) > 1 and hist[-1] / hist[-2] > stag:
            status = "stagnated"
            break
        K = Z @ (Z.T @ B)
        # the correction equation is linear in W W^T: its right-hand side is scaled by a
        # power of two to O(1) before the inner-precision solve and Z+- unscaled after
        # (exact in binary arithmetic; it keeps the shrinking residual factors inside the
        # narrow exponent range of fp16)
        W = np.hstack([Cp, Cm])
        wmax = float(np.max(np.abs(W))) if W.size else 0.0
        sc = 2.0 ** -math.floor(math.log2(wmax)) if wmax > 0 else 1.0
        (Zp, Zm), info = lradi(A, B, K, sc * W, tol_lyap, jmax, solver=solver,
                               split=Cp.shape[1], inner=inner)
        inner_steps += info["steps"]
        Z, _ = solution_factor(Z, np.asarray(Zp, float) / sc, np.asarray(Zm, float) / sc, eta_s_mult)
    return Z, dict(status=status, res_hist=np.array(hist), rel_res=hist[-1] / ctc,
                   iter0=(init["newton_steps"], init["adi_steps"]), iter=(outer, inner_steps),
                   rank=Z.shape[1], res_paper=res_paper(A, B, C, Z, hist[-1]))


def shifted_operator_apply(A, p, X):
    """Y = M_p X = (A + p I)^T X (Section 4): the operator of the shifted solves."""
    At = A.T
    Y = At @ X
    return Y + p * X


def gram(X, Y):
    """G = X^T Y (tall-skinny inner products, Section 4 complexity analysis)."""
    return X.T @ Y
