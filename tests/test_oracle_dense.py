"""Pins for the dense FP64 oracle against facts fixed by the mathematics (CPU only)."""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import care_inputs as ci
from oracle import dense as od

GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("a,b,c", [(-1.0, 1.0, 1.0), (-3.0, 0.5, 2.0), (-1e-3, 2.0, 0.1), (-50.0, 1e-2, 3.0)])
def test_scalar_closed_form(a, b, c):
    """P1: n = m = p = 1, x = (a + sqrt(a^2 + b^2 c^2)) / b^2, closed loop a - b^2 x = -sqrt(a^2 + b^2 c^2)."""
    s = math.sqrt(a * a + b * b * c * c)
    x_exact = c * c / (s - a)  # = (a + s) / b^2 without cancellation
    assert x_exact == pytest.approx((a + s) / (b * b), rel=1e-6)
    out = od.newton_care(np.array([[a]]), np.array([[b]]), np.array([[c]]), tol=1e-15, maxit=60)
    x = out["X"][0, 0]
    assert abs(x - x_exact) <= 1e-12 * abs(x_exact)
    assert abs((a - b * b * x) + math.sqrt(a * a + b * b * c * c)) <= 1e-10 * math.sqrt(a * a + b * b * c * c)
    assert od.scalar_care(a, b, c) == pytest.approx(x_exact, rel=1e-15)


def test_eigen_aligned_dense():
    """P2: A symmetric stable, B = V_S diag(beta), C = diag(gamma) V_S^T decouple the CARE:
    X* = sum_{i in S} x_i v_i v_i^T with x_i the scalar closed form."""
    n = 60
    s = ci.Stream(ci.SEED, 11)
    V = ci.haar_orthogonal(n, s)
    lam = -np.logspace(-1, 2, n)
    A = (V * lam) @ V.T
    S = [3, 17, 40]
    beta = np.array([0.7, 2.0, 0.3])
    gamma = np.array([1.5, 0.2, 4.0])
    B = V[:, S] * beta
    C = (V[:, S] * gamma).T
    X_exact = sum(od.scalar_care(lam[i], beta[t], gamma[t]) * np.outer(V[:, i], V[:, i])
                  for t, i in enumerate(S))
    X = od.newton_care(A, B, C)["X"]
    assert np.linalg.norm(X - X_exact) <= 1e-12 * np.linalg.norm(X_exact)


def _nonsym(n, sid):
    s = ci.Stream(ci.SEED, sid)
    M = s.normal(n * n).reshape(n, n) / math.sqrt(n)
    A = M - (np.max(np.linalg.eigvals(M).real) + 0.5) * np.eye(n)
    B = s.normal(n * 2).reshape(n, 2)
    C = s.normal(3 * n).reshape(3, n)
    return A, B, C


def test_newton_matches_hamiltonian_and_library():
    """P5: tiny nonsymmetric CARE -- Newton = Hamiltonian stable subspace = SciPy's CARE solver."""
    A, B, C = _nonsym(30, 12)
    X = od.newton_care(A, B, C)["X"]
    Xh = od.hamiltonian_care(A, B, C)
    Xs = sla.solve_continuous_are(A, B, C.T @ C, np.eye(B.shape[1]))
    nx = np.linalg.norm(X)
    assert np.linalg.norm(X - Xh) <= 1e-11 * nx
    assert np.linalg.norm(X - Xs) <= 1e-11 * nx


def test_newton_small_fdm_matches_library():
    """The n=400 convection-diffusion CARE (complex spectrum): Newton vs SciPy and Hamiltonian."""
    p = ci.config_small_fdm()
    A = p.A.to_dense()
    out = od.newton_care(A, p.B, p.C)
    X = out["X"]
    assert out["rel_res"] <= 1e-14
    Xs = sla.solve_continuous_are(A, p.B, p.C.T @ p.C, np.eye(1))
    assert np.linalg.norm(X - Xs) <= 1e-11 * np.linalg.norm(X)


def test_bartels_stewart_closed_forms():
    """P4: F = a I gives X = W W^T / (-2a); symmetric F = V diag(l) V^T gives
    X = V [(V^T W W^T V)_ij / (-(l_i + l_j))] V^T; general F vs SciPy."""
    n = 40
    s = ci.Stream(ci.SEED, 13)
    W = s.normal(n * 3).reshape(n, 3)
    a = -2.5
    X = od.lyap_bartels_stewart(a * np.eye(n), W @ W.T)
    assert np.allclose(X, W @ W.T / (-2 * a), rtol=0, atol=1e-13 * np.linalg.norm(W) ** 2)
    V = ci.haar_orthogonal(n, s)
    lam = -np.logspace(-2, 1, n)
    F = (V * lam) @ V.T
    G = V.T @ W @ W.T @ V
    X_exact = V @ (G / -(lam[:, None] + lam[None, :])) @ V.T
    X = od.lyap_bartels_stewart(F, W @ W.T)
    assert np.linalg.norm(X - X_exact) <= 1e-11 * np.linalg.norm(X_exact)
    A, _, _ = _nonsym(n, 14)
    X = od.lyap_bartels_stewart(A, W @ W.T)
    # residual of the equation itself, and a library cross-check
    assert np.linalg.norm(A @ X + X @ A.T + W @ W.T) <= 1e-12 * np.linalg.norm(W @ W.T) * np.linalg.norm(A) * 10
    Xs = sla.solve_continuous_lyapunov(A, -W @ W.T)
    assert np.linalg.norm(X - Xs) <= 1e-11 * np.linalg.norm(X)


def test_newton_invariants():
    """P6: X = X^T >= 0, A - B B^T X_k stable for every iterate, X_k >= X_{k+1} for k >= 1
    (Section 2, properties of exact Newton), quadratic convergence in the tail."""
    p = ci.config_dense_conditioning(1)
    A = p.A.to_dense()
    out = od.newton_care(A, p.B, p.C, keep_iterates=True)
    its = out["iterates"]
    X = out["X"]
    assert np.allclose(X, X.T, atol=0)
    assert np.min(np.linalg.eigvalsh(X)) >= -1e-12 * np.linalg.norm(X, 2)
    for Xk in its:
        assert np.max(np.linalg.eigvals(A - p.B @ (p.B.T @ Xk)).real) < 0
    for k in range(1, len(its) - 1):
        d = its[k] - its[k + 1]
        assert np.min(np.linalg.eigvalsh(0.5 * (d + d.T))) >= -1e-10 * np.linalg.norm(its[k], 2)
    h = out["res_hist"]
    # quadratic: once the residual is small, the next one is far smaller than linear contraction
    assert h[-1] <= 1e-14 * np.linalg.norm(p.C @ p.C.T)
    ctc = np.linalg.norm(p.C @ p.C.T)
    tail = [i for i in range(len(h) - 1) if h[i] < 1e-2 * h.max() and h[i + 1] > 1e-11 * ctc]
    assert len(tail) >= 3
    ratios = [h[i + 1] / h[i] for i in tail]
    assert all(ratios[j + 1] < ratios[j] for j in range(len(ratios) - 1))  # superlinear
    c0 = h[tail[0] + 1] / h[tail[0]] ** 2
    assert all(h[i + 1] <= 10.0 * c0 * h[i] ** 2 for i in tail)  # quadratic


def test_riccati_residual_zero_at_solution_and_sign():
    """A transposed or sign-flipped term in R(X) would leave a nonzero residual at the
    Hamiltonian solution of a nonsymmetric problem."""
    A, B, C = _nonsym(25, 15)
    Xh = od.hamiltonian_care(A, B, C)
    R = od.riccati_residual(A, B, C, Xh)
    assert np.linalg.norm(R) <= 1e-11 * np.linalg.norm(C.T @ C)
    wrong = A @ Xh + Xh @ A.T - Xh @ B @ B.T @ Xh + C.T @ C
    assert np.linalg.norm(wrong) > 1e-3 * np.linalg.norm(C.T @ C)


def test_lowrank_diff_fro():
    s = ci.Stream(ci.SEED, 16)
    Z = s.normal(50 * 4).reshape(50, 4)
    Y = s.normal(50 * 6).reshape(50, 6)
    d = od.lowrank_diff_fro(Z, Y)
    assert d == pytest.approx(np.linalg.norm(Z @ Z.T - Y @ Y.T), rel=1e-12)


def test_precision_table_roundoffs():
    """Section 1 precision table: the unit roundoffs used for tolerances."""
    g = json.load(open(os.path.join(GOLD, "precision_table.json")))["unit_roundoff"]
    assert 2.0 ** -53 == pytest.approx(g["fp64"], rel=5e-3)
    assert 2.0 ** -24 == pytest.approx(g["fp32"], rel=5e-3)
    assert 2.0 ** -11 == pytest.approx(g["fp16"], rel=5e-3)
    assert 2.0 ** -8 == pytest.approx(g["bf16"], rel=5e-3)
