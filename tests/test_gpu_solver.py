"""GPU parity of the solver entry points (lyap_lradi, care_residual_factor,
care_solve) against the CPU FP64 oracle, through the C ABI."""
import json
import os

import numpy as np
import pytest

import care_inputs as ci
from oracle import dense as od
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


@pytest.fixture(scope="module")
def small():
    prob = ci.config_small_fdm()
    A = prob.A.to_dense()
    X = od.newton_care(A, prob.B, prob.C)["X"]
    return prob, A, X


def dcsr(pb, prob):
    return pb.CSR.from_arrays(prob.A.n, prob.A.rowptr, prob.A.colind, prob.A.val)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 2e-4)])
def test_lyap_lradi_vs_bartels_stewart(pb, small, prec, tol):
    prob, A, X = small
    W = np.hstack([prob.C.T, ci.random_block(prob.n, 2, 61)])
    Xl = od.lyap_bartels_stewart(A.T, W @ W.T)
    Z, info = pb.lyap_lradi(dcsr(pb, prob), W, tol=1e-12 if prec == "fp64" else 1e-6, prec=prec,
                            allow=(0, 5))
    Z = Z.cpu().numpy()
    assert np.linalg.norm(Z @ Z.T - Xl) <= tol * np.linalg.norm(Xl)


def test_lyap_lradi_feedback(pb, small):
    prob, A, X = small
    K = X @ prob.B
    W = np.hstack([prob.C.T, K])
    Ak = A - prob.B @ K.T
    Xl = od.lyap_bartels_stewart(Ak.T, W @ W.T)
    Z, info = pb.lyap_lradi(dcsr(pb, prob), W, B=prob.B, K=K, tol=1e-12, prec="fp64")
    Z = Z.cpu().numpy()
    assert np.linalg.norm(Z @ Z.T - Xl) <= 1e-8 * np.linalg.norm(Xl)


@pytest.mark.parametrize("eta", [0.0, 1e-4])
def test_residual_factor_vs_oracle(pb, small, eta):
    """Algorithm 1 on the same Z: ||R||_F and C+C+^T - C-C-^T against the oracle."""
    prob, A, X = small
    w, V = np.linalg.eigh(X)
    Z = V[:, -8:] * np.sqrt(w[-8:]) + 1e-4 * ci.random_block(prob.n, 8, 62)
    Cp0, Cm0, res0, _ = ol.residual_factor(A, prob.B, prob.C, Z, eta)
    Cp, Cm, res = pb.care_residual_factor(dcsr(pb, prob), prob.B, prob.C, Z, eta)
    Cp, Cm = Cp.cpu().numpy(), Cm.cpu().numpy()
    assert res == pytest.approx(res0, rel=1e-9)
    R0 = Cp0 @ Cp0.T - Cm0 @ Cm0.T
    R1 = Cp @ Cp.T - Cm @ Cm.T
    Rfull = od.riccati_residual(A, prob.B, prob.C, Z @ Z.T)
    assert np.linalg.norm(R1 - R0) <= 1e-9 * np.linalg.norm(Rfull) + 2 * eta * np.abs(np.linalg.eigvalsh(Rfull)).max() * 10


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_care_solve_small_fdm(pb, small, prec):
    """n = 400 convection-diffusion CARE (complex spectrum, m = p = 1): residual <= 1e-12 and
    ||Z Z^T - X*||_F / ||X*||_F <= 1e-8 against Newton + Bartels-Stewart."""
    prob, A, X = small
    Z, info = pb.care_solve(dcsr(pb, prob), prob.B, prob.C, tol=1e-12, prec=prec, r_cap=256)
    Z = Z.cpu().numpy()
    assert info["status"] == "CARE_OK", info
    R = od.riccati_residual(A, prob.B, prob.C, Z @ Z.T)
    assert np.linalg.norm(R) <= 1e-12 * np.linalg.norm(prob.C.T @ prob.C) * 1.5
    assert np.linalg.norm(Z @ Z.T - X) <= 1e-8 * np.linalg.norm(X)
    # the library's factored FP64 residual agrees with the oracle's (Algorithm 1, Householder)
    # on the same Z, at the level of the evaluation error u ||F||^2 / ||C^T C||_F
    res_or = ol.residual_factor(A, prob.B, prob.C, Z, 0.0)[2] / np.linalg.norm(prob.C @ prob.C.T)
    assert abs(info["res_rel_CtC"] - res_or) <= 1e-12


@pytest.mark.parametrize("k,compress", [(0, 0), (1, 0), (2, 0), (0, 1), (1, 1)])
def test_care_solve_dense_conditioning(pb, k, compress):
    """Dense conditioning family (n = 200, m = p = 2) at kappa_2(A) = 10^k, mixed precision
    against the dense FP64 oracle: below the FP32 conditioning threshold the refinement
    reaches relative residual 1e-10 and ||Z Z^T - X*||_F / ||X*||_F <= 1e-8 (for these problems
    ||X B B^T X||_F is up to ~2000 ||C^T C||_F, so FP64 evaluation of the residual bottoms out
    near 1e-11 in this normalisation).  compress = 1 also truncates the +/- correction factors
    in FP32 before Algorithm 2; that truncation is relative to ||X_+-||, not to the correction
    X_+ - X_-, and at kappa = 100 it stalls the refinement near 1e-8 (not tested there)."""
    prob = ci.config_dense_conditioning(k)
    A = prob.A.to_dense()
    X = od.newton_care(A, prob.B, prob.C)["X"]
    # near residual 1e-10 the forward error of these problems can still exceed 1e-8 (to
    # first order X* - Z Z^T = L_cl^{-1}(R(Z Z^T)), L_cl the closed-loop Lyapunov operator
    # at Z Z^T; at kappa = 100 it reaches ~4e-8), so they are refined to 1e-11, where the
    # FP64 evaluation floor may end the run by the stagnation test just above it
    tol = 1e-11
    o = pb.default_options(inner_compress=compress)
    Z, info = pb.care_solve(dcsr(pb, prob), prob.B, prob.C, tol=tol, prec="mixed", r_cap=200, opts=o, allow=(5, 6))
    Z = Z.cpu().numpy()
    err = np.linalg.norm(Z @ Z.T - X) / np.linalg.norm(X)
    Xc = Z @ Z.T
    est = np.linalg.norm(od.lyap_bartels_stewart((A - prob.B @ (prob.B.T @ Xc)).T,
                                                 od.riccati_residual(A, prob.B, prob.C, Xc))) / np.linalg.norm(X)
    assert info["status"] in ("CARE_OK", "CARE_STAGNATED", "CARE_NOT_CONVERGED"), (info, err, est)
    assert info["res_rel_CtC"] <= 1e-10, (info, err, est)
    # the error against the oracle is the one the final residual implies (first-order
    # estimate est, from the oracle's dense Lyapunov solve), and <= 1e-8 once that is small
    assert err <= max(1e-8, 1.5 * est), (info, err, est)


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("k", range(7))
def test_care_solve_conditioning_sweep_dense_direct(pb, k):
    """The Lyapunov-conditioning threshold (Theorem 1; Table 1's experiment, Section
    5.1) on the n = 200 dense family, kappa_2(A) = 10^k, with dense-direct shifted
    solves as Section 5.1 uses, against the oracle's outcome at the same k
    (tests/golden/dense200_sweep.json, written by make_dense200_sweep.py): where the
    oracle's FP32-inner refinement converges (k <= 3) the mixed GPU path reaches
    relative residual 1e-10 and ||Z Z^T - X*||_F / ||X*||_F <= 1e-8; at k = 4 the
    FP32-inner path stalls while FP64 inner solves still reach the oracle's FP64
    level; beyond (k >= 5) neither precision converges, as in the oracle."""
    with open(os.path.join(GOLDEN, "dense200_sweep.json")) as f:
        g = json.load(f)
    o32, o64 = g[f"{k}/fp32"], g[f"{k}/fp64"]
    prob = ci.config_dense_conditioning(k)
    A = prob.A.to_dense()
    X = od.newton_care(A, prob.B, prob.C)["X"]
    o = pb.default_options(krylov=pb.KRYLOV_DENSE_LU)
    Z, info = pb.care_solve(dcsr(pb, prob), prob.B, prob.C, tol=1e-12, prec="mixed", r_cap=600, opts=o,
                            allow=(5, 6, 7, 8))
    Z = Z.cpu().numpy()
    err = np.linalg.norm(Z @ Z.T - X) / np.linalg.norm(X)
    rel = info["res_rel_CtC"]
    if o32["status"] == "ok":
        assert rel <= 1e-10 and err <= 1e-8, (info, err, o32)
    else:
        assert info["status"] != "CARE_OK" and rel > 1e-9, (info, err, o32)
    if k == 4:
        Z64, i64 = pb.care_solve(dcsr(pb, prob), prob.B, prob.C, tol=1e-12, prec="fp64", r_cap=600, opts=o,
                                 allow=(5, 6, 7, 8))
        assert o64["rel_res"] < 1e-9 and i64["res_rel_CtC"] <= 10 * o64["rel_res"], (i64, o64)
    if k >= 5:
        assert o64["status"] != "ok" and o32["status"] != "ok"


def test_care_solve_eigen_aligned_closed_form(pb):
    """P3: Laplacian (no convection) on a 100x100 grid with B, C along analytic modes: the exact
    X* is known; mixed precision reaches it."""
    pr = ci.eigen_aligned_problem(100, 2, [(1, 1), (2, 3), (5, 2)], [0.8, 1.5, 0.3], [2.0, 0.5, 3.0])
    Z, info = pb.care_solve(dcsr(pb, pr), pr.B, pr.C, tol=1e-12, prec="mixed", r_cap=64)
    Z = Z.cpu().numpy()
    x = od.scalar_care(pr.meta["lams"], pr.meta["beta"], pr.meta["gamma"])
    Zx = pr.meta["V"] * np.sqrt(x)
    assert info["status"] == "CARE_OK", info
    assert od.lowrank_diff_fro(Z, Zx) <= 1e-9 * od.lowrank_fro(Zx)


def test_care_solve_eigen_aligned_3d_full_size(pb):
    """P3 at the 3D workload's size: Laplacian on a 100^3 grid (n = 1e6, nnz = 6.94e6) with B, C
    along three analytic modes; the exact X* is known at this size."""
    pr = ci.eigen_aligned_problem(100, 3, [(1, 1, 1), (2, 1, 3), (1, 4, 2)], [0.6, 1.2, 0.4], [1.5, 0.7, 2.5])
    Z, info = pb.care_solve(dcsr(pb, pr), pr.B, pr.C, tol=1e-10, prec="mixed", r_cap=64)
    Z = Z.cpu().numpy()
    x = od.scalar_care(pr.meta["lams"], pr.meta["beta"], pr.meta["gamma"])
    Zx = pr.meta["V"] * np.sqrt(x)
    assert info["status"] == "CARE_OK", info
    assert od.lowrank_diff_fro(Z, Zx) <= 1e-8 * od.lowrank_fro(Zx)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_care_solve_small_fdm_gmres(pb, small, prec):
    """The n = 400 case with restarted GMRES + ILU(0) shifted solves (the paper's
    Section 5.2 solver): residual <= 1e-12 and the dense Newton X* to 1e-8."""
    prob, A, X = small
    o = pb.default_options(krylov=pb.KRYLOV_GMRES)
    Z, info = pb.care_solve(dcsr(pb, prob), prob.B, prob.C, tol=1e-12, prec=prec, r_cap=256, opts=o)
    Z = Z.cpu().numpy()
    assert info["status"] == "CARE_OK", info
    assert np.linalg.norm(Z @ Z.T - X) <= 1e-8 * np.linalg.norm(X)
