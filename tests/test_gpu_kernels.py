"""GPU parity of the kernel-level entry points (SpMM, Gram, SMW shifted solve)
against the CPU oracle, through the C ABI."""
import numpy as np
import scipy.sparse as sp
import pytest

import care_inputs as ci
from oracle import lowrank as ol

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


def _ops(pb, prob):
    A = prob.A
    dA = pb.CSR.from_arrays(A.n, A.rowptr, A.colind, A.val)
    return dA, pb.Operator(dA), A.to_scipy()


@pytest.mark.parametrize("N,b", [(20, 1), (20, 3), (23, 8), (31, 13), (40, 64), (17, 130)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("shift", [0.0, -250.0, complex(-300.0, 900.0)])
def test_spmm_parity(pb, N, b, dtype, shift):
    """Y = (A^T + p I) X element by element against the oracle, ragged widths, complex shifts,
    and widths above one kernel chunk (130 reals)."""
    prob = ci.config_small_fdm(N)
    dA, op, As = _ops(pb, prob)
    cplx = isinstance(shift, complex)
    if cplx and b > 64:
        b = 64
    X = ci.random_block(prob.n, b, 31)
    if cplx:
        X = X + 1j * ci.random_block(prob.n, b, 32)
    ref = ol.shifted_operator_apply(As, shift, X)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if cplx:
        Xt = torch.tensor(X, dtype=torch.complex128 if dtype == "f64" else torch.complex64, device="cuda")
    else:
        Xt = torch.tensor(X, dtype=tdt, device="cuda")
    Y = pb.spmm(op, Xt, shift).cpu().numpy().astype(np.complex128 if cplx else np.float64)
    # rounding bound: |A^T| |X| + |p| |X| with gamma_{k} of the precision (k <= 6 terms); the FP32
    # operator is applied as sum_j a_ij (x_j - x_i) + (s_i + p) x_i, which adds (sum_j |a_ij|) |x_i|
    rowabs = np.asarray(abs(As.T).sum(axis=1)).ravel()[:, None]
    bound = np.abs(As.T) @ np.abs(X) + abs(shift) * np.abs(X) + rowabs * np.abs(X)
    u = U64 if dtype == "f64" else U32
    # FP32 path also rounds A and X to FP32 (two more roundings per term)
    k = 8 if dtype == "f64" else 12
    assert np.all(np.abs(Y - ref) <= k * u * bound + 1e-300)


def test_spmm_large_ragged(pb):
    """n = 250,000 operator (the 500x500 grid) on a 10-column block: sampled rows."""
    prob = ci.config_fdm2d(500, 1, 1)
    dA, op, As = _ops(pb, prob)
    X = ci.random_block(prob.n, 10, 33)
    Y = pb.spmm(op, torch.tensor(X, dtype=torch.float32, device="cuda"), -1000.0).cpu().numpy()
    rows = np.random.default_rng(0).choice(prob.n, 2000, replace=False)
    ref = (As.T[rows] @ X) - 1000.0 * X[rows]
    rowabs = np.asarray(abs(As.T[rows]).sum(axis=1)).ravel()[:, None]
    bound = np.abs(As.T[rows]) @ np.abs(X) + 1000.0 * np.abs(X[rows]) + rowabs * np.abs(X[rows])
    assert np.all(np.abs(Y[rows] - ref) <= 12 * U32 * bound)


@pytest.mark.parametrize("n,a,b", [(1, 1, 1), (100, 3, 5), (1000, 64, 64), (5003, 65, 7), (20000, 130, 200)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gram_parity(pb, n, a, b, dtype):
    X = ci.random_block(n, a, 41)
    Y = ci.random_block(n, b, 42)
    ref = ol.gram(X, Y)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    G = pb.gram(torch.tensor(X, dtype=tdt, device="cuda"), torch.tensor(Y, dtype=tdt, device="cuda")).cpu().numpy()
    if dtype == "f32":
        Xr, Yr = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
        ref = ol.gram(Xr, Yr)
    bound = np.abs(X).T @ np.abs(Y)
    u = U64 if dtype == "f64" else U32
    assert np.all(np.abs(G - ref) <= (n + 2) * u * bound + 1e-300)


@pytest.mark.parametrize("n,a", [(100, 1), (1000, 64), (5003, 65), (20000, 130), (3000, 257)])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_gram_symmetric_path(pb, n, a, dtype):
    """X^T X with Y the same buffer computes only the tiles on and above the diagonal and
    mirrors them: exactly symmetric, and like the general product on a copy (whose
    split-K slicing, hence summation order, may differ) within the rounding bound of the
    oracle's product."""
    tdt = torch.float64 if dtype == "f64" else torch.float32
    X = torch.tensor(ci.random_block(n, a, 44), dtype=tdt, device="cuda")
    Gs = pb.gram(X, X).cpu().numpy()
    Gg = pb.gram(X, X.clone()).cpu().numpy()
    assert np.array_equal(Gs, Gs.T)
    Xh = X.double().cpu().numpy()
    u = U64 if dtype == "f64" else U32
    bound = (n + 2) * u * (np.abs(Xh).T @ np.abs(Xh))
    ref = ol.gram(Xh, Xh)
    assert np.all(np.abs(Gs - ref) <= bound)
    assert np.all(np.abs(Gg - ref) <= bound)


def test_gram_deterministic(pb):
    X = torch.tensor(ci.random_block(300000, 12, 43), dtype=torch.float32, device="cuda")
    g1 = pb.gram(X, X)
    g2 = pb.gram(X, X)
    assert torch.equal(g1, g2)


@pytest.mark.parametrize("krylov", ["bicgstab", "gmres"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
@pytest.mark.parametrize("shift", [-400.0, complex(-900.0, 1500.0)])
@pytest.mark.parametrize("feedback", [False, True])
def test_shifted_solve_parity(pb, krylov, prec, tol, shift, feedback):
    """SMW + block Krylov (BiCGStab, or restarted GMRES as in Section 5.2) vs the
    oracle's sparse-LU SMW solve (Section 4); the solution error is bounded by the
    per-column relative residual tolerance times the conditioning of M_p."""
    prob = ci.config_small_fdm()
    dA, op, As = _ops(pb, prob)
    W = ci.random_block(prob.n, 3, 51)
    K = 1e-2 * ci.random_block(prob.n, 1, 52) if feedback else None
    B = prob.B if feedback else None
    ref = ol.smw_solve(ol.ShiftedSolver(As), B, K, shift, W)
    o = pb.default_options(krylov=pb.KRYLOV_GMRES if krylov == "gmres" else pb.KRYLOV_BICGSTAB)
    V, iters = pb.shifted_solve(op, W, shift, B=B, K=K, prec=prec, opts=o)
    V = V.cpu().numpy()
    assert iters > 0
    assert np.linalg.norm(V - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("precond", ["none", "jacobi", "ilu0"])
@pytest.mark.parametrize("shift", [-150.0, complex(-1500.0, 2500.0)])
def test_gmres_restarts_and_preconditioners(pb, precond, shift):
    """GMRES with a short restart (several cycles) and each preconditioner reaches
    the FP64 tolerance on the 100x100 operator; per-column residuals are checked
    against the operator itself."""
    prob = ci.config_fdm2d(100, 2, 2)
    dA, op, As = _ops(pb, prob)
    W = ci.random_block(prob.n, 5, 54)
    pc = {"none": pb.PRECOND_NONE, "jacobi": pb.PRECOND_JACOBI, "ilu0": pb.PRECOND_ILU0}[precond]
    o = pb.default_options(krylov=pb.KRYLOV_GMRES, gmres_restart_hi=8, precond=pc, krylov_maxit_hi=4000)
    V, it = pb.shifted_solve(op, W, shift, prec="fp64", opts=o)
    V = V.cpu().numpy()
    M = (As + shift * sp.eye(prob.n)).T
    R = W - M @ V
    assert np.all(np.linalg.norm(R, axis=0) <= 2e-10 * np.linalg.norm(W, axis=0))
    if precond == "none":
        assert it > 8  # restarted at least once


@pytest.mark.parametrize("shift", [-150.0, -2000.0, complex(-1500.0, 2500.0)])
def test_ilu0_preconditioner_parity_and_gain(pb, shift):
    """ILU(0) (fixed-point factorisation, Jacobi triangular sweeps) gives the same solution
    as the unpreconditioned solve and needs fewer iterations on the 100x100 operator."""
    prob = ci.config_fdm2d(100, 2, 2)
    dA, op, As = _ops(pb, prob)
    W = ci.random_block(prob.n, 4, 53)
    ref = ol.smw_solve(ol.ShiftedSolver(As), None, None, shift, W)
    its = {}
    for name, pc in (("none", pb.PRECOND_NONE), ("ilu0", pb.PRECOND_ILU0)):
        o = pb.default_options(precond=pc, krylov_maxit_hi=2000)
        V, it = pb.shifted_solve(op, W, shift, prec="fp64", opts=o)
        V = V.cpu().numpy()
        its[name] = it
        assert np.linalg.norm(V - ref) <= 1e-8 * np.linalg.norm(ref), name
    assert its["ilu0"] < 0.6 * its["none"], its


def test_spmm_fp32_difference_form_smooth_accuracy(pb):
    """On a smooth block the FP32 operator keeps FP32 relative accuracy in A^T x (the
    difference form avoids the ~400x cancellation of the 1/h^2 stencil)."""
    prob = ci.config_fdm2d(500, 1, 1)
    dA, op, As = _ops(pb, prob)
    v, lam = ci.laplacian_mode(500, 2, (1, 1))
    X = np.stack([v, 2 * v], 1)
    Y = pb.spmm(op, torch.tensor(X, dtype=torch.float32, device="cuda"), 0.0).cpu().numpy().astype(np.float64)
    ref = As.T @ X.astype(np.float32).astype(np.float64)
    assert np.linalg.norm(Y - ref) <= 50 * U32 * np.linalg.norm(ref)


def test_autotune_picks_valid_config_and_keeps_parity(pb):
    """The autotuner returns one of its candidate configurations, and a shifted solve with
    the tuned options still matches the oracle."""
    prob = ci.config_fdm2d(100, 2, 2)
    dA, op, As = _ops(pb, prob)
    import time
    t0 = time.perf_counter()
    o, best_ms = pb.autotune(op, 2, 4, prec="fp64")
    t_first = time.perf_counter() - t0
    assert best_ms > 0
    assert o.krylov in (pb.KRYLOV_BICGSTAB, pb.KRYLOV_GMRES)
    assert o.krylov_chunk in (32, 64) and o.tri_sweeps in (1, 2, 3)
    assert o.precond in (pb.PRECOND_NONE, pb.PRECOND_ILU0, pb.PRECOND_ILU0_EXACT)
    vpt, ctas, blk = pb.launch_shape()
    assert len(vpt) == 5 and all(v in (1, 2, 4) for v in vpt) and ctas in (4, 8) and blk in (0, 1)
    W = ci.random_block(prob.n, 4, 54)
    ref = ol.smw_solve(ol.ShiftedSolver(As), None, None, -500.0, W)
    V, _ = pb.shifted_solve(op, W, -500.0, prec="fp64", opts=o)
    assert np.linalg.norm(V.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    # the choice is cached per operator shape: the same answer without timing again
    t0 = time.perf_counter()
    o2, best2 = pb.autotune(op, 2, 4, prec="fp64")
    t_second = time.perf_counter() - t0
    assert (o2.krylov, o2.precond, o2.tri_sweeps, o2.krylov_chunk, best2) == (
        o.krylov, o.precond, o.tri_sweeps, o.krylov_chunk, best_ms)
    assert pb.launch_shape() == (vpt, ctas, blk)
    assert t_second < 0.5 * t_first
