"""Tensor-core (tcgen05 + TMA) products through the C ABI: the FP64-accurate
sliced Gram and X S products against exact integer arithmetic and against the
FP64 error bound, the TF32 / BF16 Grams against their input-rounding bound, and
the solver with every FP64 product on the tensor cores against the dense
Newton oracle."""
import numpy as np
import pytest

import care_inputs as ci
from oracle import dense as od

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    if not m.tc_available():
        pytest.skip("tensor-core path needs sm_103")
    return m


def _dev(A, dt=torch.float64):
    return torch.tensor(np.ascontiguousarray(A), dtype=dt, device="cuda")


@pytest.mark.parametrize("n,a,b,sym", [(3000, 70, 90, False), (5000, 130, 130, True), (777, 1, 200, False),
                                      (40000, 200, 64, False), (33000, 257, 257, True)])
def test_gram_f64_exact_on_integers(pb, n, a, b, sym):
    """Integer entries of at most 11 bits: every slice, product and chunk sum is exact,
    so the sliced tensor-core Gram equals the exact product bit for bit (several
    128-row chunks, ragged tiles, split rows, and the mirrored symmetric form; the
    33000-row case crosses a 32768-row slab)."""
    rng = np.random.default_rng(n + a)
    X = rng.integers(-1024, 1025, size=(n, a)).astype(np.float64)
    Y = X if sym else rng.integers(-1024, 1025, size=(n, b)).astype(np.float64)
    exact = (X.astype(np.int64).T @ Y.astype(np.int64)).astype(np.float64)
    Xd = _dev(X)
    G = pb.gram_tc(Xd, Xd if sym else _dev(Y), "f64").cpu().numpy()
    assert np.array_equal(G, exact)
    if sym:
        assert np.array_equal(G, G.T)


def _fp64_bound(X, Y):
    """(n+2) u |X|^T |Y| plus the 49-bit input rounding relative to each column's
    power-of-two scale M (|dx| <= 2^-50 M_i) and the dropped / tail terms (< 2^-48 M_i M_j n)."""
    n = X.shape[0]
    Mx = 2.0 ** np.ceil(np.log2(np.maximum(np.abs(X).max(axis=0), 1e-300)))
    My = 2.0 ** np.ceil(np.log2(np.maximum(np.abs(Y).max(axis=0), 1e-300)))
    ax, ay = np.abs(X), np.abs(Y)
    return ((n + 2) * U64 * (ax.T @ ay) + 2.0 ** -49 * (Mx[:, None] * ay.sum(0)[None, :] + ax.sum(0)[:, None] *
                                                         My[None, :]) + n * 2.0 ** -47 * Mx[:, None] * My[None, :])


@pytest.mark.parametrize("n,a,b,sym,kind", [(20000, 96, 160, False, "normal"), (50000, 300, 300, True, "normal"),
                                            (12345, 65, 129, False, "decaying"), (70000, 128, 64, False, "scaled")])
def test_gram_f64_within_fp64_bound(pb, n, a, b, sym, kind):
    """Random data (normal, rows decaying over 8 decades, columns scaled over 12 decades):
    elementwise within the FP64 bound, and normwise as close to the exact product as
    the FP64 CUDA-core Gram."""
    rng = np.random.default_rng(a * b)
    X = rng.standard_normal((n, a))
    Y = X if sym else rng.standard_normal((n, b))
    if kind == "decaying":
        w = np.logspace(0, -8, n)[:, None]
        X, Y = X * w, Y * w
    if kind == "scaled":
        X = X * np.logspace(-6, 6, a)[None, :]
        Y = Y * np.logspace(3, -3, b)[None, :]
    ref = X.T @ Y
    Xd = _dev(X)
    G = pb.gram_tc(Xd, Xd if sym else _dev(Y), "f64").cpu().numpy()
    assert np.all(np.abs(G - ref) <= _fp64_bound(X, Y))
    Gs = pb.gram(Xd, Xd if sym else _dev(Y)).cpu().numpy()
    nrm = np.linalg.norm(np.abs(X).T @ np.abs(Y))
    assert np.linalg.norm(G - ref) <= max(4 * np.linalg.norm(Gs - ref), 1e-15 * nrm)


@pytest.mark.parametrize("n,a,b,beta", [(1000, 64, 64, 0.0), (40000, 300, 130, 0.5), (130, 1000, 65, -1.0),
                                        (70001, 77, 512, 0.0)])
def test_gemm_ts_f64_tc(pb, n, a, b, beta):
    """Y = alpha X S + beta Y on the tensor cores against FP64, elementwise within
    (a+2) u |alpha||X||S| + u |beta Y| + the row-scale input rounding."""
    rng = np.random.default_rng(n + b)
    X = rng.standard_normal((n, a)) * np.logspace(0, -3, a)[None, :]
    S = rng.standard_normal((a, b))
    Y0 = rng.standard_normal((n, b))
    alpha = -1.5
    ref = alpha * (X @ S) + beta * Y0
    Yd = _dev(Y0)
    out = pb.gemm_ts(_dev(X), _dev(S), alpha, beta, Yd, tc=True).cpu().numpy()
    Mx = 2.0 ** np.ceil(np.log2(np.abs(X).max(axis=1)))
    Ms = 2.0 ** np.ceil(np.log2(np.abs(S).max(axis=0)))
    bound = abs(alpha) * ((a + 2) * U64 * (np.abs(X) @ np.abs(S)) + 2.0 ** -49 * (
        Mx[:, None] * np.abs(S).sum(0)[None, :] + np.abs(X).sum(1)[:, None] * Ms[None, :]) +
        a * 2.0 ** -47 * Mx[:, None] * Ms[None, :]) + 2 * U64 * np.abs(beta * Y0) + 2 * U64 * np.abs(ref)
    assert np.all(np.abs(out - ref) <= bound)
    # the CUDA-core path of the same entry point agrees within the same bound
    cc = pb.gemm_ts(_dev(X), _dev(S), alpha, beta, _dev(Y0), tc=False).cpu().numpy()
    assert np.all(np.abs(cc - ref) <= bound)


def test_gemm_ts_exact_on_integers(pb):
    rng = np.random.default_rng(5)
    X = rng.integers(-1000, 1001, size=(5000, 200)).astype(np.float64)
    S = rng.integers(-1000, 1001, size=(200, 96)).astype(np.float64)
    exact = (X.astype(np.int64) @ S.astype(np.int64)).astype(np.float64)
    out = pb.gemm_ts(_dev(X), _dev(S), 1.0, 0.0, None, tc=True).cpu().numpy()
    assert np.array_equal(out, exact)


@pytest.mark.parametrize("mode,u_in", [("tf32", 2.0 ** -10), ("bf16", 2.0 ** -8)])
@pytest.mark.parametrize("n,a,b,sym", [(30000, 64, 64, True), (9999, 100, 33, False)])
def test_gram_lowp(pb, mode, u_in, n, a, b, sym):
    """TF32 / BF16 inputs, FP32 accumulation: within 2 u_in |X|^T|Y| + n u_32 |X|^T|Y|."""
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, a)).astype(np.float32)
    Y = X if sym else rng.standard_normal((n, b)).astype(np.float32)
    Xd = _dev(X, torch.float32)
    G = pb.gram_tc(Xd, Xd if sym else _dev(Y, torch.float32), mode).cpu().numpy()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = X64.T @ Y64
    bound = (2 * u_in + n * 2.0 ** -23) * (np.abs(X64).T @ np.abs(Y64))
    assert np.all(np.abs(G - ref) <= bound)
    # and it is really low precision: TF32/BF16 rounding is visible
    assert np.abs(G - ref).max() > 1e-6 * np.abs(ref).max()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_care_solve_with_every_fp64_product_on_tensor_cores(pb, prec):
    """n = 400 convection-diffusion CARE with every FP64 product of the solver on the
    tensor cores (Algorithms 1-2 and, for prec = fp64, the FP64 LR-ADI): residual <= 2e-11
    and ||ZZ^T - X*|| / ||X*|| <= 1e-8 against Newton + Bartels-Stewart.  The sliced
    products' error is relative to each operand column's largest entry (56-bit fixed
    point), not to every entry as in FP64 arithmetic; on this problem, whose factor
    columns are localised modes, that puts the refinement's floor near 7e-12 with the
    FP64 inner solves also on the tensor cores (1e-13 on the CUDA cores), still two
    orders below the 1e-10 target."""
    prob = ci.config_small_fdm()
    X = od.newton_care(prob.A.to_dense(), prob.B, prob.C)["X"]
    A = pb.CSR.from_arrays(prob.A.n, prob.A.rowptr, prob.A.colind, prob.A.val)
    pb.set_tensor_cores(2)
    try:
        Z, info = pb.care_solve(A, prob.B, prob.C, tol=1e-11, prec=prec, r_cap=256, allow=(6,))
    finally:
        pb.set_tensor_cores(1)
    # at the floor the 0.999 stagnation test may end the run just above 1e-11
    assert info["status"] in ("CARE_OK", "CARE_STAGNATED") and info["res_rel_CtC"] <= 2e-11, info
    assert info["tc_calls"][0] > 0
    Z = Z.cpu().numpy()
    assert np.linalg.norm(Z @ Z.T - X) <= 1e-8 * np.linalg.norm(X)
    R = od.riccati_residual(prob.A.to_dense(), prob.B, prob.C, Z @ Z.T)
    assert np.linalg.norm(R) <= 2e-11 * np.linalg.norm(prob.C.T @ prob.C) * 1.5


@pytest.mark.parametrize("prec", ["mixed_tf32", "mixed_bf16"])
def test_care_solve_lowp_shift_grams(pb, prec):
    """CARE_PREC_MIXED_TF32 / _BF16: the Grams of the shift generation run on the tensor
    cores in TF32 / BF16; the refinement still reaches residual 1e-12 and the oracle's
    X* to 1e-8 (the shifts only steer the convergence of LR-ADI)."""
    prob = ci.config_small_fdm()
    X = od.newton_care(prob.A.to_dense(), prob.B, prob.C)["X"]
    A = pb.CSR.from_arrays(prob.A.n, prob.A.rowptr, prob.A.colind, prob.A.val)
    Z, info = pb.care_solve(A, prob.B, prob.C, tol=1e-12, prec=prec, r_cap=256)
    assert info["status"] == "CARE_OK", info
    assert info["lowp_gram_calls"] > 0
    Z = Z.cpu().numpy()
    assert np.linalg.norm(Z @ Z.T - X) <= 1e-8 * np.linalg.norm(X)


@pytest.mark.parametrize("n,a,b,sym", [(4000, 96, 80, False), (40000, 130, 130, True)])
def test_gram_f32acc_exact_on_integers_and_bound(pb, n, a, b, sym):
    """FP32 operands, four slices (28-bit fixed point), all ten pairs exact: integer
    entries of up to 11 bits give the exact product; random data stays within the
    input-rounding bound 2^-29 relative to each column's power-of-two scale plus the
    dropped pairs (< 2^-28 M_i M_j per term)."""
    rng = np.random.default_rng(n + 3)
    Xi = rng.integers(-1024, 1025, size=(n, a)).astype(np.float32)
    Yi = Xi if sym else rng.integers(-1024, 1025, size=(n, b)).astype(np.float32)
    exact = (Xi.astype(np.int64).T @ Yi.astype(np.int64)).astype(np.float64)
    Xd = _dev(Xi, torch.float32)
    G = pb.gram_tc(Xd, Xd if sym else _dev(Yi, torch.float32), "f32").cpu().numpy()
    assert np.array_equal(G, exact)
    X = (rng.standard_normal((n, a)) * np.logspace(0, -2, a)[None, :]).astype(np.float32)
    Y = X if sym else rng.standard_normal((n, b)).astype(np.float32)
    Xd = _dev(X, torch.float32)
    G = pb.gram_tc(Xd, Xd if sym else _dev(Y, torch.float32), "f32").cpu().numpy()
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = X64.T @ Y64
    Mx = 2.0 ** np.ceil(np.log2(np.abs(X64).max(axis=0)))
    My = 2.0 ** np.ceil(np.log2(np.abs(Y64).max(axis=0)))
    bound = (2.0 ** -28 * (Mx[:, None] * np.abs(Y64).sum(0)[None, :] + np.abs(X64).sum(0)[:, None] * My[None, :]) +
             n * 2.0 ** -27 * Mx[:, None] * My[None, :] + 4 * U64 * np.abs(ref))
    assert np.all(np.abs(G - ref) <= bound)


def test_gemm_ts_f32acc(pb):
    rng = np.random.default_rng(11)
    n, a, b = 50000, 300, 96
    X = rng.standard_normal((n, a)).astype(np.float32)
    S = rng.standard_normal((a, b))
    Y0 = rng.standard_normal((n, b)).astype(np.float32)
    out = pb.gemm_ts(_dev(X, torch.float32), _dev(S), 0.5, -1.0, _dev(Y0, torch.float32), tc=True).cpu().numpy()
    X64 = X.astype(np.float64)
    ref = 0.5 * (X64 @ S) - Y0.astype(np.float64)
    Mx = 2.0 ** np.ceil(np.log2(np.abs(X64).max(axis=1)))
    Ms = 2.0 ** np.ceil(np.log2(np.abs(S).max(axis=0)))
    bound = 0.5 * (2.0 ** -28 * (Mx[:, None] * np.abs(S).sum(0)[None, :] + np.abs(X64).sum(1)[:, None] * Ms[None, :])
                   + a * 2.0 ** -27 * Mx[:, None] * Ms[None, :]) + 2.0 ** -23 * (np.abs(ref) + np.abs(Y0))
    assert np.all(np.abs(out - ref) <= bound)
