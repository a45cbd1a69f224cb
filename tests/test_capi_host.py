"""C-ABI library checks that need no GPU: it loads, exports every declared symbol,
and its host small-dense routines agree with LAPACK (via NumPy)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2607_14742_b300 as pb

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "care_b300.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted({n for n in names if n not in ("if", "while", "for", "return", "sizeof")})


def test_library_loads_and_exports_every_declared_symbol():
    L = pb.lib()
    names = declared_functions()
    assert "care_solve" in names and "lyap_lradi" in names and "care_residual_factor" in names
    for name in names:
        assert hasattr(L, name), name
        assert ctypes.cast(getattr(L, name), ctypes.c_void_p).value


def test_status_strings_and_defaults():
    names = ["CARE_OK", "CARE_ERR_INVALID_ARG", "CARE_ERR_CUDA", "CARE_ERR_WORKSPACE", "CARE_ERR_RANK_CAPACITY",
             "CARE_NOT_CONVERGED", "CARE_STAGNATED", "CARE_INNER_FAILED", "CARE_UNSTABLE", "CARE_NONFINITE",
             "CARE_ERR_SMALL_DENSE", "CARE_TIMEOUT"]
    for code, name in enumerate(names):
        assert pb.status_string(code) == name
    o = pb.default_options()
    # the library's own defaults beyond the paper's: GMRES restarts (Section 5.2), the joint
    # FP64 compression of the FP32 correction factors, BiCGStab + sweep ILU(0)
    assert (o.gmres_restart_lo, o.gmres_restart_hi) == (30, 50)
    assert o.inner_compress == 2
    assert (o.krylov, o.precond) == (pb.KRYLOV_BICGSTAB, pb.PRECOND_ILU0)
    # Section 5 parameter list
    assert (o.kmax, o.jmax) == (20, 50)
    assert o.eta_r_rel == 1e-4 and o.eta_s_mult == 10.0
    assert o.tau_L_lo == 1e-5 and o.tau_L_hi == 1e-12
    assert o.krylov_tol_lo == 1e-5 and o.krylov_tol_hi == 1e-10
    assert (o.krylov_maxit_lo, o.krylov_maxit_hi) == (100, 200)
    assert o.stag_ratio == 0.999
    assert "sm_103a" in pb.version()


@pytest.mark.parametrize("n", [1, 2, 3, 7, 31, 64, 150, 517])
def test_host_symeig_matches_lapack(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    A = M + M.T
    w, V = pb.host_symeig(A)
    wr = np.linalg.eigvalsh(A)
    scale = max(1.0, np.abs(wr).max())
    assert np.abs(w - wr).max() <= 1e-13 * scale * n
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(A @ V - V * w).max() <= 1e-13 * scale * n


@pytest.mark.parametrize("n", [5, 37, 150, 333])
def test_host_symeig_outside_selects_the_same_eigenpairs(n):
    """Eigenvectors formed only for eigenvalues outside (lo, hi), as Algorithms 1-2 request
    them: the same eigenvalues as the full decomposition, the selected columns agree with the
    full eigenvectors up to sign, the others are zero (sizes cover several 16-column blocks
    and a ragged last block)."""
    rng = np.random.default_rng(100 + n)
    M = rng.standard_normal((n, n))
    A = M + M.T
    w, V = pb.host_symeig(A)
    lo, hi = np.quantile(w, 0.2), np.quantile(w, 0.7)
    ws, Vs = pb.host_symeig_outside(A, lo, hi)
    assert np.array_equal(ws, w)
    keep = (w <= lo) | (w >= hi)
    assert np.all(Vs[:, ~keep] == 0.0)
    sgn = np.sign(np.sum(V[:, keep] * Vs[:, keep], axis=0))
    assert np.all(sgn != 0)
    assert np.abs(Vs[:, keep] - V[:, keep] * sgn).max() <= 1e-12
    scale = max(1.0, np.abs(w).max())
    assert np.abs(A @ Vs[:, keep] - Vs[:, keep] * w[keep]).max() <= 1e-13 * scale * n
    # nothing selected / everything selected
    w0, V0 = pb.host_symeig_outside(A, -np.inf, np.inf)
    assert np.array_equal(w0, w) and np.all(V0 == 0.0)
    w1, V1 = pb.host_symeig_outside(A, np.inf, -np.inf)
    assert np.abs(np.abs(np.sum(V1 * V, axis=0)) - 1.0).max() <= 1e-12


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (7, 5, 3), (130, 67, 301), (257, 257, 1000)])
def test_host_gemm_nt(m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, k))
    B = rng.standard_normal((n, k))
    d = rng.choice([-1.0, 1.0, 0.5], size=k)
    bound = k * 2.0 ** -52 * (np.abs(A) @ np.abs(B).T)
    assert np.all(np.abs(pb.host_gemm_nt(A, B) - A @ B.T) <= 2 * bound)
    assert np.all(np.abs(pb.host_gemm_nt(A, B, d) - (A * d) @ B.T) <= 2 * bound)
    if m == n:
        S = pb.host_gemm_nt(A, A, d, sym=True)
        assert np.array_equal(S, S.T)
        assert np.all(np.abs(S - (A * d) @ A.T) <= 2 * k * 2.0 ** -52 * (np.abs(A) @ np.abs(A).T))


@pytest.mark.parametrize("n", [1, 5, 64, 200, 700])
def test_host_cholesky_and_upper_inverse(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    G = M @ M.T + n * np.eye(n)
    R = pb.host_cholesky_upper(G)
    assert np.allclose(np.tril(R, -1), 0.0)
    assert np.abs(R.T @ R - G).max() <= 1e-13 * np.abs(G).max() * n
    assert np.allclose(R, np.linalg.cholesky(G).T, rtol=0, atol=1e-12 * np.sqrt(np.abs(G).max()) * n)
    Ri = pb.host_upper_inverse(R)
    assert np.allclose(np.tril(Ri, -1), 0.0)
    assert np.abs(R @ Ri - np.eye(n)).max() <= 1e-12 * n
    with pytest.raises(pb.CareError):
        pb.host_cholesky_upper(-np.eye(3))


@pytest.mark.parametrize("c,rank", [(1, 1), (9, 4), (150, 150), (300, 211)])
def test_host_pivoted_cholesky_rank_revealing(c, rank):
    """G = X^T X with X of rank r: the pivoted factor has rank r, upper triangular
    in pivot order, reproduces G, and the pivots are the largest Schur diagonals."""
    rng = np.random.default_rng(c * 7 + rank)
    X = rng.standard_normal((c + 50, rank)) @ rng.standard_normal((rank, c))
    G = X.T @ X
    piv, R = pb.host_pivoted_cholesky(G, 1e-10 * np.abs(G).max())
    assert len(piv) == rank and len(set(piv.tolist())) == rank
    assert np.abs(R.T @ R - G).max() <= 1e-9 * np.abs(G).max()
    Rp = R[:, piv]
    assert np.allclose(np.tril(Rp, -1), 0.0)
    assert np.all(np.diag(Rp) > 0) and np.all(np.diff(np.diag(Rp)) <= 1e-9 * Rp[0, 0])
    assert piv[0] == np.argmax(np.diag(G))
    p2, R2 = pb.host_pivoted_cholesky(G, 0.0, max_rank=3)
    assert len(p2) == min(3, rank) and np.array_equal(p2, piv[:len(p2)])


@pytest.mark.parametrize("case", ["wide", "rank_deficient", "clustered", "clustered_large", "small", "zero",
                                  "decaying"])
def test_host_sym_lmax(case):
    """Largest eigenvalue as LR-ADI's stopping test needs it, against LAPACK: within the
    routine's residual bound (1e-10 relative; clustered leading eigenvalues may return
    any member of the cluster within that bound)."""
    rng = np.random.default_rng(len(case))
    if case == "wide":
        W = rng.standard_normal((3000, 700)); G = W.T @ W
    elif case == "rank_deficient":
        W = rng.standard_normal((400, 150)) @ rng.standard_normal((150, 900)); G = W.T @ W
    elif case == "clustered":
        Q, _ = np.linalg.qr(rng.standard_normal((300, 300)))
        d = np.concatenate([np.full(5, 7.0), 7.0 - 1e-9 * np.arange(5), rng.uniform(0, 6.9, 290)])
        G = (Q * d) @ Q.T
    elif case == "small":
        W = rng.standard_normal((50, 40)); G = W.T @ W
    elif case == "clustered_large":
        Q, _ = np.linalg.qr(rng.standard_normal((900, 900)))
        d = np.concatenate([np.full(5, 7.0), 7.0 - 1e-9 * np.arange(5), rng.uniform(0, 6.9, 890)])
        G = (Q * d) @ Q.T
    elif case == "zero":
        G = np.zeros((800, 800))
    else:
        Q, _ = np.linalg.qr(rng.standard_normal((800, 800)))
        G = (Q * np.logspace(0, -14, 800)) @ Q.T
    ref = np.linalg.eigvalsh(G)[-1]
    got = pb.host_sym_lmax(G)
    assert got <= ref * (1 + 1e-12) + 1e-300
    assert abs(got - ref) <= 1e-10 * max(abs(ref), 1e-300) + 1e-300, (got, ref)


def test_host_symeig_degenerate():
    w, V = pb.host_symeig(np.eye(6))
    assert np.allclose(w, 1.0) and np.allclose(V.T @ V, np.eye(6))
    w, _ = pb.host_symeig(np.zeros((3, 3)))
    assert np.all(w == 0)
    # clustered spectrum with a rank-2 perturbation
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    d = np.concatenate([np.full(20, 1.0), np.full(18, 1.0 + 1e-12), [5.0, -3.0]])
    A = (Q * d) @ Q.T
    w, V = pb.host_symeig(A)
    assert np.abs(np.sort(d) - w).max() < 1e-13 * 5 * 40
    assert np.abs(V.T @ V - np.eye(40)).max() < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 9, 33, 64])
def test_host_eigvals_matches_lapack(n):
    rng = np.random.default_rng(100 + n)
    M = rng.standard_normal((n, n))
    ev = pb.host_eigvals(M)
    er = np.linalg.eigvals(M)
    scale = max(1.0, np.abs(er).max())
    # same multiset: greedy matching
    left = list(er)
    for e in ev:
        k = int(np.argmin(np.abs(np.array(left) - e)))
        assert abs(left[k] - e) <= 1e-10 * scale
        left.pop(k)


def test_host_eigvals_structured():
    # companion-like and rotation blocks (complex pairs), triangular (already Schur)
    R = np.array([[0.0, -2.0], [2.0, 0.0]])
    ev = np.sort_complex(pb.host_eigvals(R))
    assert np.allclose(ev, [-2j, 2j])
    T = np.triu(np.arange(1.0, 26.0).reshape(5, 5))
    assert np.allclose(np.sort(pb.host_eigvals(T).real), np.sort(np.diag(T)))


def test_entry_points_reject_invalid_arguments_before_any_device_work():
    """Every entry point checks its arguments first and returns CARE_ERR_INVALID_ARG
    (status 1) without touching a device, so these calls are safe on a host with no GPU."""
    import ctypes as ct
    L = pb.lib()
    INVALID = 1
    sz = ct.c_size_t(0)
    op0 = pb.op_t()
    bad_csr = pb.csr_t(-1, 0, None, None, None)
    ok_csr = pb.csr_t(4, 4, 16, 16, 16)  # never dereferenced: another argument is invalid
    o = pb.default_options()
    dummy = ct.c_void_p(256)
    cases = {
        "op_size n<0": L.care_op_size(-1, 0, ct.byref(sz)),
        "op_size null": L.care_op_size(4, 3, None),
        "op_prepare null A": L.care_op_prepare(None, dummy, 0, None, ct.byref(op0)),
        "op_prepare n<0": L.care_op_prepare(ct.byref(bad_csr), dummy, 0, None, ct.byref(op0)),
        "spmm dtype": L.care_spmm(ct.byref(op0), 2, 0, 0.0, 0.0, None, 4, 4, None, 4, None),
        "spmm real with imaginary shift": L.care_spmm(ct.byref(op0), 0, 0, 0.0, 1.0, None, 4, 4, None, 4, None),
        "gram n<0": L.care_gram(0, -1, 2, 2, dummy, 2, dummy, 2, dummy, 2, dummy, 1024, None),
        "gram dtype": L.care_gram(3, 10, 2, 2, dummy, 2, dummy, 2, dummy, 2, dummy, 1024, None),
        "gram ldx<a": L.care_gram(0, 10, 3, 2, dummy, 2, dummy, 2, dummy, 2, dummy, 1024, None),
        "gram null G": L.care_gram(0, 10, 2, 2, dummy, 2, dummy, 2, None, 2, dummy, 1024, None),
        "gram_noalloc over limit": L.care_gram_noalloc(0, 10, 1100, 1000, dummy, 1100, dummy, 1000, dummy, 1000,
                                                       None),
        "shifted ws null op": L.care_shifted_solve_workspace_size(None, 1, 2, 1, ct.byref(o), ct.byref(sz)),
        "workspace n<0": L.care_workspace_size(-1, 0, 1, 1, 8, 1, ct.byref(o), ct.byref(sz)),
        "workspace r_cap 0": L.care_workspace_size(4, 4, 1, 1, 0, 1, ct.byref(o), ct.byref(sz)),
        "solve null A": L.care_solve(None, dummy, 4, 1, dummy, 1, 1, 1e-10, 1, ct.byref(o), dummy, 4, 8, dummy,
                                     1024, None, None),
        "solve null B": L.care_solve(ct.byref(ok_csr), None, 4, 1, dummy, 1, 1, 1e-10, 1, ct.byref(o), dummy, 4,
                                     8, dummy, 1024, None, None),
        "solve tol 0": L.care_solve(ct.byref(ok_csr), dummy, 4, 1, dummy, 1, 1, 0.0, 1, ct.byref(o), dummy, 4, 8,
                                    dummy, 1024, None, None),
        "lradi null A": L.lyap_lradi(None, None, 4, None, 4, 0, dummy, 4, 1, 1e-5, 1, ct.byref(o), dummy, 4, 8,
                                     dummy, 1024, None, None),
        "resfac null A": L.care_residual_factor(None, dummy, 4, 1, dummy, 1, 1, dummy, 4, 1, 1e-4, None, 4, None,
                                                None, 4, None, 8, None, dummy, 1024, None),
        "autotune null op": L.care_autotune(None, 1, 2, 1, ct.byref(o), dummy, 1024, None, None),
        "batched workspace 0 workers": L.care_workspace_size_batched(1, None, None, None, None, 1, ct.byref(o), 0,
                                                                     ct.byref(sz)),
        "batched count<0": L.care_solve_batched(-1, None, None, None, None, None, None, None, 1e-10, 1,
                                                ct.byref(o), None, None, None, 1, None, 0, None, None),
        "batched persistent count>256": L.care_solve_batched_persistent(
            257, None, None, None, None, None, None, None, 1e-10, 1, ct.byref(o), None, None, None, None, 0, None,
            None, None),
        "batched persistent null arrays": L.care_solve_batched_persistent(
            2, None, None, None, None, None, None, None, 1e-10, 1, ct.byref(o), None, None, None, dummy, 1024, None,
            None, None),
        "persistent workspace count>256": L.care_workspace_size_batched_persistent(257, None, None, None, None, 1,
                                                                                   ct.byref(o), ct.byref(sz)),
        "ilu0 null op": L.care_ilu0(None, 0, 1, -1.0, 0.0, dummy, dummy, 1024, None),
        "ilu0 dtype": L.care_ilu0(ct.byref(op0), 2, 1, -1.0, 0.0, dummy, dummy, 1024, None),
        "launch shape vpt 3": L.care_set_launch_shape(3, 8, 0),
        "launch shape ctas 9": L.care_set_launch_shape(1, 9, 0),
        "launch shape row order 2": L.care_set_launch_shape(1, 8, 2),
        "host symeig n<0": L.care_host_symeig(-1, None, None, None),
        "host gemm sym m!=n": L.care_host_gemm_nt(3, 2, 1, dummy, 1, dummy, 1, None, dummy, 2, 1),
    }
    bad = {k: v for k, v in cases.items() if v != INVALID}
    assert not bad, bad


def test_launch_shape_round_trip():
    """The process-wide launch shape (host state only): set applies one vectors-per-
    thread value to every width class, get reads the table back; the library's
    defaults are set again afterwards."""
    try:
        pb.set_launch_shape(2, 4, 1)
        assert pb.launch_shape() == ((2, 2, 2, 2, 2), 4, 1)
        pb.set_launch_shape(4, 8, 0)
        assert pb.launch_shape() == ((4, 4, 4, 4, 4), 8, 0)
    finally:
        pb.set_launch_shape(1, 8, 0)
    assert pb.launch_shape() == ((1, 1, 1, 1, 1), 8, 0)


def test_workspace_size_grows_with_problem():
    a = pb.workspace_size(400, 1920, 1, 1, 64, "mixed")
    b = pb.workspace_size(250000, 1248000, 5, 5, 512, "mixed")
    c = pb.workspace_size(250000, 1248000, 5, 5, 512, "fp64")
    assert 0 < a < b < c


_DETERMINISM_SCRIPT = r"""
import hashlib, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import paper_2607_14742_b300 as pb
rng = np.random.default_rng(20260)
h = hashlib.sha256()
for n in (150, 611):
    # small integers: the BLAS products below are exact in any order, so the inputs
    # do not depend on the BLAS thread count either
    M = rng.integers(-8, 9, size=(n, n)).astype(np.float64)
    A = M + M.T
    w, V = pb.host_symeig(A)
    h.update(w.tobytes()); h.update(V.tobytes())
    ws, Vs = pb.host_symeig_outside(A, np.quantile(w, 0.3), np.quantile(w, 0.8))
    h.update(ws.tobytes()); h.update(Vs.tobytes())
    G = M @ M.T + n * np.eye(n)
    h.update(np.float64(pb.host_sym_lmax(G)).tobytes())
    h.update(pb.host_cholesky_upper(G).tobytes())
    piv, R = pb.host_pivoted_cholesky(G, 1e-12 * np.abs(G).max())
    h.update(piv.tobytes()); h.update(R.tobytes())
    h.update(pb.host_gemm_nt(M, M, sym=True).tobytes())
    h.update(pb.host_upper_inverse(np.triu(M) + n * np.eye(n)).tobytes())
print(h.hexdigest())
"""


def test_host_dense_bitwise_independent_of_thread_count():
    """The host small-dense routines give bitwise identical results for any OpenMP
    thread count (the batched solver runs them with a share of the cores per worker,
    and its instances must equal individual solves bit for bit)."""
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    digests = set()
    for nt in (1, 3, 8):
        env = dict(os.environ, OMP_NUM_THREADS=str(nt), OMP_DYNAMIC="false")
        r = subprocess.run([sys.executable, "-c", _DETERMINISM_SCRIPT, root], env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0, r.stderr
        digests.add(r.stdout.strip())
    assert len(digests) == 1, digests
