"""The device symmetric eigendecomposition of Algorithms 1-2 (tridiagonalisation,
bisection, inverse iteration, back-transformation) against LAPACK through NumPy:
eigenvalues within the backward-stable bound, selected eigenvectors with small
residuals and orthonormal, on random, indefinite low-rank, clustered and
graded spectra (the shapes of H = T M T^T and P = Gamma N Gamma^T)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2607_14742_b300 as m
    m.lib()
    return m


def _case(kind, n, rng):
    if kind == "random":
        M = rng.standard_normal((n, n))
        return M + M.T
    if kind == "indefinite_lowrank":
        # T M T^T with M = [[0, I, 0], [I, 0, 0], [0, 0, -I]]-like signature: rank 3k
        k = n // 6
        T = rng.standard_normal((n, 3 * k))
        d = np.concatenate([np.ones(k), -np.ones(k), np.ones(k) * 0.5])
        return (T * d) @ T.T
    if kind == "clustered":
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.concatenate([np.full(n // 4, 1.0) + 1e-12 * rng.standard_normal(n // 4),
                              np.linspace(-3, 3, n - n // 4)])
        return (Q * lam) @ Q.T
    if kind == "graded":
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = np.logspace(0, -14, n) * rng.choice([-1, 1], n)
        return (Q * lam) @ Q.T
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["random", "indefinite_lowrank", "clustered", "graded"])
@pytest.mark.parametrize("n", [1, 2, 7, 130, 700])
def test_symeig_vs_lapack(pb, kind, n):
    rng = np.random.default_rng(n * 7 + len(kind))
    A = _case(kind, n, rng) if n > 2 else rng.standard_normal((n, n)) + rng.standard_normal((n, n)).T
    A = 0.5 * (A + A.T)
    w, V, ns = pb.symeig(torch.tensor(A, device="cuda"))
    wr = np.linalg.eigvalsh(A)
    nrm = np.abs(wr).max() if n else 1.0
    assert np.all(np.abs(w - wr) <= 8 * n * EPS * max(nrm, 1e-300))
    assert ns == n
    V = V.cpu().numpy()
    res = np.abs(A @ V.T - V.T * w).max()
    assert res <= 16 * n * EPS * nrm
    assert np.abs(V @ V.T - np.eye(n)).max() <= 1e-10 * max(n, 1)


def test_symeig_selected_only(pb):
    """Eigenvectors only outside (lo, hi), as the truncations request them."""
    rng = np.random.default_rng(3)
    A = _case("indefinite_lowrank", 400, rng)
    wr, Vr = np.linalg.eigh(A)
    eta = 1e-4 * np.abs(wr).max()
    w, V, ns = pb.symeig(torch.tensor(A, device="cuda"), -eta, eta)
    keep = (wr <= -eta) | (wr >= eta)
    assert ns == keep.sum()
    V = V.cpu().numpy()
    sgn = np.sign(np.sum(V * Vr[:, keep].T, axis=1))
    assert np.abs(V - (Vr[:, keep] * sgn).T).max() <= 1e-9
