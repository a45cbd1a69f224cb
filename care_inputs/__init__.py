"""Seeded synthetic inputs for the sparse CARE  A^T X + X A - X B B^T X + C^T C = 0.

This module holds input generators only: it contains none of the solver's
arithmetic, so both the CPU oracle (``oracle/``) and the GPU library's tests
and benchmark may use it without sharing any method code.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value k of stream s is mix64(seed_s + (k + 1) * 0x9E3779B97F4A7C15), mapped to
a double in [0, 1) by its top 53 bits.  Normal variates use the Box-Muller
transform on consecutive pairs.  The paper fixes MATLAB's ``rng(1220)``
(Section 5); that generator cannot be reproduced here, so the seed 1220 is
kept and the generator replaced.

Operators (the paper's SuiteSparse matrices are not available, so these
synthetic operators stand in for them):
  * 2D/3D convection-diffusion  L u = -Lap(u) + c . grad(u)  on the unit
    square/cube, Dirichlet boundary, central differences, h = 1/(N+1),
    lexicographic order with x fastest; the CARE uses A = -L (stable).
  * the pure Dirichlet Laplacian (c = 0) with its analytic sine eigenvectors,
    used for closed-form large-n checks.
  * dense conditioning family  A = Q(-diag(lambda) + 0.1 N)Q^T.
  * the paper's dense Example 1 (Section 5.1) and banded Toeplitz example
    (Section 5.2).

CSR arrays are (rowptr int32[n+1], colind int32[nnz], val float64[nnz]) for A
itself (not A^T), columns sorted within each row.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED = 1220
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


class Stream:
    """Counter-based SplitMix64 stream; ``Stream(seed, sid)`` are independent."""

    def __init__(self, seed: int = SEED, sid: int = 0):
        base = _mix64(np.array([np.uint64(seed) ^ _mix64(np.array([sid], np.uint64))[0]],
                               dtype=np.uint64))[0]
        self._base = np.uint64(base)
        self._k = 0

    def bits(self, count: int) -> np.ndarray:
        ks = np.arange(self._k + 1, self._k + 1 + count, dtype=np.uint64)
        self._k += count
        with np.errstate(over="ignore"):
            return _mix64(self._base + ks * _GOLDEN)

    def uniform(self, count: int) -> np.ndarray:
        return (self.bits(count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, count: int) -> np.ndarray:
        m = (count + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[0::2]  # (0, 1]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = r * np.cos(2.0 * math.pi * u2)
        z[1::2] = r * np.sin(2.0 * math.pi * u2)
        return z[:count]

    def integers(self, lo: int, hi: int, count: int) -> np.ndarray:
        """Uniform integers in [lo, hi] inclusive."""
        return lo + np.floor(self.uniform(count) * (hi - lo + 1)).astype(np.int64)


@dataclasses.dataclass
class CSR:
    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.val.size)

    def to_scipy(self):
        import scipy.sparse as sp
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))

    def to_dense(self) -> np.ndarray:
        D = np.zeros((self.n, self.n))
        for i in range(self.n):
            s, e = self.rowptr[i], self.rowptr[i + 1]
            D[i, self.colind[s:e]] += self.val[s:e]
        return D

    @staticmethod
    def from_dense(D: np.ndarray) -> "CSR":
        n = D.shape[0]
        rows, cols = np.nonzero(D)
        rowptr = np.zeros(n + 1, np.int64)
        np.add.at(rowptr, rows + 1, 1)
        rowptr = np.cumsum(rowptr)
        return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), D[rows, cols].astype(np.float64))


@dataclasses.dataclass
class CareProblem:
    name: str
    A: CSR
    B: np.ndarray  # n x m float64
    C: np.ndarray  # p x n float64
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self):
        return self.A.n

    @property
    def m(self):
        return self.B.shape[1]

    @property
    def p(self):
        return self.C.shape[0]


def _stencil_csr(dims, coeff_fn) -> CSR:
    """Assemble A = -L for the (2d+1)-point central-difference stencil."""
    N = dims[0]
    d = len(dims)
    n = N ** d
    h = 1.0 / (N + 1)
    idx = np.arange(n, dtype=np.int64)
    coords = [(idx // (N ** k)) % N for k in range(d)]  # x fastest
    diag_val, off = coeff_fn(h)
    rows, cols, vals = [idx], [idx], [np.full(n, diag_val)]
    for k in range(d):
        for sgn in (-1, +1):
            ok = (coords[k] + sgn >= 0) & (coords[k] + sgn < N)
            r = idx[ok]
            rows.append(r)
            cols.append(r + sgn * (N ** k))
            vals.append(np.full(r.size, off[k][sgn]))
    rows = np.concatenate(rows)
    cols = np.concatenate(cols)
    vals = np.concatenate(vals)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def convection_diffusion(N: int, conv) -> CSR:
    """A = -L, L u = -Lap(u) + sum_d conv[d] du/dx_d, on an N^d interior grid.

    Row P of L: (2d/h^2) u_P - sum (1/h^2) u_nb + conv_d (u_{+d} - u_{-d}) / (2h).
    """
    d = len(conv)

    def coeffs(h):
        ih2 = 1.0 / (h * h)
        off = []
        for k in range(d):
            # A = -L:  +1/h^2 for each neighbour, -/+ conv/(2h) for the +/- neighbour
            off.append({+1: ih2 - conv[k] / (2 * h), -1: ih2 + conv[k] / (2 * h)})
        return -2.0 * d * ih2, off

    return _stencil_csr([N] * d, coeffs)


def dirichlet_laplacian(N: int, d: int) -> CSR:
    """A = +Lap_h (negative definite): the c = 0 case of ``convection_diffusion``."""
    return convection_diffusion(N, [0.0] * d)


def laplacian_mode(N: int, d: int, k) -> tuple[np.ndarray, float]:
    """Unit-norm eigenvector and eigenvalue of ``dirichlet_laplacian(N, d)``.

    v(j_1..j_d) = prod_t sqrt(2h) sin(k_t pi j_t h), j_t = 1..N (x fastest);
    lambda = -(4/h^2) sum_t sin^2(k_t pi h / 2).
    """
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)
    v = np.ones(1)
    lam = 0.0
    for t in range(d):
        f = math.sqrt(2 * h) * np.sin(k[t] * math.pi * j * h)
        v = np.kron(f, v)  # x fastest => first factor varies fastest
        lam -= (4.0 / (h * h)) * math.sin(k[t] * math.pi * h / 2) ** 2
    return v, lam


def _fdm_problem(name, N, conv, m, p, dist, seed=SEED) -> CareProblem:
    A = convection_diffusion(N, conv)
    n = A.n
    s = Stream(seed, 0)
    if dist == "uniform":
        B = s.uniform(n * m).reshape(m, n).T.copy()     # column-major draw order
        C = s.uniform(p * n).reshape(p, n)
    else:
        B = (s.normal(n * m) / math.sqrt(n)).reshape(m, n).T.copy()
        C = (s.normal(p * n) / math.sqrt(n)).reshape(p, n)
    return CareProblem(name, A, B, C, dict(grid=N, conv=list(conv), dist=dist, seed=seed))


def config_small_fdm(N: int = 20) -> CareProblem:
    """2D convection-diffusion (10, 100), 20x20 grid (n=400), m = p = 1, U[0,1)."""
    return _fdm_problem(f"fdm2d_{N}x{N}_m1_p1", N, (10.0, 100.0), 1, 1, "uniform")


def config_fdm2d(N: int = 500, m: int = 5, p: int = 5) -> CareProblem:
    """2D convection-diffusion (10, 100), 500x500 grid (n=250,000), m = p = 5, U[0,1)."""
    return _fdm_problem(f"fdm2d_{N}x{N}_m{m}_p{p}", N, (10.0, 100.0), m, p, "uniform")


def config_fdm3d(N: int = 100, m: int = 10, p: int = 10) -> CareProblem:
    """3D convection-diffusion (10, 50, 100), 100^3 grid (n=1e6), m = p = 10, N(0,1)/sqrt(n)."""
    return _fdm_problem(f"fdm3d_{N}^3_m{m}_p{p}", N, (10.0, 50.0, 100.0), m, p, "normal")


def haar_orthogonal(n: int, s: Stream) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with R's signs fixed."""
    G = s.normal(n * n).reshape(n, n)
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


def config_dense_conditioning(k: int, n: int = 200, m: int = 2, p: int = 2,
                              literal: bool = False) -> CareProblem:
    """A = Q(-Lambda + 0.1 Lambda^{1/2} N Lambda^{1/2})Q^T, lambda log-spaced in [10^-k, 1]
    (ascending), N strictly upper N(0,1)/sqrt(n), Q Haar; B, C ~ N(0,1).

    The non-normal part is scaled by Lambda^{1/2} on both sides so that
    kappa_2(A) = 10^k: with the unscaled 0.1 N (``literal=True``) the
    triangular core is numerically singular for k >= 3 (kappa_2 > 1e16) and its
    computed eigenvalues leave the left half-plane.  The scaled core is
    similar to -Lambda + 0.1 Lambda N, so its eigenvalues are exactly -lambda."""
    s = Stream(SEED, 100 + k)
    Q = haar_orthogonal(n, s)
    lam = np.logspace(-k, 0, n)
    Nm = np.triu(s.normal(n * n).reshape(n, n), 1) / math.sqrt(n)
    if not literal:
        sq = np.sqrt(lam)
        Nm = sq[:, None] * Nm * sq[None, :]
    Ad = Q @ (-np.diag(lam) + 0.1 * Nm) @ Q.T
    B = s.normal(n * m).reshape(m, n).T.copy()
    C = s.normal(p * n).reshape(p, n)
    return CareProblem(f"dense_cond_k{k}_n{n}", CSR.from_dense(Ad), B, C, dict(k=k, dense=True))


def paper_example1(n: int = 1000, m: int = 10, p: int = 5, q: float = 1.0) -> CareProblem:
    """Section 5.1, Example 1: A = -V diag(logspace(0, q, n)) V^T, V the symmetric
    orthogonal sine matrix V_ij = sqrt(2/(n+1)) sin(i j pi/(n+1)), B = 0.2 ones,
    C = 0.1 ones; kappa_2(A) = 10^q."""
    i = np.arange(1, n + 1)
    V = math.sqrt(2.0 / (n + 1)) * np.sin(np.outer(i, i) * math.pi / (n + 1))
    Ad = -(V * np.logspace(0, q, n)) @ V.T
    return CareProblem(f"example1_n{n}_q{q}", CSR.from_dense(Ad), 0.2 * np.ones((n, m)),
                       0.1 * np.ones((p, n)), dict(q=q, dense=True))


def paper_toeplitz(n: int, m: int = 10, p: int = 5) -> CareProblem:
    """Section 5.2 Toeplitz example: diagonal -2.8, sub-diagonal 1, super-diagonals
    -1 at offsets 1, 2, 3; B (n x m) random with ||B||_F = 1, C (p x n) random."""
    rows, cols, vals = [], [], []
    for off, v in ((-1, 1.0), (0, -2.8), (1, -1.0), (2, -1.0), (3, -1.0)):
        r = np.arange(max(0, -off), min(n, n - off))
        rows.append(r), cols.append(r + off), vals.append(np.full(r.size, v))
    rows, cols, vals = map(np.concatenate, (rows, cols, vals))
    order = np.lexsort((cols, rows))
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, rows[order] + 1, 1)
    A = CSR(n, np.cumsum(rowptr).astype(np.int32), cols[order].astype(np.int32), vals[order])
    s = Stream(SEED, 7)
    B = s.uniform(n * m).reshape(m, n).T.copy()
    B /= np.linalg.norm(B)
    C = s.uniform(p * n).reshape(p, n)
    return CareProblem(f"toeplitz_n{n}", A, B, C)


def config_batched(count: int = 64, side_lo: int = 64, side_hi: int = 512, mp_hi: int = 8):
    """64 independent 2D convection-diffusion CAREs, grid side ~ U{64..512},
    m, p ~ U{1..8}, B and C ~ U[0,1) from per-instance streams."""
    s = Stream(SEED, 500)
    sides = s.integers(side_lo, side_hi, count)
    ms = s.integers(1, mp_hi, count)
    ps = s.integers(1, mp_hi, count)
    out = []
    for i in range(count):
        pr = _fdm_problem(f"batch{i}", int(sides[i]), (10.0, 100.0), int(ms[i]), int(ps[i]),
                          "uniform", seed=SEED + 1 + i)
        out.append(pr)
    return out


def eigen_aligned_problem(N: int, d: int, modes, beta, gamma) -> CareProblem:
    """CARE with A = dirichlet_laplacian(N, d), B = V_S diag(beta), C = diag(gamma) V_S^T,
    where V_S are the analytic unit eigenvectors of ``modes``; the Riccati equation
    then decouples along those eigenvectors."""
    A = dirichlet_laplacian(N, d)
    vs, lams = [], []
    for k in modes:
        v, lam = laplacian_mode(N, d, k)
        vs.append(v)
        lams.append(lam)
    V = np.stack(vs, axis=1)
    B = V * np.asarray(beta, float)
    C = (V * np.asarray(gamma, float)).T.copy()
    return CareProblem(f"aligned_{d}d_N{N}", A, B, C, dict(V=V, lams=np.array(lams),
                                                          beta=np.asarray(beta, float),
                                                          gamma=np.asarray(gamma, float)))


def random_block(n: int, b: int, sid: int, seed: int = SEED) -> np.ndarray:
    """n x b float64 block of U[-1, 1) entries (column-major draw order)."""
    return (2.0 * Stream(seed, sid).uniform(n * b) - 1.0).reshape(b, n).T.copy()
