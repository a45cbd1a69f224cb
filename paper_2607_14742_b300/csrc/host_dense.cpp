// Small dense host routines for the q x q, s x s, h x h and m x m matrices of
// Algorithms 1-2, the projection shifts and the SMW capacitance matrix.
// Textbook algorithms (Golub & Van Loan, Matrix Computations, 4th ed.):
//   symmetric eigenproblem: Householder tridiagonalisation (Alg. 8.3.1) and the
//     implicit symmetric QR step with Wilkinson shift (Alg. 8.3.2) with
//     deflation; the requested eigenvectors are formed afterwards from the
//     recorded rotations and the stored reflectors;
//   nonsymmetric eigenvalues: Householder Hessenberg reduction (Alg. 7.4.2) and
//     the Francis double-shift QR step (Alg. 7.5.1) with deflation;
//   Cholesky (Alg. 4.2.2, also with complete diagonal pivoting) and LU with
//   partial pivoting (Alg. 3.4.1); triangular inverse by back substitution;
//   products A diag(d) B^T of row-major blocks.
// All matrices are column-major.
#include <algorithm>
#if defined(__SSE2__)
#include <immintrin.h>
#endif
#include <cmath>
#include <cstdint>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "dense.cuh"

namespace care {

namespace {

inline double& at(std::vector<double>& a, int n, int i, int j) { return a[(size_t)j * n + i]; }

// Givens pair (c, s) with [c s; -s c]^T [x; z] = [r; 0].
inline void givens(double x, double z, double& c, double& s) {
  if (z == 0.0) {
    c = 1.0;
    s = 0.0;
  } else if (std::fabs(z) > std::fabs(x)) {
    const double t = -x / z;
    s = 1.0 / std::sqrt(1.0 + t * t);
    c = s * t;
  } else {
    const double t = -z / x;
    c = 1.0 / std::sqrt(1.0 + t * t);
    s = c * t;
  }
}

}  // namespace

// dot product of contiguous vectors (vectorised reduction)
static inline double dotc(const double* x, const double* y, int k) {
  double s = 0.0;
#pragma omp simd reduction(+ : s)
  for (int l = 0; l < k; ++l) s += x[l] * y[l];
  return s;
}

// Eigenvectors.  With Q_T = G_1 G_2 ... G_N the product of the QR-step
// rotations and H_k the tridiagonalisation reflectors, eigenvector t is
// V(:, t) = H_0 H_1 ... H_{n-3} G_1 ... G_N e_j (j its tridiagonal index).
// Only the requested eigenvectors are formed: the rotations are recorded
// during the QR phase and applied afterwards, last to first, to blocks of
// SYM_BLK unit vectors (a block of n x 16 values stays in L2 while the
// rotations stream past), then the reflectors are applied to the same block.
namespace {
constexpr int SYM_BLK = 16;

struct Sweep {
  int l, u;
  size_t off;  // first rotation of the sweep in rc / rs
};

// y <- G_1 ... G_N y for a block stored as yb[k * 16 + jj] (16 independent
// vectors): sweeps and their rotations in reverse order; rotation k of a sweep
// maps (y_k, y_k+1) to (c y_k + s y_k+1, -s y_k + c y_k+1).
void apply_rotations_reverse(double* yb, const std::vector<Sweep>& sw, const std::vector<double>& rc,
                             const std::vector<double>& rs) {
  static_assert(SYM_BLK == 16, "register blocking assumes 16 vectors");
  for (size_t q = sw.size(); q-- > 0;) {
    const Sweep& w = sw[q];
    if (w.u <= w.l) continue;
    const double* cc = &rc[w.off];
    const double* ss = &rs[w.off];
#if defined(__AVX2__) && defined(__FMA__)
    double* x = yb + (size_t)w.u * SYM_BLK;
    __m256d t0 = _mm256_loadu_pd(x), t1 = _mm256_loadu_pd(x + 4), t2 = _mm256_loadu_pd(x + 8),
            t3 = _mm256_loadu_pd(x + 12);
    for (int k = w.u - 1; k >= w.l; --k) {
      x -= SYM_BLK;  // x = y_k, x + 16 = y_k+1
      const __m256d c = _mm256_set1_pd(cc[k - w.l]), s = _mm256_set1_pd(ss[k - w.l]);
      const __m256d a0 = _mm256_loadu_pd(x), a1 = _mm256_loadu_pd(x + 4), a2 = _mm256_loadu_pd(x + 8),
                    a3 = _mm256_loadu_pd(x + 12);
      // y_k+1 = c t - s a;  t = c a + s t
      _mm256_storeu_pd(x + SYM_BLK, _mm256_fmsub_pd(c, t0, _mm256_mul_pd(s, a0)));
      _mm256_storeu_pd(x + SYM_BLK + 4, _mm256_fmsub_pd(c, t1, _mm256_mul_pd(s, a1)));
      _mm256_storeu_pd(x + SYM_BLK + 8, _mm256_fmsub_pd(c, t2, _mm256_mul_pd(s, a2)));
      _mm256_storeu_pd(x + SYM_BLK + 12, _mm256_fmsub_pd(c, t3, _mm256_mul_pd(s, a3)));
      t0 = _mm256_fmadd_pd(s, t0, _mm256_mul_pd(c, a0));
      t1 = _mm256_fmadd_pd(s, t1, _mm256_mul_pd(c, a1));
      t2 = _mm256_fmadd_pd(s, t2, _mm256_mul_pd(c, a2));
      t3 = _mm256_fmadd_pd(s, t3, _mm256_mul_pd(c, a3));
    }
    _mm256_storeu_pd(x, t0);
    _mm256_storeu_pd(x + 4, t1);
    _mm256_storeu_pd(x + 8, t2);
    _mm256_storeu_pd(x + 12, t3);
#else
    double t[SYM_BLK];
    for (int jj = 0; jj < SYM_BLK; ++jj) t[jj] = yb[(size_t)w.u * SYM_BLK + jj];
    for (int k = w.u - 1; k >= w.l; --k) {
      const double c = cc[k - w.l], sn = ss[k - w.l];
      double* yk = yb + (size_t)k * SYM_BLK;
      double* yk1 = yk + SYM_BLK;
      for (int jj = 0; jj < SYM_BLK; ++jj) {
        const double a = yk[jj];
        yk1[jj] = c * t[jj] - sn * a;
        t[jj] = c * a + sn * t[jj];
      }
    }
    for (int jj = 0; jj < SYM_BLK; ++jj) yb[(size_t)w.l * SYM_BLK + jj] = t[jj];
#endif
  }
}
}  // namespace

bool host_symeig(int n, const double* A, double* w, double* V) { return host_symeig_select(n, A, w, V, nullptr); }

bool host_symeig_select(int n, const double* A, double* w, double* V,
                        const std::function<bool(double, double)>& want) {
  if (n <= 0) return true;
  // a: working copy (column-major == row-major for the symmetric matrix)
  std::vector<double> a(A, A + (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) {
      const double s = 0.5 * (at(a, n, i, j) + at(a, n, j, i));
      at(a, n, i, j) = s;
      at(a, n, j, i) = s;
    }
  const bool vec = V != nullptr;
  const bool par = n >= 96;
  // 1. Householder tridiagonalisation A <- H_k A H_k, H_k = I - beta_k v_k v_k^T with
  //    v_k supported on k+1..n-1 (Alg. 8.3.1); the reflectors are kept for the
  //    eigenvectors.  Panels of TRI_NB reflectors (the blocked form of the same
  //    reduction, as in LAPACK's dsytrd): within a panel the trailing matrix is not
  //    updated; each column is brought up to date from the panel's (v_t, w_t) just
  //    before its reflector is formed, and p = beta A v is corrected by the same
  //    terms.  After the panel the trailing lower triangle receives all of its
  //    rank-2 updates A -= V W^T + W V^T in one pass.
  constexpr int TRI_NB = 32;
  std::vector<double> hv, hbeta;
  std::vector<size_t> hoff;
  if (vec) {
    hv.resize((size_t)n * (n - 1) / 2 + 1);
    hbeta.assign(n, 0.0);
    hoff.assign(n, 0);
  }
  std::vector<double> v(n), p(n), wv(n), pbuf;
  std::vector<double> Vp((size_t)TRI_NB * n), Wp((size_t)TRI_NB * n), y1(TRI_NB), y2(TRI_NB);
  size_t voff = 0;
  for (int k0 = 0; k0 + 2 < n; k0 += TRI_NB) {
    const int kend = std::min(k0 + TRI_NB, n - 2);  // reflectors k0 .. kend-1
    std::fill(Vp.begin(), Vp.end(), 0.0);
    std::fill(Wp.begin(), Wp.end(), 0.0);
    for (int k = k0; k < kend; ++k) {
      const int jj = k - k0;
      const int m = n - k - 1;
      if (vec) hoff[k] = voff;
      voff += m;
      // column k (rows k..n-1) with the panel's earlier rank-2 updates applied
      double* colfull = &a[(size_t)k * n];
      for (int t = 0; t < jj; ++t) {
        const double wk = Wp[(size_t)t * n + k], vk = Vp[(size_t)t * n + k];
        const double* vt = &Vp[(size_t)t * n];
        const double* wt = &Wp[(size_t)t * n];
#pragma omp simd
        for (int g = k; g < n; ++g) colfull[g] -= vt[g] * wk + wt[g] * vk;
      }
      // ||a(k+1:n, k)|| with scaling by the largest entry (contiguous column)
      const double* colk = colfull + k + 1;
      double amax = 0.0;
      for (int i = 0; i < m; ++i) amax = std::max(amax, std::fabs(colk[i]));
      if (amax == 0.0) continue;
      double ss = 0.0;
      const double ia = 1.0 / amax;
#pragma omp simd reduction(+ : ss)
      for (int i = 0; i < m; ++i) ss += (colk[i] * ia) * (colk[i] * ia);
      const double xnorm = amax * std::sqrt(ss);
      const double x0 = colk[0];
      const double alpha = x0 > 0 ? -xnorm : xnorm;
      for (int i = 0; i < m; ++i) v[i] = colk[i];
      v[0] -= alpha;
      const double vn2 = dotc(v.data(), v.data(), m);
      if (vn2 == 0.0) continue;
      const double beta = 2.0 / vn2;
      // p = A22 v from the stored lower triangle of A22 (column j holds A22(i, j),
      // i >= j, contiguously): column j gives p_j its inner product with v[j..]
      // and adds A22(i, j) v_j to p_i, i > j.  The columns are dealt in blocks
      // of 16 to a fixed number of partial vectors (block b to partial b mod
      // SYMV_PARTS), each partial is formed by one thread in column order, and
      // the partials are summed in index order: the result is bitwise the same
      // for any number of threads.
      constexpr int SYMV_PARTS = 32;
      std::fill(p.begin(), p.begin() + m, 0.0);
      const bool parm = par && m >= 96;
      const int nblk = (m + 15) / 16;
      const int nparts = parm ? std::min(SYMV_PARTS, nblk) : 1;
      pbuf.assign((size_t)nparts * m, 0.0);
#pragma omp parallel for if (parm) schedule(dynamic, 1)
      for (int t = 0; t < nparts; ++t) {
        double* pt = &pbuf[(size_t)t * m];
        for (int blk = t; blk < nblk; blk += nparts) {
          const int jend = std::min(m, 16 * blk + 16);
          for (int j = 16 * blk; j < jend; ++j) {
            const double* col = &a[(size_t)(k + 1 + j) * n + k + 1];
            const double vj = v[j];
            double sj = 0.0;
#pragma omp simd reduction(+ : sj)
            for (int i = j; i < m; ++i) {
              sj += col[i] * v[i];
              pt[i] += col[i] * vj;
            }
            pt[j] += sj - col[j] * vj;  // the diagonal entry counted once
          }
        }
      }
      for (int t = 0; t < nparts; ++t)
        for (int i = 0; i < m; ++i) p[i] += pbuf[(size_t)t * m + i];
      // the panel's pending updates: A22 v -= V (W^T v) + W (V^T v)
      for (int t = 0; t < jj; ++t) {
        y1[t] = dotc(&Wp[(size_t)t * n + k + 1], v.data(), m);
        y2[t] = dotc(&Vp[(size_t)t * n + k + 1], v.data(), m);
      }
      for (int t = 0; t < jj; ++t) {
        const double* vt = &Vp[(size_t)t * n + k + 1];
        const double* wt = &Wp[(size_t)t * n + k + 1];
        const double a1 = y1[t], a2 = y2[t];
#pragma omp simd
        for (int i = 0; i < m; ++i) p[i] -= vt[i] * a1 + wt[i] * a2;
      }
      for (int i = 0; i < m; ++i) p[i] *= beta;
      const double pv = dotc(p.data(), v.data(), m);
      const double K = 0.5 * beta * pv;
      for (int i = 0; i < m; ++i) wv[i] = p[i] - K * v[i];
      std::copy(v.begin(), v.begin() + m, Vp.begin() + (size_t)jj * n + k + 1);
      std::copy(wv.begin(), wv.begin() + m, Wp.begin() + (size_t)jj * n + k + 1);
      // only the lower triangle is kept up to date: the subdiagonal entry is all
      // that later steps read of column k
      at(a, n, k + 1, k) = alpha;
      if (vec) {
        std::copy(v.begin(), v.begin() + m, hv.begin() + hoff[k]);
        hbeta[k] = beta;
      }
    }
    // trailing lower triangle (columns >= kend): A -= V W^T + W V^T over the panel
    const int np_ = kend - k0;
#pragma omp parallel for if (par && n - kend >= 96) schedule(dynamic, 8)
    for (int j = kend; j < n; ++j) {
      double* col = &a[(size_t)j * n];
      for (int t = 0; t < np_; ++t) {
        const double wj = Wp[(size_t)t * n + j], vj = Vp[(size_t)t * n + j];
        if (wj == 0.0 && vj == 0.0) continue;
        const double* vt = &Vp[(size_t)t * n];
        const double* wt = &Wp[(size_t)t * n];
#pragma omp simd
        for (int g = j; g < n; ++g) col[g] -= vt[g] * wj + wt[g] * vj;
      }
    }
  }
  std::vector<double> d(n), e(n, 0.0);
  for (int i = 0; i < n; ++i) d[i] = at(a, n, i, i);
  for (int i = 0; i + 1 < n; ++i) e[i] = at(a, n, i + 1, i);
  std::vector<double>().swap(a);
  // 2. implicit symmetric QR with Wilkinson shift on the tridiagonal (d, e); the
  //    rotations are recorded for the eigenvectors
  std::vector<Sweep> sweeps;
  std::vector<double> rc, rs;
  const double eps = 2.220446049250313e-16;
  int u = n - 1;
  long iters = 0;
  while (u > 0) {
    if (std::fabs(e[u - 1]) <= eps * (std::fabs(d[u - 1]) + std::fabs(d[u]))) {
      e[u - 1] = 0.0;
      --u;
      continue;
    }
    int l = u - 1;
    while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
    if (l > 0) e[l - 1] = 0.0;
    if (++iters > 60L * n) return false;
    const double dd = 0.5 * (d[u - 1] - d[u]);
    const double eu = e[u - 1];
    const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, eu);
    const double mu = d[u] - (den != 0.0 ? eu * eu / den : 0.0);
    double x = d[l] - mu, z = e[l];
    double bulge = 0.0;
    if (vec) sweeps.push_back(Sweep{l, u, rc.size()});
    for (int k = l; k < u; ++k) {
      double c, s;
      givens(x, z, c, s);
      if (vec) {
        rc.push_back(c);
        rs.push_back(s);
      }
      if (k > l) e[k - 1] = c * e[k - 1] - s * bulge;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk - 2.0 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk + 2.0 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk - dk1) + (c * c - s * s) * ek;
      if (k + 1 < u) {
        bulge = -s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
        z = bulge;
      }
    }
  }
  // 3. sort ascending
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int x1, int x2) { return d[x1] < d[x2]; });
  double wmax = 0.0;
  for (int i = 0; i < n; ++i) {
    w[i] = d[idx[i]];
    if (!std::isfinite(w[i])) return false;
    wmax = std::max(wmax, std::fabs(w[i]));
  }
  if (!vec) return true;
  // 4. the requested eigenvectors, SYM_BLK at a time; the other columns are zero
  std::vector<int> sel;
  for (int t = 0; t < n; ++t) {
    if (!want || want(w[t], wmax))
      sel.push_back(t);
    else
      std::fill(V + (size_t)t * n, V + (size_t)(t + 1) * n, 0.0);
  }
  const int nsel = (int)sel.size();
  const int nbk = (nsel + SYM_BLK - 1) / SYM_BLK;
#pragma omp parallel for if (par && nbk > 1) schedule(dynamic, 1)
  for (int bk = 0; bk < nbk; ++bk) {
#if defined(__SSE2__)
    // eigenvector entries decay exponentially along the tridiagonal; subnormal
    // values (below 2.2e-308, far under the accuracy of any entry) are flushed
    // to zero in this thread while the block is formed, then the mode is
    // restored (subnormal operands cost microcode assists on x86)
    const unsigned int csr = _mm_getcsr();
    _mm_setcsr(csr | 0x8040u);  // FTZ | DAZ
#endif
    const int j0 = bk * SYM_BLK;
    const int jn = std::min(SYM_BLK, nsel - j0);
    std::vector<double> yb((size_t)n * SYM_BLK, 0.0);
    for (int jj = 0; jj < jn; ++jj) yb[(size_t)idx[sel[j0 + jj]] * SYM_BLK + jj] = 1.0;
    apply_rotations_reverse(yb.data(), sweeps, rc, rs);
    for (int k = n - 3; k >= 0; --k) {
      const double beta = hbeta[k];
      if (beta == 0.0) continue;
      const int m = n - k - 1;
      const double* vk = &hv[hoff[k]];
      double dot[SYM_BLK] = {};
      for (int i = 0; i < m; ++i) {
        const double vi = vk[i];
        const double* row = &yb[(size_t)(k + 1 + i) * SYM_BLK];
#pragma omp simd
        for (int jj = 0; jj < SYM_BLK; ++jj) dot[jj] += vi * row[jj];
      }
      for (int jj = 0; jj < SYM_BLK; ++jj) dot[jj] *= beta;
      for (int i = 0; i < m; ++i) {
        const double vi = vk[i];
        double* row = &yb[(size_t)(k + 1 + i) * SYM_BLK];
#pragma omp simd
        for (int jj = 0; jj < SYM_BLK; ++jj) row[jj] -= vi * dot[jj];
      }
    }
    for (int jj = 0; jj < jn; ++jj) {
      double* out = V + (size_t)sel[j0 + jj] * n;
      for (int i = 0; i < n; ++i) out[i] = yb[(size_t)i * SYM_BLK + jj];
    }
#if defined(__SSE2__)
    _mm_setcsr(csr);
#endif
  }
  return true;
}

double host_sym_lmax(int n, const double* G) {
  // Largest eigenvalue of the symmetric n x n matrix G by Lanczos with full
  // reorthogonalisation (Golub & Van Loan, Sec. 10.1): the largest Ritz value
  // theta of the k x k tridiagonal T_k is returned once its residual bound
  // |beta_k s_k| (s_k the last entry of its Ritz vector; checked every 4 steps)
  // is below 1e-10 theta, so that an eigenvalue of G lies within 1e-10 theta of
  // it.  Matrices with n < 700 (where the full computation is as fast), and a
  // run that has not converged after kmax steps, use the full eigenvalue
  // computation.  The start vector is a fixed pseudo-random one.
  if (n <= 0) return 0.0;
  auto full = [&]() {
    std::vector<double> w(n);
    if (!host_symeig(n, G, w.data(), nullptr)) return std::nan("");
    return w[n - 1];
  };
  if (n < 700) return full();
  const int kmax = std::min(n, 160);
  std::vector<double> Q((size_t)kmax * n), w(n), alpha, beta;
  uint64_t st = 0x243f6a8885a308d3ull;
  double nrm = 0.0;
  for (int i = 0; i < n; ++i) {
    st += 0x9e3779b97f4a7c15ull;
    uint64_t z = st;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z ^= z >> 31;
    Q[i] = (double)(z >> 11) * 0x1.0p-53 - 0.5;
    nrm += Q[i] * Q[i];
  }
  nrm = std::sqrt(nrm);
  for (int i = 0; i < n; ++i) Q[i] /= nrm;
  const bool par = n >= 512;
  for (int k = 0; k < kmax; ++k) {
    const double* q = &Q[(size_t)k * n];
#pragma omp parallel for if (par) schedule(static)
    for (int i = 0; i < n; ++i) w[i] = dotc(G + (size_t)i * n, q, n);
    alpha.push_back(dotc(q, w.data(), n));
    // full reorthogonalisation against q_0 .. q_k, twice
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j <= k; ++j) {
        const double* qj = &Q[(size_t)j * n];
        const double h = dotc(qj, w.data(), n);
        for (int i = 0; i < n; ++i) w[i] -= h * qj[i];
      }
    const double bk = std::sqrt(dotc(w.data(), w.data(), n));
    const bool last = k + 1 == kmax || bk <= 1e-300;
    if (k % 4 != 3 && !last) {
      beta.push_back(bk);
      double* qn = &Q[(size_t)(k + 1) * n];
      for (int i = 0; i < n; ++i) qn[i] = w[i] / bk;
      continue;
    }
    // largest eigenpair of T_{k+1}
    const int m = k + 1;
    std::vector<double> T((size_t)m * m, 0.0), ev(m), V((size_t)m * m);
    for (int i = 0; i < m; ++i) {
      T[(size_t)i * m + i] = alpha[i];
      if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = beta[i];
    }
    if (!host_symeig(m, T.data(), ev.data(), V.data())) return full();
    const double theta = ev[m - 1];
    const double sk = V[(size_t)(m - 1) * m + (m - 1)];
    const double scale = std::max(std::fabs(theta), 1e-300);
    if (std::fabs(bk * sk) <= 1e-10 * scale || bk <= 1e-300) return theta;
    if (k + 1 == n) return theta;  // T_n is similar to G
    beta.push_back(bk);
    if (k + 1 < kmax) {
      double* qn = &Q[(size_t)(k + 1) * n];
      for (int i = 0; i < n; ++i) qn[i] = w[i] / bk;
    }
  }
  return full();
}

bool host_eigvals(int n, const double* A, double* wr, double* wi) {
  if (n <= 0) return true;
  std::vector<double> h(A, A + (size_t)n * n);
  auto H = [&](int i, int j) -> double& { return h[(size_t)j * n + i]; };
  // Hessenberg reduction
  std::vector<double> v(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double xnorm = 0.0;
    for (int i = 0; i < m; ++i) xnorm = std::hypot(xnorm, H(k + 1 + i, k));
    if (xnorm == 0.0) continue;
    const double alpha = H(k + 1, k) > 0 ? -xnorm : xnorm;
    for (int i = 0; i < m; ++i) v[i] = H(k + 1 + i, k);
    v[0] -= alpha;
    double vn2 = 0.0;
    for (int i = 0; i < m; ++i) vn2 += v[i] * v[i];
    if (vn2 == 0.0) continue;
    const double beta = 2.0 / vn2;
    // rows: H[k+1:, :] -= beta v (v^T H[k+1:, :])
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += v[i] * H(k + 1 + i, j);
      s *= beta;
      for (int i = 0; i < m; ++i) H(k + 1 + i, j) -= s * v[i];
    }
    // columns: H[:, k+1:] -= beta (H[:, k+1:] v) v^T
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += H(r, k + 1 + i) * v[i];
      s *= beta;
      for (int i = 0; i < m; ++i) H(r, k + 1 + i) -= s * v[i];
    }
    for (int i = k + 2; i < n; ++i) H(i, k) = 0.0;
  }
  const double eps = 2.220446049250313e-16;
  int u = n - 1;
  int iters = 0, total = 0;
  while (u >= 0) {
    if (u == 0) {
      wr[0] = H(0, 0);
      wi[0] = 0.0;
      break;
    }
    int l = u;
    while (l > 0) {
      double s = std::fabs(H(l - 1, l - 1)) + std::fabs(H(l, l));
      if (s == 0.0) s = 1.0;
      if (std::fabs(H(l, l - 1)) <= eps * s) break;
      --l;
    }
    if (l > 0) H(l, l - 1) = 0.0;
    if (l == u) {
      wr[u] = H(u, u);
      wi[u] = 0.0;
      --u;
      iters = 0;
      continue;
    }
    if (l == u - 1) {
      // eigenvalues of the trailing 2 x 2 block
      const double a11 = H(u - 1, u - 1), a12 = H(u - 1, u), a21 = H(u, u - 1), a22 = H(u, u);
      const double tr = 0.5 * (a11 + a22);
      const double det = a11 * a22 - a12 * a21;
      const double disc = tr * tr - det;
      if (disc >= 0) {
        const double sq = std::sqrt(disc);
        const double r1 = tr + (tr >= 0 ? sq : -sq);
        const double r2 = (r1 != 0.0) ? det / r1 : tr - (tr >= 0 ? sq : -sq);
        wr[u - 1] = r1; wi[u - 1] = 0.0;
        wr[u] = r2; wi[u] = 0.0;
      } else {
        const double sq = std::sqrt(-disc);
        wr[u - 1] = tr; wi[u - 1] = sq;
        wr[u] = tr; wi[u] = -sq;
      }
      u -= 2;
      iters = 0;
      continue;
    }
    if (++total > 100 * n) return false;
    ++iters;
    // Francis double shift (exceptional shifts every 10 stalled iterations)
    double s, t;
    if (iters % 10 == 0) {
      const double ex = std::fabs(H(u, u - 1)) + std::fabs(H(u - 1, u - 2));
      s = 1.5 * ex;
      t = ex * ex;
    } else {
      s = H(u - 1, u - 1) + H(u, u);
      t = H(u - 1, u - 1) * H(u, u) - H(u - 1, u) * H(u, u - 1);
    }
    double x = H(l, l) * H(l, l) + H(l, l + 1) * H(l + 1, l) - s * H(l, l) + t;
    double y = H(l + 1, l) * (H(l, l) + H(l + 1, l + 1) - s);
    double z = H(l + 1, l) * H(l + 2, l + 1);
    for (int k = l; k <= u - 2; ++k) {
      // 3-element Householder P = I - beta w w^T with P [x y z]^T = alpha e1
      double nrm = std::sqrt(x * x + y * y + z * z);
      if (nrm != 0.0) {
        const double alpha = x > 0 ? -nrm : nrm;
        double w0 = x - alpha, w1 = y, w2 = z;
        const double wn2 = w0 * w0 + w1 * w1 + w2 * w2;
        if (wn2 != 0.0) {
          const double beta = 2.0 / wn2;
          const int c0 = std::max(l, k - 1);
          for (int j = c0; j <= u; ++j) {
            const double sj = beta * (w0 * H(k, j) + w1 * H(k + 1, j) + w2 * H(k + 2, j));
            H(k, j) -= sj * w0; H(k + 1, j) -= sj * w1; H(k + 2, j) -= sj * w2;
          }
          const int r1 = std::min(k + 3, u);
          for (int r = l; r <= r1; ++r) {
            const double sr = beta * (H(r, k) * w0 + H(r, k + 1) * w1 + H(r, k + 2) * w2);
            H(r, k) -= sr * w0; H(r, k + 1) -= sr * w1; H(r, k + 2) -= sr * w2;
          }
        }
      }
      x = H(k + 1, k);
      y = H(k + 2, k);
      if (k < u - 2) z = H(k + 3, k);
    }
    // final 2-element reflector on rows/cols u-1, u
    {
      double nrm = std::hypot(x, y);
      if (nrm != 0.0) {
        const double alpha = x > 0 ? -nrm : nrm;
        double w0 = x - alpha, w1 = y;
        const double wn2 = w0 * w0 + w1 * w1;
        if (wn2 != 0.0) {
          const double beta = 2.0 / wn2;
          for (int j = std::max(l, u - 2); j <= u; ++j) {
            const double sj = beta * (w0 * H(u - 1, j) + w1 * H(u, j));
            H(u - 1, j) -= sj * w0; H(u, j) -= sj * w1;
          }
          for (int r = l; r <= u; ++r) {
            const double sr = beta * (H(r, u - 1) * w0 + H(r, u) * w1);
            H(r, u - 1) -= sr * w0; H(r, u) -= sr * w1;
          }
        }
      }
    }
  }
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(wr[i]) || !std::isfinite(wi[i])) return false;
  return true;
}

bool host_cholesky_upper(int n, const double* G, double* R) {
  // G = R^T R, R upper triangular (column-major: R[j * n + k] = R(k, j), so the
  // first j entries of column j are contiguous).  Column by column (Alg. 4.2.2
  // in its dot-product form); the entries of row j right of the diagonal are
  // independent and computed in parallel.
  for (size_t i = 0; i < (size_t)n * n; ++i) R[i] = 0.0;
  const bool par = n >= 128;
  for (int j = 0; j < n; ++j) {
    const double* rj = R + (size_t)j * n;
    const double s = G[(size_t)j * n + j] - dotc(rj, rj, j);
    if (!(s > 0.0)) return false;
    const double rjj = std::sqrt(s);
    R[(size_t)j * n + j] = rjj;
#pragma omp parallel for if (par && n - j > 64) schedule(static)
    for (int i = j + 1; i < n; ++i) {
      double* ri = R + (size_t)i * n;
      ri[j] = (G[(size_t)i * n + j] - dotc(rj, ri, j)) / rjj;
    }
  }
  return true;
}

int host_pivoted_cholesky(int c, const double* G, double tol, int max_rank, std::vector<int>& piv,
                          std::vector<double>& R) {
  // Outer loop of Alg. 4.2.2 with complete (diagonal) pivoting: the next pivot is
  // the largest remaining diagonal entry d_j of the Schur complement.  The factor
  // is also kept transposed (Rt[i * c + l] = R(l, i)) so that the inner products
  // over the earlier pivots are contiguous.
  std::vector<double> d(c);
  for (int j = 0; j < c; ++j) d[j] = G[(size_t)j * c + j];
  std::vector<char> used(c, 0);
  std::vector<double> Rt((size_t)c * c, 0.0);
  R.assign(0, 0.0);
  piv.clear();
  int r = 0;
  const bool par = c >= 128;
  while (r < c && (max_rank <= 0 || r < max_rank)) {
    int jp = -1;
    double best = tol;
    for (int j = 0; j < c; ++j)
      if (!used[j] && d[j] > best) {
        best = d[j];
        jp = j;
      }
    if (jp < 0) break;
    used[jp] = 1;
    piv.push_back(jp);
    R.resize((size_t)(r + 1) * c, 0.0);
    double* rk = &R[(size_t)r * c];
    const double rkk = std::sqrt(d[jp]);
    rk[jp] = rkk;
    Rt[(size_t)jp * c + r] = rkk;
    const double* tj = &Rt[(size_t)jp * c];
#pragma omp parallel for if (par && (long)c * r > 100000) schedule(static)
    for (int i = 0; i < c; ++i) {
      if (used[i]) continue;
      const double v = (G[(size_t)jp * c + i] - dotc(tj, &Rt[(size_t)i * c], r)) / rkk;
      rk[i] = v;
      Rt[(size_t)i * c + r] = v;
      d[i] -= v * v;
    }
    ++r;
  }
  return r;
}

void host_upper_inverse(int r, const double* U, double* Ui) {
  // Ui = U^{-1} for upper triangular U (both row-major); column j of Ui by back
  // substitution, rows of U read contiguously; the columns are independent
  std::fill(Ui, Ui + (size_t)r * r, 0.0);
#pragma omp parallel if (r >= 128)
  {
    std::vector<double> x(r);
#pragma omp for schedule(dynamic, 8)
    for (int j = 0; j < r; ++j) {
      for (int i = j; i >= 0; --i) {
        const double* ui = U + (size_t)i * r;
        const double s = (i == j ? 1.0 : 0.0) - dotc(ui + i + 1, &x[i + 1], j - i);
        x[i] = s / ui[i];
      }
      for (int i = 0; i <= j; ++i) Ui[(size_t)i * r + j] = x[i];
    }
  }
}

void host_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, const double* dk,
                  double* C, int ldc, bool sym) {
  // C = A diag(dk) B^T, A (m x k) and B (n x k) row-major: inner products of rows.
  // 4 x 2 tiles of C share their row loads (8 vectorised reductions per pass);
  // sym (A diag(dk) A^T) computes the tiles on and above the diagonal and mirrors.
  std::vector<double> Bs;
  if (dk) {
    Bs.resize((size_t)n * k);
    for (int j = 0; j < n; ++j)
      for (int l = 0; l < k; ++l) Bs[(size_t)j * k + l] = B[(size_t)j * ldb + l] * dk[l];
    B = Bs.data();
    ldb = k;
  }
  const int mt = (m + 3) / 4;
#pragma omp parallel for if ((long)m * n * k > 2000000) schedule(dynamic, 1)
  for (int ti = 0; ti < mt; ++ti) {
    const int i0 = 4 * ti;
    const int j_begin = sym ? i0 : 0;
    for (int j0 = j_begin; j0 < n; j0 += 2) {
      if (i0 + 4 <= m && j0 + 2 <= n) {
        const double *a0 = A + (size_t)i0 * lda, *a1 = a0 + lda, *a2 = a1 + lda, *a3 = a2 + lda;
        const double *b0 = B + (size_t)j0 * ldb, *b1 = b0 + ldb;
        double s00 = 0, s01 = 0, s10 = 0, s11 = 0, s20 = 0, s21 = 0, s30 = 0, s31 = 0;
#pragma omp simd reduction(+ : s00, s01, s10, s11, s20, s21, s30, s31)
        for (int l = 0; l < k; ++l) {
          const double x0 = b0[l], x1 = b1[l];
          s00 += a0[l] * x0;
          s01 += a0[l] * x1;
          s10 += a1[l] * x0;
          s11 += a1[l] * x1;
          s20 += a2[l] * x0;
          s21 += a2[l] * x1;
          s30 += a3[l] * x0;
          s31 += a3[l] * x1;
        }
        const double t[4][2] = {{s00, s01}, {s10, s11}, {s20, s21}, {s30, s31}};
        for (int u = 0; u < 4; ++u)
          for (int v = 0; v < 2; ++v) C[(size_t)(i0 + u) * ldc + j0 + v] = t[u][v];
      } else {
        for (int i = i0; i < std::min(m, i0 + 4); ++i)
          for (int j = j0; j < std::min(n, j0 + 2); ++j)
            C[(size_t)i * ldc + j] = dotc(A + (size_t)i * lda, B + (size_t)j * ldb, k);
      }
    }
  }
  if (sym)
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < std::min(i, n); ++j)
        if (j < (i / 4) * 4) C[(size_t)i * ldc + j] = C[(size_t)j * ldc + i];
}

bool host_lu_solve_complex(int n, std::vector<cd> A, cd* B, int k) {
  auto a = [&](int i, int j) -> cd& { return A[(size_t)j * n + i]; };
  auto b = [&](int i, int j) -> cd& { return B[(size_t)j * n + i]; };
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = std::hypot(a(c, c).re, a(c, c).im);
    for (int r = c + 1; r < n; ++r) {
      const double v = std::hypot(a(r, c).re, a(r, c).im);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0) || !std::isfinite(best)) return false;
    if (piv != c) {
      for (int j = 0; j < n; ++j) std::swap(a(c, j), a(piv, j));
      for (int j = 0; j < k; ++j) std::swap(b(c, j), b(piv, j));
    }
    for (int r = c + 1; r < n; ++r) {
      const cd f = cdivz(a(r, c), a(c, c));
      for (int j = c; j < n; ++j) {
        const cd t = cmul(f, a(c, j));
        a(r, j).re -= t.re; a(r, j).im -= t.im;
      }
      for (int j = 0; j < k; ++j) {
        const cd t = cmul(f, b(c, j));
        b(r, j).re -= t.re; b(r, j).im -= t.im;
      }
    }
  }
  for (int j = 0; j < k; ++j)
    for (int r = n - 1; r >= 0; --r) {
      cd s = b(r, j);
      for (int c = r + 1; c < n; ++c) {
        const cd t = cmul(a(r, c), b(c, j));
        s.re -= t.re; s.im -= t.im;
      }
      b(r, j) = cdivz(s, a(r, r));
    }
  return true;
}

}  // namespace care
