// FP64 symmetric eigendecomposition on the GPU for the small dense matrices of
// Algorithms 1-2 (H = T M T^T and P = Gamma N Gamma^T, up to a few thousand):
// every eigenvalue, and eigenvectors only for the eigenvalues the truncation keeps.
//
//  1. Householder tridiagonalisation Q^T A Q = T (Golub & Van Loan, Alg. 8.3.1) in
//     one cooperative kernel: per column, every CTA forms the reflector from the
//     current row (redundantly, no exchange), p = beta A22 v is computed row-wise
//     across the grid, a grid barrier, then w = p - (beta/2)(p^T v) v and the
//     rank-2 update A22 -= v w^T + w v^T row-wise, a grid barrier.  The full
//     symmetric matrix is kept (both triangles), so every access is a contiguous row.
//  2. Eigenvalues of T by bisection on Sturm counts (Golub & Van Loan, Sec. 8.4.1;
//     the counting recurrence of LAPACK's dstebz), one thread per eigenvalue,
//     to an absolute accuracy of a few units of roundoff of ||T||.
//  3. Eigenvectors of T by inverse iteration with a partially pivoted LU of
//     T - lambda I (Golub & Van Loan, Sec. 8.4.3 / 7.6.1), one CTA per cluster:
//     eigenvalues closer than 1e-6 ||T||_1 (and, for callers that weight the
//     vectors by their eigenvalues, closer than 1e-3 of their magnitude) form a
//     cluster whose vectors are orthogonalised against each other after every
//     solve (as LAPACK's dstein does with its absolute 1e-3 window), by modified
//     Gram-Schmidt twice.
//  4. Back-transformation x <- H_0 ... H_{n-3} x, one CTA per group of vectors
//     held in shared memory.
// Results are deterministic (fixed reduction orders, no atomics).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "dense.cuh"

namespace cg = cooperative_groups;

namespace care {
namespace {

constexpr int SY_THREADS = 256;

// block-wide sum in a fixed order (all threads receive the result)
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // sh may still be read from the previous call
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;
}

// A (n x n, row-major, symmetric, full storage) -> T = (d, e); reflector k in
// Vh[k][k+1 .. n), tau[k] its beta (0: identity).  p: scratch of n doubles.
__global__ void __launch_bounds__(SY_THREADS) k_sytrd(int n, double* A, long lda, double* __restrict__ d,
                                                      double* __restrict__ e, double* __restrict__ tau,
                                                      double* __restrict__ Vh, double* p) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[SY_THREADS / 32];
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    // A is rewritten by other CTAs between the grid barriers: every read of it (and
    // of p) bypasses L1 (__ldcg), whose lines are not kept coherent across SMs
    const double* xk = A + (long)k * lda + k + 1;  // column k below the diagonal = row k right of it
    double s = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double x = __ldcg(xk + i);
      s += x * x;
    }
    const double xx = block_sum(s, sh);
    const double x0 = __ldcg(xk);
    const double xn = sqrt(xx);
    const double alpha = x0 > 0 ? -xn : xn;
    const double v0 = x0 - alpha;
    const double vn2 = xx - x0 * x0 + v0 * v0;
    const double beta = (xx > 0.0 && vn2 > 0.0) ? 2.0 / vn2 : 0.0;
    if (beta != 0.0) {
      // p_i = beta sum_j A22(i, j) v_j, one warp per row
      for (int i = gwarp; i < m; i += nwarps) {
        const double* ai = A + (long)(k + 1 + i) * lda + k + 1;
        double t = 0.0;
        for (int j = lane; j < m; j += 32) t += __ldcg(ai + j) * (j == 0 ? v0 : __ldcg(xk + j));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) p[i] = beta * t;
      }
    }
    grid.sync();
    if (beta != 0.0) {
      double t = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x) t += __ldcg(p + i) * (i == 0 ? v0 : __ldcg(xk + i));
      const double K = 0.5 * beta * block_sum(t, sh);
      // A22 -= v w^T + w v^T, w = p - K v (rows split over the warps of the grid)
      for (int i = gwarp; i < m; i += nwarps) {
        double* ai = A + (long)(k + 1 + i) * lda + k + 1;
        const double vi = i == 0 ? v0 : __ldcg(xk + i);
        const double wi = __ldcg(p + i) - K * vi;
        for (int j = lane; j < m; j += 32) {
          const double vj = j == 0 ? v0 : __ldcg(xk + j);
          const double wj = __ldcg(p + j) - K * vj;
          ai[j] = __ldcg(ai + j) - (vi * wj + wi * vj);
        }
      }
    }
    if (blockIdx.x == 0) {
      for (int i = threadIdx.x; i < m; i += blockDim.x) Vh[(long)k * n + k + 1 + i] = i == 0 ? v0 : __ldcg(xk + i);
      if (threadIdx.x == 0) {
        d[k] = __ldcg(A + (long)k * lda + k);
        e[k] = beta != 0.0 ? alpha : x0;
        tau[k] = beta;
      }
    }
    grid.sync();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(A + (long)(n - 2) * lda + n - 2);
      e[n - 2] = __ldcg(A + (long)(n - 1) * lda + n - 2);
      tau[n - 2] = 0.0;
    }
    d[n - 1] = __ldcg(A + (long)(n - 1) * lda + n - 1);
    tau[n - 1] = 0.0;
  }
}

// number of eigenvalues of T (d, e2 = e^2) below x
__device__ __forceinline__ int sturm_count(int n, const double* d, const double* e2, double x, double pivmin) {
  int cnt = 0;
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  cnt += q < 0.0;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

// w[i] = i-th smallest eigenvalue of T (ascending), bisection on [gl, gu]
__global__ void k_stebz(int n, const double* __restrict__ d, const double* __restrict__ e2, double gl, double gu,
                        double pivmin, double atol, double* __restrict__ w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double lo = gl, hi = gu;
  for (int it = 0; it < 200 && hi - lo > atol + 4.440892098500626e-16 * fmax(fabs(lo), fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(n, d, e2, mid, pivmin) > i) hi = mid;
    else lo = mid;
  }
  w[i] = 0.5 * (lo + hi);
}

// Inverse iteration for the selected eigenvalues, one CTA per cluster
// [cstart[c], cstart[c+1]) of the selected list lam[]; vector j -> X[j * n ..).
// Thread 0 factors T - lambda I (partially pivoted LU) and runs the triangular
// solves (inherently sequential); the CTA orthogonalises against the earlier
// vectors of the cluster and normalises in parallel.  Scratch per cluster: 5 n
// doubles and n pivots.
// (scratch and X are shared between the CTA's threads through global memory, so they
// are not declared __restrict__: the compiler must not keep their values in
// registers across the barriers)
__global__ void __launch_bounds__(128) k_stein(int n, const double* __restrict__ d, const double* __restrict__ e,
                                               int nclus, const int* __restrict__ cstart,
                                               const double* __restrict__ lam, double onenrm, double* X,
                                               double* scratch, int* iscratch) {
  const int c = blockIdx.x;
  if (c >= nclus) return;
  __shared__ double sh[4];
  const double eps = 2.220446049250313e-16;
  const double eps3 = eps * onenrm;
  double* dl = scratch + (long)c * 5 * n;
  double* dd = dl + n;
  double* du = dd + n;
  double* du2 = du + n;
  double* b = du2 + n;
  int* piv = iscratch + (long)c * n;
  auto csum = [&](double v) {  // CTA sum (4 warps), fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    return (sh[0] + sh[1]) + (sh[2] + sh[3]);
  };
  double lprev = -INFINITY;
  for (int j = cstart[c]; j < cstart[c + 1]; ++j) {
    double l = lam[j];
    if (l - lprev < 10.0 * eps3) l = lprev + 10.0 * eps3;  // separate equal eigenvalues
    lprev = l;
    if (threadIdx.x == 0) {
      // LU with partial pivoting of the tridiagonal T - l I (dgttrf)
      for (int i = 0; i < n; ++i) dd[i] = d[i] - l;
      for (int i = 0; i + 1 < n; ++i) {
        dl[i] = e[i];
        du[i] = e[i];
      }
      for (int i = 0; i + 2 < n; ++i) du2[i] = 0.0;
      for (int i = 0; i + 1 < n; ++i) {
        if (fabs(dd[i]) >= fabs(dl[i])) {
          piv[i] = i;
          const double f = dd[i] != 0.0 ? dl[i] / dd[i] : 0.0;
          dl[i] = f;
          dd[i + 1] -= f * du[i];
        } else {
          piv[i] = i + 1;
          const double f = dd[i] / dl[i];
          dd[i] = dl[i];
          dl[i] = f;
          const double t = du[i];
          du[i] = dd[i + 1];
          dd[i + 1] = t - f * dd[i + 1];
          if (i + 2 < n) {
            du2[i] = du[i + 1];
            du[i + 1] = -f * du[i + 1];
          }
        }
      }
      for (int i = 0; i < n; ++i)
        if (fabs(dd[i]) < eps3) dd[i] = dd[i] < 0 ? -eps3 : eps3;
      piv[n - 1] = n - 1;
    }
    // deterministic start vector (SplitMix64 hash of the eigenvalue's position)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      unsigned long long z = (unsigned long long)(j * 1315423911ull + i) * 0x9E3779B97F4A7C15ull + 0x1220ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      b[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    __syncthreads();
    for (int it = 0; it < 4; ++it) {
      if (threadIdx.x == 0) {
        // solve (L U) y = b in place: forward with the row interchanges, then back
        for (int i = 0; i + 1 < n; ++i) {
          if (piv[i] == i) {
            b[i + 1] -= dl[i] * b[i];
          } else {
            const double t = b[i];
            b[i] = b[i + 1];
            b[i + 1] = t - dl[i] * b[i];
          }
        }
        for (int i = n - 1; i >= 0; --i) {
          double sres = b[i];
          if (i + 1 < n) sres -= du[i] * b[i + 1];
          if (i + 2 < n) sres -= du2[i] * b[i + 2];
          b[i] = sres / dd[i];
        }
      }
      __syncthreads();
      // orthogonalise against the earlier vectors of the cluster (modified
      // Gram-Schmidt, twice)
      for (int pass = 0; pass < 2; ++pass)
        for (int q = cstart[c]; q < j; ++q) {
          const double* xq = X + (long)q * n;
          double t = 0.0;
          for (int i = threadIdx.x; i < n; i += blockDim.x) t += xq[i] * b[i];
          t = csum(t);
          for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] -= t * xq[i];
          __syncthreads();
        }
      double t = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) t += b[i] * b[i];
      const double nrm = sqrt(csum(t));
      const double sc = nrm > 0.0 ? 1.0 / nrm : 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] *= sc;
      __syncthreads();
    }
    // sign convention: the largest entry (first on ties) positive
    __shared__ int s_im;
    if (threadIdx.x == 0) {
      int im = 0;
      for (int i = 1; i < n; ++i)
        if (fabs(b[i]) > fabs(b[im])) im = i;
      s_im = im;
    }
    __syncthreads();
    const double sg = b[s_im] < 0 ? -1.0 : 1.0;
    double* x = X + (long)j * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = sg * b[i];
    __syncthreads();
  }
}

// x <- H_0 H_1 ... H_{n-3} x for VB vectors per CTA (rows of X, length n), held in
// shared memory; reflector k is Vh[k][k+1 .. n) with beta tau[k].
template <int VB>
__global__ void __launch_bounds__(SY_THREADS) k_ormtr(int n, int nv, const double* __restrict__ Vh,
                                                      const double* __restrict__ tau, double* __restrict__ X) {
  extern __shared__ double xs[];  // VB x n
  __shared__ double sh[VB][SY_THREADS / 32];
  const int v0 = blockIdx.x * VB;
  const int nb = min(VB, nv - v0);
  for (int q = 0; q < nb; ++q)
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[q * n + i] = X[(long)(v0 + q) * n + i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = n - 3; k >= 0; --k) {
    const double beta = tau[k];
    if (beta == 0.0) continue;
    const int m = n - k - 1;
    const double* u = Vh + (long)k * n + k + 1;
    double t[VB];
#pragma unroll
    for (int q = 0; q < VB; ++q) t[q] = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double ui = u[i];
#pragma unroll
      for (int q = 0; q < VB; ++q) t[q] += ui * xs[q * n + k + 1 + i];
    }
#pragma unroll
    for (int q = 0; q < VB; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t[q] += __shfl_xor_sync(0xffffffffu, t[q], o);
      if (lane == 0) sh[q][warp] = t[q];
    }
    __syncthreads();
    double dq[VB];
#pragma unroll
    for (int q = 0; q < VB; ++q) {
      double s = 0.0;
      for (int w = 0; w < SY_THREADS / 32; ++w) s += sh[q][w];
      dq[q] = beta * s;
    }
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double ui = u[i];
#pragma unroll
      for (int q = 0; q < VB; ++q)
        if (q < nb) xs[q * n + k + 1 + i] -= dq[q] * ui;
    }
    __syncthreads();
  }
  for (int q = 0; q < nb; ++q)
    for (int i = threadIdx.x; i < n; i += blockDim.x) X[(long)(v0 + q) * n + i] = xs[q * n + i];
}

__global__ void k_sym_copy(int n, const double* __restrict__ S, long lds, double* __restrict__ A, long lda) {
  // A = (S + S^T) / 2 (exactly symmetric working copy)
  const long total = (long)n * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t / n), j = (int)(t % n);
    A[(long)i * lda + j] = 0.5 * (S[(long)i * lds + j] + S[(long)j * lds + i]);
  }
}

__global__ void k_square(int n, const double* __restrict__ e, double* __restrict__ e2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) e2[i] = e[i] * e[i];
}

}  // namespace

size_t dev_symeig_work_elems(int n) {
  // A copy, reflectors (2 n^2); d, e, e^2, tau, p, eigenvalues (6 n + 8); inverse
  // iteration: 5 n doubles and n pivots per cluster (at most n clusters), then the
  // n + 1 cluster starts
  const size_t nn = (size_t)n * n;
  return 7 * nn + 6 * (size_t)n + 8 + (nn + n + 2) / 2 + 8;
}

// Eigenvalues (ascending, host w) of the symmetric n x n S (device, row-major, lds)
// and the eigenvectors of those selected by want(w_i, max|w|) into V (device, row i
// of V = eigenvector of w[sel[i]], length n), returning the selected indices.
std::vector<int> dev_symeig_select(int n, const double* S, int lds, std::vector<double>& w, double* V,
                                   const std::function<bool(double, double)>& want, double* work,
                                   size_t work_elems, cudaStream_t s, bool weighted) {
  std::vector<int> sel;
  w.assign(n, 0.0);
  if (n == 0) return sel;
  CARE_REQUIRE(work_elems >= dev_symeig_work_elems(n), CARE_ERR_WORKSPACE, "symeig: scratch too small");
  const size_t nn = (size_t)n * n;
  double* A = work;
  double* Vh = A + nn;
  double* d = Vh + nn;
  double* e = d + n;
  double* e2 = e + n;
  double* tau = e2 + n;
  double* p = tau + n;
  double* wd = p + n;
  double* sc = wd + n + 8;
  int* isc = reinterpret_cast<int*>(sc + 5 * nn);
  k_sym_copy<<<device_sms() * 4, 256, 0, s>>>(n, S, lds, A, n);
  CARE_LAUNCH();
  if (n == 1) {
    CARE_CUDA(cudaMemcpyAsync(w.data(), A, sizeof(double), cudaMemcpyDeviceToHost, s));
    CARE_CUDA(cudaStreamSynchronize(s));
    if (want(w[0], std::fabs(w[0]))) {
      const double one = 1.0;
      CARE_CUDA(cudaMemcpyAsync(V, &one, sizeof(double), cudaMemcpyHostToDevice, s));
      CARE_CUDA(cudaStreamSynchronize(s));
      sel.push_back(0);
    }
    return sel;
  }
  CARE_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  {
    // one CTA per SM, cooperative (the grid barriers need every CTA resident)
    int per_sm = 0;
    CARE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sytrd, SY_THREADS, 0));
    CARE_REQUIRE(per_sm >= 1, CARE_ERR_CUDA, "symeig: k_sytrd cannot be resident");
    const int grid = device_sms() * std::min(per_sm, 2);
    long lda = n;
    void* args[] = {(void*)&n, (void*)&A, (void*)&lda, (void*)&d, (void*)&e, (void*)&tau, (void*)&Vh, (void*)&p};
    CARE_CUDA(cudaLaunchCooperativeKernel((const void*)k_sytrd, dim3(grid), dim3(SY_THREADS), args, 0, s));
    count_launch();
  }
  // Gershgorin bounds and pivmin from (d, e) on the host (2n doubles)
  std::vector<double> hd(n), he(n);
  CARE_CUDA(cudaMemcpyAsync(hd.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaMemcpyAsync(he.data(), e, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  double gl = INFINITY, gu = -INFINITY, emax2 = 0.0, tnorm = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(he[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(he[i]) : 0.0);
    gl = std::min(gl, hd[i] - r);
    gu = std::max(gu, hd[i] + r);
    tnorm = std::max(tnorm, std::fabs(hd[i]) + r);
    if (i + 1 < n) emax2 = std::max(emax2, he[i] * he[i]);
  }
  CARE_REQUIRE(std::isfinite(gl) && std::isfinite(gu), CARE_NONFINITE, "symeig: non-finite matrix");
  const double eps = 2.220446049250313e-16;
  const double pivmin = 2.2250738585072014e-308 * std::max(1.0, emax2);
  const double pad = 2.0 * eps * tnorm * n + 2.0 * pivmin;
  gl -= pad;
  gu += pad;
  k_square<<<(n + 255) / 256, 256, 0, s>>>(n - 1, e, e2);
  CARE_LAUNCH();
  k_stebz<<<(n + 127) / 128, 128, 0, s>>>(n, d, e2, gl, gu, pivmin, 2.0 * eps * tnorm, wd);
  CARE_LAUNCH();
  CARE_CUDA(cudaMemcpyAsync(w.data(), wd, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  double wmax = 0.0;
  for (int i = 0; i < n; ++i) {
    CARE_REQUIRE(std::isfinite(w[i]), CARE_NONFINITE, "symeig: non-finite eigenvalue");
    wmax = std::max(wmax, std::fabs(w[i]));
  }
  for (int i = 0; i < n; ++i)
    if (want(w[i], wmax)) sel.push_back(i);
  const int k = (int)sel.size();
  if (k == 0) return sel;
  // clusters of the selected eigenvalues.  Inverse iteration leaves the vectors of
  // eigenvalues a gap g apart orthogonal to about eps ||T|| / g, so a new cluster
  // starts where the gap exceeds 1e-6 ||T||_1 (vectors of closer eigenvalues are
  // orthogonalised explicitly).  For weighted use (products that weight each vector
  // by its eigenvalue, V diag(lambda) V^T or V diag(sqrt|lambda|)) what matters is
  // |lambda| eps ||T|| / g, and a cluster also ends where the gap exceeds
  // 1e-3 max(|lambda_q|, |lambda_q-1|): that keeps the weighted loss of
  // orthogonality below about 1e3 eps ||T|| and splits the dense run of small
  // eigenvalues (hundreds within 1e-6 ||T|| of zero in the truncations) that would
  // otherwise be one cluster orthogonalised vector by vector in a single CTA.
  std::vector<double> lam(k);
  std::vector<int> cst;
  for (int q = 0; q < k; ++q) {
    lam[q] = w[sel[q]];
    const double gap = q > 0 ? lam[q] - lam[q - 1] : 0.0;
    if (q == 0 || gap > 1e-6 * tnorm ||
        (weighted && gap > 1e-3 * std::max(std::fabs(lam[q]), std::fabs(lam[q - 1]))))
      cst.push_back(q);
  }
  cst.push_back(k);
  const int ncl = (int)cst.size() - 1;
  // eigenvalues and cluster starts to the device (w is no longer needed there;
  // the cluster starts follow the n x n pivot array of the inverse iterations)
  double* dlam = wd;
  int* dcst = isc + nn;
  CARE_CUDA(cudaMemcpyAsync(dlam, lam.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
  CARE_CUDA(cudaMemcpyAsync(dcst, cst.data(), sizeof(int) * (ncl + 1), cudaMemcpyHostToDevice, s));
  k_stein<<<ncl, 128, 0, s>>>(n, d, e, ncl, dcst, dlam, tnorm, V, sc, isc);
  CARE_LAUNCH();
  constexpr int VB = 4;
  const size_t shm = (size_t)VB * n * sizeof(double);
  CARE_REQUIRE(shm <= 200 * 1024, CARE_ERR_INVALID_ARG, "symeig: n too large for the back-transformation");
  {
    static std::once_flag once[64];
    static cudaError_t attr_err[64];
    int dev = 0;
    CARE_CUDA(cudaGetDevice(&dev));
    std::call_once(once[dev & 63], [&] {
      attr_err[dev & 63] = cudaFuncSetAttribute(k_ormtr<VB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    CARE_CUDA(attr_err[dev & 63]);
  }
  k_ormtr<VB><<<(k + VB - 1) / VB, SY_THREADS, shm, s>>>(n, k, Vh, tau, V);
  CARE_LAUNCH();
  return sel;
}

}  // namespace care
