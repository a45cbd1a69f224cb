// Dense-direct shifted solves: M_p X = RHS with M_p = (A + p I)^T formed densely
// from the prepared operator and factored by LU with partial pivoting, the solver
// class that the complexity analysis of Section 4 calls dense direct and that the
// stability experiments of Section 5.1 use for every shifted system.  For small
// and dense problems (the conditioning sweep) where a Krylov solve in the inner
// precision would stall before the Lyapunov-conditioning threshold is reached.
//
//  * Form: one thread per row of A^T scatters the row into M_p (column-major,
//    leading dimension n, complex interleaved when p is complex); the diagonal is
//    summed in FP64 with p and rounded once.
//  * Factor: one cooperative kernel, right-looking LU with partial pivoting
//    (largest |re| + |im| in the pivot column, the first of equal ones).  Column j
//    belongs to CTA j mod G for the whole factorisation, so a CTA only ever reads
//    its own writes to M.  Every CTA finds the pivot of step k itself from a copy
//    of column k that its owner wrote during step k - 1 into one of two buffers;
//    one grid barrier per step.  The LAPACK convention holds: rows of the L part
//    are exchanged too, ipiv[k] = the row exchanged with row k at step k.
//  * Solve: one CTA per right-hand-side column, the column in shared memory; the
//    row exchanges, then the unit lower and the upper triangular sweep, one
//    barrier per row.
// All arithmetic is in the precision T of the solve (FP32 for the inner solves
// of the mixed path, FP64 otherwise).
#include <cooperative_groups.h>

#include <algorithm>

#include "krylov.cuh"

namespace cg = cooperative_groups;

namespace care {
namespace {

constexpr int DLU_THREADS = 256;

template <class T>
struct C2 {
  T re, im;
};
template <class T>
__device__ __forceinline__ C2<T> c2mul(C2<T> a, C2<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <class T>
__device__ __forceinline__ C2<T> c2inv(C2<T> a) {
  const T d = a.re * a.re + a.im * a.im;
  return {a.re / d, -a.im / d};
}

template <class T, bool CPLX>
__device__ __forceinline__ C2<T> ld_c(const T* p, size_t i) {
  if constexpr (CPLX) return {p[2 * i], p[2 * i + 1]};
  else return {p[i], T(0)};
}
template <class T, bool CPLX>
__device__ __forceinline__ C2<T> ldcg_c(const T* p, size_t i) {
  if constexpr (CPLX) return {__ldcg(p + 2 * i), __ldcg(p + 2 * i + 1)};
  else return {__ldcg(p + i), T(0)};
}
template <class T, bool CPLX>
__device__ __forceinline__ void st_c(T* p, size_t i, C2<T> v) {
  if constexpr (CPLX) {
    p[2 * i] = v.re;
    p[2 * i + 1] = v.im;
  } else {
    p[i] = v.re;
  }
}
template <class T, bool CPLX>
__device__ __forceinline__ C2<T> mul_c(C2<T> a, C2<T> b) {
  if constexpr (CPLX) return c2mul(a, b);
  else return {a.re * b.re, T(0)};
}

template <class T, bool CPLX>
__global__ void k_dlu_form(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                           const double* __restrict__ val, double sre, double sim, T* __restrict__ M) {
  constexpr int E = CPLX ? 2 : 1;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    double dsum = sre;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      if (j == i) dsum += val[k];
      else M[((size_t)j * n + i) * E] += (T)val[k];
    }
    const size_t d = ((size_t)i * n + i) * E;
    M[d] = (T)dsum;
    if constexpr (CPLX) M[d + 1] = (T)sim;
  }
}

// argmax of a over the CTA (ties: the smaller index); returns the winning index
__device__ int block_argmax(double a, int idx, double* sv, int* si, double* best_out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double oa = __shfl_xor_sync(0xffffffffu, a, o);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (oa > a || (oa == a && oi < idx)) {
      a = oa;
      idx = oi;
    }
  }
  __syncthreads();  // sv / si reuse across calls
  if (lane == 0) {
    sv[wid] = a;
    si[wid] = idx;
  }
  __syncthreads();
  double ba = sv[0];
  int bi = si[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
    if (sv[w] > ba || (sv[w] == ba && si[w] < bi)) {
      ba = sv[w];
      bi = si[w];
    }
  *best_out = ba;
  return bi;
}

template <class T, bool CPLX>
__global__ void __launch_bounds__(DLU_THREADS) k_dlu_factor(int n, T* __restrict__ M, int* __restrict__ ipiv,
                                                             T* cbuf, int* __restrict__ info) {
  constexpr int E = CPLX ? 2 : 1;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sv[DLU_THREADS / 32];
  __shared__ int si[DLU_THREADS / 32];
  const int G = gridDim.x, tid = threadIdx.x, bd = blockDim.x;
  if (blockIdx.x == 0)
    for (int i = tid; i < n * E; i += bd) cbuf[i] = M[i];
  grid.sync();
  for (int k = 0; k < n; ++k) {
    const T* cb = cbuf + (size_t)(k & 1) * n * E;
    T* cnext = cbuf + (size_t)((k + 1) & 1) * n * E;
    // pivot of column k (every CTA, same data, same order: the same answer)
    double a = -1.0;
    int ai = n;
    for (int i = k + tid; i < n; i += bd) {
      const C2<T> v = ldcg_c<T, CPLX>(cb, i);
      const double m = fabs((double)v.re) + fabs((double)v.im);
      if (m > a) {
        a = m;
        ai = i;
      }
    }
    double best = 0.0;
    int p = block_argmax(a, ai, sv, si, &best);
    if (p >= n) p = k;  // no comparable entry (all NaN): treated as singular below
    const C2<T> ck = ldcg_c<T, CPLX>(cb, k);
    C2<T> pv = ldcg_c<T, CPLX>(cb, p);
    if (!(best > 0.0)) {  // exactly singular (or NaN): record the step, keep going finitely
      if (blockIdx.x == 0 && tid == 0) atomicCAS(info, 0, k + 1);
      pv = {T(1), T(0)};
    }
    const C2<T> inv = CPLX ? c2inv(pv) : C2<T>{T(1) / pv.re, T(0)};
    for (int j = blockIdx.x; j < n; j += G) {
      T* col = M + (size_t)j * n * E;
      if (j < k) {
        if (p != k && tid == 0) {
          const C2<T> x = ld_c<T, CPLX>(col, k), y = ld_c<T, CPLX>(col, p);
          st_c<T, CPLX>(col, k, y);
          st_c<T, CPLX>(col, p, x);
        }
      } else if (j == k) {
        for (int i = k + tid; i < n; i += bd) {
          if (i == k) {
            st_c<T, CPLX>(col, k, pv);
          } else {
            const C2<T> v = i == p ? ck : ldcg_c<T, CPLX>(cb, i);
            st_c<T, CPLX>(col, i, mul_c<T, CPLX>(v, inv));
          }
        }
      } else {
        const C2<T> uk = ld_c<T, CPLX>(col, p);   // becomes row k of U
        const C2<T> old = ld_c<T, CPLX>(col, k);  // moves to row p
        __syncthreads();                          // both read before any write of this column
        for (int i = k + tid; i < n; i += bd) {
          if (i == k) {
            st_c<T, CPLX>(col, k, uk);
            continue;
          }
          const C2<T> v = i == p ? old : ld_c<T, CPLX>(col, i);
          const C2<T> l = mul_c<T, CPLX>(i == p ? ck : ldcg_c<T, CPLX>(cb, i), inv);
          const C2<T> t = mul_c<T, CPLX>(l, uk);
          const C2<T> r{v.re - t.re, v.im - t.im};
          st_c<T, CPLX>(col, i, r);
          if (j == k + 1) st_c<T, CPLX>(cnext, i, r);
        }
      }
    }
    if (blockIdx.x == 0 && tid == 0) ipiv[k] = p;
    grid.sync();
  }
}

template <class T, bool CPLX>
__global__ void __launch_bounds__(DLU_THREADS) k_dlu_solve(int n, const T* __restrict__ M, const int* __restrict__ ipiv,
                                                            const T* __restrict__ rhs, int ld_rhs, T* __restrict__ sol,
                                                            int ld_sol) {
  constexpr int E = CPLX ? 2 : 1;
  extern __shared__ __align__(16) unsigned char dlu_sm[];
  T* x = reinterpret_cast<T*>(dlu_sm);
  const int c = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < n; i += bd)
    for (int e = 0; e < E; ++e) x[(size_t)i * E + e] = rhs[(size_t)i * ld_rhs + (size_t)c * E + e];
  __syncthreads();
  if (tid == 0)
    for (int k = 0; k < n; ++k) {
      const int p = ipiv[k];
      if (p != k)
        for (int e = 0; e < E; ++e) {
          const T t = x[(size_t)k * E + e];
          x[(size_t)k * E + e] = x[(size_t)p * E + e];
          x[(size_t)p * E + e] = t;
        }
    }
  __syncthreads();
  // L y = P b (unit diagonal)
  for (int k = 0; k + 1 < n; ++k) {
    const T* col = M + (size_t)k * n * E;
    const C2<T> xk = ld_c<T, CPLX>(x, k);
    for (int i = k + 1 + tid; i < n; i += bd) {
      const C2<T> t = mul_c<T, CPLX>(ld_c<T, CPLX>(col, i), xk);
      const C2<T> xi = ld_c<T, CPLX>(x, i);
      st_c<T, CPLX>(x, i, C2<T>{xi.re - t.re, xi.im - t.im});
    }
    __syncthreads();
  }
  // U x = y; x_k goes straight to the output, the update uses it from registers
  for (int k = n - 1; k >= 0; --k) {
    const T* col = M + (size_t)k * n * E;
    const C2<T> d = ld_c<T, CPLX>(col, k);
    const C2<T> xk = mul_c<T, CPLX>(ld_c<T, CPLX>(x, k), CPLX ? c2inv(d) : C2<T>{T(1) / d.re, T(0)});
    if (tid == 0)
      for (int e = 0; e < E; ++e) sol[(size_t)k * ld_sol + (size_t)c * E + e] = e == 0 ? xk.re : xk.im;
    for (int i = tid; i < k; i += bd) {
      const C2<T> t = mul_c<T, CPLX>(ld_c<T, CPLX>(col, i), xk);
      const C2<T> xi = ld_c<T, CPLX>(x, i);
      st_c<T, CPLX>(x, i, C2<T>{xi.re - t.re, xi.im - t.im});
    }
    __syncthreads();
  }
}

template <class T, bool CPLX>
void dlu_run(const care_op& op, cd sigma, const T* rhs, int ld_rhs, T* sol, int ld_sol, int ncol,
             const DluWork<T>& w, cudaStream_t s) {
  constexpr int E = CPLX ? 2 : 1;
  const int n = op.n;
  CARE_CUDA(cudaMemsetAsync(w.M, 0, sizeof(T) * (size_t)n * n * E, s));
  CARE_CUDA(cudaMemsetAsync(w.info, 0, sizeof(int), s));
  k_dlu_form<T, CPLX><<<std::max(1, std::min(device_sms() * 4, (n + 255) / 256)), 256, 0, s>>>(
      n, op.rowptr_t, op.colind_t, op.val64_t, sigma.re, sigma.im, w.M);
  CARE_LAUNCH();
  {
    int per_sm = 0;
    CARE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dlu_factor<T, CPLX>, DLU_THREADS, 0));
    CARE_REQUIRE(per_sm >= 1, CARE_ERR_CUDA, "dense LU: factor kernel cannot be resident");
    const int grid = std::max(1, std::min(n, device_sms() * std::min(per_sm, 2)));
    int nn = n;
    T* Mp = w.M;
    int* ip = w.ipiv;
    T* cb = w.cbuf;
    int* inf = w.info;
    void* args[] = {(void*)&nn, (void*)&Mp, (void*)&ip, (void*)&cb, (void*)&inf};
    CARE_CUDA(cudaLaunchCooperativeKernel((const void*)k_dlu_factor<T, CPLX>, dim3(grid), dim3(DLU_THREADS), args, 0, s));
    count_launch();
  }
  const size_t smem = sizeof(T) * (size_t)n * E;
  if (smem > 48 * 1024)
    CARE_CUDA(cudaFuncSetAttribute(k_dlu_solve<T, CPLX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_dlu_solve<T, CPLX><<<ncol, DLU_THREADS, smem, s>>>(n, w.M, w.ipiv, rhs, ld_rhs, sol, ld_sol);
  CARE_LAUNCH();
}

}  // namespace

template <class T>
DluWork<T> dlu_alloc(Arena& ar, int n) {
  CARE_REQUIRE(n >= 0 && n <= CARE_DENSE_LU_MAX_N, CARE_ERR_INVALID_ARG,
               "dense LU shifted solves: n exceeds CARE_DENSE_LU_MAX_N");
  DluWork<T> w;
  w.n = n;
  w.M = ar.get<T>((size_t)n * n * 2);
  w.ipiv = ar.get<int>((size_t)std::max(n, 1));
  w.cbuf = ar.get<T>((size_t)4 * std::max(n, 1));
  w.info = ar.get<int>(1);
  return w;
}
template DluWork<float> dlu_alloc<float>(Arena&, int);
template DluWork<double> dlu_alloc<double>(Arena&, int);

template <class T>
KrylovResult dense_lu_solve(const care_op& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol, int ld_sol,
                            int cols, const DluWork<T>& w, cudaStream_t s) {
  KrylovResult r;
  CARE_REQUIRE(w.M != nullptr && op.n <= w.n, CARE_ERR_INVALID_ARG, "dense LU: workspace missing or too small");
  CARE_REQUIRE(!cplx || cols % 2 == 0, CARE_ERR_INVALID_ARG, "dense LU: odd complex width");
  if (op.n == 0 || cols == 0) return r;
  const int ncol = cplx ? cols / 2 : cols;
  if (cplx) dlu_run<T, true>(op, sigma, rhs, ld_rhs, sol, ld_sol, ncol, w, s);
  else dlu_run<T, false>(op, sigma, rhs, ld_rhs, sol, ld_sol, ncol, w, s);
  int info = 0;
  CARE_CUDA(cudaMemcpyAsync(&info, w.info, sizeof(int), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  r.iters = 1;
  r.unconverged = info != 0 ? cols : 0;
  return r;
}
template KrylovResult dense_lu_solve<float>(const care_op&, cd, bool, const float*, int, float*, int, int,
                                            const DluWork<float>&, cudaStream_t);
template KrylovResult dense_lu_solve<double>(const care_op&, cd, bool, const double*, int, double*, int, int,
                                             const DluWork<double>&, cudaStream_t);

}  // namespace care
