// CSR SpMM with fused shift and per-column dot products, and the block
// BiCGStab solver for the shifted systems M_p X = W, M_p = (A + p I)^T
// (Section 4: the dominant cost of NLR-ADI and LR-ADI is applying M_p^{-1} to
// block right-hand sides).
//
// Layout: blocks are row-major n x w with a leading dimension ld (reals), so a
// CSR row of A^T gathers whole contiguous rows of X.  A row is handled by TPR
// threads, each owning NVPT 16-byte vectors (float4 / double2) of the row;
// complex blocks interleave (re, im) so a vector holds whole complex entries.
// Grids are a multiple of the SM count and grid-stride over rows.
//
// Dot products are accumulated per thread in the working precision, combined
// per CTA in FP64 in a fixed order, written as per-CTA partials, and summed in
// a fixed order by the last CTA to finish (threadfence reduction), which then
// updates the per-column recurrence scalars.  Results are bitwise reproducible.
#include <cmath>

#include "krylov.cuh"

namespace care {

OpT<double> op64(const care_op& o) {
  OpT<double> r;
  r.n = o.n; r.nnz = o.nnz; r.rp = o.rowptr_t; r.ci = o.colind_t; r.val = o.val64_t; r.diag = o.diag64;
  r.diag_const = o.diag_const != 0;
  return r;
}
OpT<float> op32(const care_op& o) {
  OpT<float> r;
  r.n = o.n; r.nnz = o.nnz; r.rp = o.rowptr_t; r.ci = o.colind_t; r.val = o.val32_t; r.diag = o.diag32;
  r.diag_const = o.diag_const != 0;
  return r;
}

enum FinMode { FIN_NONE = 0, FIN_INIT = 1, FIN_ALPHA = 2, FIN_OMEGA = 3, FIN_RHO = 4 };

template <int TPR>
struct RowIter {
  int lane_v;
  long row, stride;
  __device__ RowIter() {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    constexpr int RPW = 32 / TPR;
    lane_v = lane % TPR;
    row = (long)(tid >> 5) * RPW + lane / TPR;
    stride = (long)(gridDim.x * blockDim.x / 32) * RPW;
  }
};

// ---------------------------------------------------------------- dots ----
struct DotOut {
  double* partial;  // [gridDim.x][ndot * w]
  double* out;      // [ndot * w]
  unsigned* counter;
};

// Per-CTA combine of the thread accumulators (fixed order), partial write,
// and the last CTA's fixed-order sum over CTAs.  Returns true in the last CTA
// (all its threads) after `out` is complete.
template <class T, int TPR, int NVPT, int NDOT>
__device__ bool dot_reduce(const T (&acc)[NDOT][NVPT * (16 / sizeof(T))], int w, const DotOut& d) {
  constexpr int VEC = 16 / sizeof(T), NS = NVPT * VEC;
  __shared__ double sm[kBlock * NDOT * NS];
  __shared__ bool s_last;
#pragma unroll
  for (int q = 0; q < NDOT; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) sm[(threadIdx.x * NDOT + q) * NS + e] = (double)acc[q][e];
  __syncthreads();
  const int items = NDOT * w;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it / w, slot = it % w;
    const int v = slot / VEC, e = slot % VEC;
    const int lv = v % TPR, k = v / TPR;
    double sum = 0.0;
    for (int t = lv; t < kBlock; t += TPR) sum += sm[(t * NDOT + q) * NS + k * VEC + e];
    d.partial[(size_t)blockIdx.x * items + it] = sum;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned prev = atomicAdd(d.counter, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  const int G = gridDim.x;
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    int g = 0;
    for (; g + 3 < G; g += 4) {
      s0 += __ldcg(d.partial + (size_t)(g + 0) * items + it);
      s1 += __ldcg(d.partial + (size_t)(g + 1) * items + it);
      s2 += __ldcg(d.partial + (size_t)(g + 2) * items + it);
      s3 += __ldcg(d.partial + (size_t)(g + 3) * items + it);
    }
    for (; g < G; ++g) s0 += __ldcg(d.partial + (size_t)g * items + it);
    d.out[it] = (s0 + s1) + (s2 + s3);
  }
  if (threadIdx.x == 0) *d.counter = 0u;
  __threadfence();
  __syncthreads();
  return true;
}

// Accumulate conj(a) * b over one vector into acc (complex: slot pairs hold re, im).
template <class T, bool CPLX, int VEC>
__device__ __forceinline__ void acc_dot(T* acc, const T (&a)[VEC], const T (&b)[VEC]) {
  if constexpr (CPLX) {
#pragma unroll
    for (int q = 0; q < VEC; q += 2) {
      acc[q] += a[q] * b[q] + a[q + 1] * b[q + 1];
      acc[q + 1] += a[q] * b[q + 1] - a[q + 1] * b[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < VEC; ++q) acc[q] += a[q] * b[q];
  }
}

// Last-CTA update of the per-column BiCGStab scalars from the reduced dots.
__device__ void kfinalize(int mode, const double* out, int w, bool cplx, KState* st, KHeader* hdr,
                          double tol2) {
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  const int nst = cplx ? w / 2 : w;
  for (int j = threadIdx.x; j < nst; j += blockDim.x) {
    KState q = st[j];
    cd d0 = cplx ? cd{out[2 * j], out[2 * j + 1]} : cd{out[j], 0.0};
    cd d1 = cplx ? cd{out[w + 2 * j], out[w + 2 * j + 1]} : cd{out[w + j], 0.0};
    if (mode == FIN_INIT) {
      q.rho_re = d0.re; q.rho_im = d0.im;
      q.bnorm2 = d1.re; q.rnorm2 = d1.re;
      q.alpha_re = 1; q.alpha_im = 0; q.omega_re = 1; q.omega_im = 0; q.beta_re = 0; q.beta_im = 0;
      q.iters = 0;
      q.flag = (d1.re > 0.0 && isfinite(d1.re)) ? 0 : (d1.re == 0.0 ? 1 : 2);
    } else if (q.flag == 0) {
      if (mode == FIN_ALPHA) {
        if (!(d0.re != 0.0 || d0.im != 0.0) || !isfinite(d0.re) || !isfinite(d0.im)) {
          q.flag = 2;
        } else {
          cd a = cdivz(cd{q.rho_re, q.rho_im}, d0);
          q.alpha_re = a.re; q.alpha_im = a.im;
        }
      } else if (mode == FIN_OMEGA) {
        // omega = <t, s> / <t, t>;  d0 = <s, t> = conj(<t, s>), d1 = <t, t>
        if (d1.re > 0.0 && isfinite(d1.re)) {
          q.omega_re = d0.re / d1.re; q.omega_im = -d0.im / d1.re;
        } else {
          q.omega_re = 0; q.omega_im = 0;
        }
      } else if (mode == FIN_RHO) {
        q.iters += 1;
        q.rnorm2 = d1.re;
        if (!isfinite(d1.re)) {
          q.flag = 2;
        } else if (d1.re <= tol2 * q.bnorm2) {
          q.flag = 1;
        } else {
          const bool om0 = (q.omega_re == 0.0 && q.omega_im == 0.0);
          const bool rh0 = (q.rho_re == 0.0 && q.rho_im == 0.0);
          if (om0 || rh0 || (d0.re == 0.0 && d0.im == 0.0)) {
            q.flag = 2;
          } else {
            cd b = cmul(cdivz(d0, cd{q.rho_re, q.rho_im}), cdivz(cd{q.alpha_re, q.alpha_im}, cd{q.omega_re, q.omega_im}));
            q.beta_re = b.re; q.beta_im = b.im;
            q.rho_re = d0.re; q.rho_im = d0.im;
          }
        }
      }
    }
    st[j] = q;
    if (q.flag == 0) atomicAdd(&s_active, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0 && (mode == FIN_INIT || mode == FIN_RHO)) hdr->n_active = s_active;
}

// --------------------------------------------------------------- SpMM -----
template <class T>
struct SpmmArgs {
  long n;
  const int* rp;
  const int* ci;
  const T* av;
  const T* X;
  int ldx;
  T* Y;
  int ldy;
  int nvec;  // 16-byte vectors per row processed
  double sre, sim;
  const T* w0;  // dot operands (row-major, ldy); nullptr = Y itself
  const T* w1;
  DotOut dots;
  int mode;
  KState* st;
  KHeader* hdr;
  double tol2;
};

template <class T, int TPR, int NVPT, bool CPLX, int NDOT>
__global__ void __launch_bounds__(kBlock) k_spmm(SpmmArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T), NS = NVPT * VEC;
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  RowIter<TPR> it;
  T acc[ND][NS];
#pragma unroll
  for (int q = 0; q < ND; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) acc[q][e] = T(0);
  const T sre = (T)a.sre, sim = (T)a.sim;
  for (long row = it.row; row < a.n; row += it.stride) {
    const int s = __ldg(a.rp + row), e = __ldg(a.rp + row + 1);
    T y[NVPT][VEC];
#pragma unroll
    for (int k = 0; k < NVPT; ++k)
#pragma unroll
      for (int q = 0; q < VEC; ++q) y[k][q] = T(0);
    for (int j = s; j < e; ++j) {
      const int c = __ldg(a.ci + j);
      const T av = __ldg(a.av + j);
      const T* xr = a.X + (size_t)c * a.ldx;
#pragma unroll
      for (int k = 0; k < NVPT; ++k) {
        const int v = it.lane_v + k * TPR;
        if (v < a.nvec) {
          T x[VEC];
          vload(xr + v * VEC, x);
#pragma unroll
          for (int q = 0; q < VEC; ++q) y[k][q] = fma(av, x[q], y[k][q]);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v < a.nvec) {
        T xi[VEC];
        vload(a.X + (size_t)row * a.ldx + v * VEC, xi);
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            const T yr = y[k][q] + sre * xi[q] - sim * xi[q + 1];
            const T yi = y[k][q + 1] + sre * xi[q + 1] + sim * xi[q];
            y[k][q] = yr;
            y[k][q + 1] = yi;
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) y[k][q] = fma(sre, xi[q], y[k][q]);
        }
        vstore(a.Y + (size_t)row * a.ldy + v * VEC, y[k]);
        if constexpr (NDOT > 0) {
          T w[VEC];
          if (a.w0) vload(a.w0 + (size_t)row * a.ldy + v * VEC, w);
          else
#pragma unroll
            for (int q = 0; q < VEC; ++q) w[q] = y[k][q];
          acc_dot<T, CPLX, VEC>(&acc[0][k * VEC], w, y[k]);
        }
        if constexpr (NDOT > 1) {
          T w[VEC];
          if (a.w1) vload(a.w1 + (size_t)row * a.ldy + v * VEC, w);
          else
#pragma unroll
            for (int q = 0; q < VEC; ++q) w[q] = y[k][q];
          acc_dot<T, CPLX, VEC>(&acc[1][k * VEC], w, y[k]);
        }
      }
    }
  }
  if constexpr (NDOT > 0) {
    if (dot_reduce<T, TPR, NVPT, NDOT>(acc, a.nvec * VEC, a.dots))
      kfinalize(a.mode, a.dots.out, a.nvec * VEC, CPLX, a.st, a.hdr, a.tol2);
  }
}

template <class T, int NDOT, bool CPLX>
static void launch_spmm(const SpmmArgs<T>& a, cudaStream_t s) {
  const int nv = a.nvec;
  int tpr = tpr_for(nv);
  const int nvpt = (nv + 31) / 32;
  const int grid = grid_rows(a.n, tpr);
#define CARE_SPMM_CASE(TP, NV)                                                          \
  if (tpr == TP && nvpt == NV) {                                                        \
    k_spmm<T, TP, NV, CPLX, NDOT><<<grid, kBlock, 0, s>>>(a);                           \
    CARE_LAUNCH();                                                                      \
    return;                                                                             \
  }
  CARE_SPMM_CASE(1, 1) CARE_SPMM_CASE(2, 1) CARE_SPMM_CASE(4, 1) CARE_SPMM_CASE(8, 1)
  CARE_SPMM_CASE(16, 1) CARE_SPMM_CASE(32, 1) CARE_SPMM_CASE(32, 2)
#undef CARE_SPMM_CASE
  CARE_THROW(CARE_ERR_INVALID_ARG, "spmm: block too wide");
}

template <class T>
void spmm(const OpT<T>& op, cd sigma, bool cplx, const T* X, int ldx, T* Y, int ldy, int cols,
          cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T);
  CARE_REQUIRE(ldx % VEC == 0 && ldy % VEC == 0, CARE_ERR_INVALID_ARG, "spmm: ld not a vector multiple");
  CARE_REQUIRE(((uintptr_t)X % 16) == 0 && ((uintptr_t)Y % 16) == 0, CARE_ERR_INVALID_ARG,
               "spmm: blocks must be 16-byte aligned");
  CARE_REQUIRE(!cplx || cols % 2 == 0, CARE_ERR_INVALID_ARG, "spmm: odd complex width");
  if (op.n == 0 || cols == 0) return;
  // process in chunks of <= kMaxRealCols reals (64 vectors FP64 / 32 FP32)
  const int chunk = kMaxRealCols;
  for (int c0 = 0; c0 < cols; c0 += chunk) {
    const int w = (cols - c0 < chunk) ? cols - c0 : chunk;
    SpmmArgs<T> a{};
    a.n = op.n; a.rp = op.rp; a.ci = op.ci; a.av = op.val;
    a.X = X + c0; a.ldx = ldx; a.Y = Y + c0; a.ldy = ldy;
    a.nvec = (w + VEC - 1) / VEC;
    a.sre = sigma.re; a.sim = sigma.im;
    if (cplx) launch_spmm<T, 0, true>(a, s);
    else launch_spmm<T, 0, false>(a, s);
  }
}
template void spmm<float>(const OpT<float>&, cd, bool, const float*, int, float*, int, int, cudaStream_t);
template void spmm<double>(const OpT<double>&, cd, bool, const double*, int, double*, int, int, cudaStream_t);

// ----------------------------------------------------- BiCGStab kernels ---
template <class T>
struct KArgs {
  long n;
  int ld;    // row stride of the internal blocks (reals)
  int nvec;  // vectors per row
  T *X, *R, *Rh, *P, *V, *S, *Tt, *Ph, *Sh;
  const T* Dinv;  // row-wise 1/(a_ii + sigma): 1 real or 2 reals (complex) per row
  const T* rhs;
  int ld_rhs;
  T* sol;
  int ld_sol;
  int cols;  // valid real columns (rhs / sol width)
  KState* st;
  KHeader* hdr;
  DotOut dots;
  double tol2;
};

// scalar of column slot q of vector v (complex: pairs share one state entry)
template <bool CPLX>
__device__ __forceinline__ int state_index(int slot) { return CPLX ? slot / 2 : slot; }

// y = a * x (complex multiply on interleaved pairs when CPLX)
template <class T, bool CPLX, int VEC>
__device__ __forceinline__ void scal_mul(T (&y)[VEC], const cd* a, const T (&x)[VEC]) {
  if constexpr (CPLX) {
#pragma unroll
    for (int q = 0; q < VEC; q += 2) {
      const cd s = a[q / 2];
      y[q] = (T)s.re * x[q] - (T)s.im * x[q + 1];
      y[q + 1] = (T)s.re * x[q + 1] + (T)s.im * x[q];
    }
  } else {
#pragma unroll
    for (int q = 0; q < VEC; ++q) y[q] = (T)a[q].re * x[q];
  }
}

template <class T, bool CPLX, int VEC>
__device__ __forceinline__ void apply_dinv(T (&y)[VEC], const T* dinv, long row, const T (&x)[VEC]) {
  if constexpr (CPLX) {
    const T dr = dinv[2 * row], di = dinv[2 * row + 1];
#pragma unroll
    for (int q = 0; q < VEC; q += 2) {
      y[q] = dr * x[q] - di * x[q + 1];
      y[q + 1] = dr * x[q + 1] + di * x[q];
    }
  } else {
    const T d = dinv[row];
#pragma unroll
    for (int q = 0; q < VEC; ++q) y[q] = d * x[q];
  }
}

// Load the per-column scalars a thread needs once (its columns never change).
template <bool CPLX, int VEC, int NVPT, int TPR>
struct ThreadCols {
  static constexpr int NC = CPLX ? VEC / 2 : VEC;
  cd s0[NVPT][NC], s1[NVPT][NC];
  bool act[NVPT][NC];
};

// init: r = rhs (zero beyond cols), rhat = r, x = p = v = 0; dots <rhat, r>, <r, r>
template <class T, int TPR, int NVPT, bool CPLX, bool PREC>
__global__ void __launch_bounds__(kBlock) k_bicg_init(KArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T), NS = NVPT * VEC;
  RowIter<TPR> it;
  T acc[2][NS];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) acc[q][e] = T(0);
  for (long row = it.row; row < a.n; row += it.stride) {
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v >= a.nvec) continue;
      T r[VEC], z[VEC];
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const int c = v * VEC + q;
        r[q] = (c < a.cols) ? a.rhs[(size_t)row * a.ld_rhs + c] : T(0);
        z[q] = T(0);
      }
      const size_t off = (size_t)row * a.ld + v * VEC;
      vstore(a.R + off, r);
      vstore(a.Rh + off, r);
      vstore(a.X + off, z);
      vstore(a.P + off, z);
      vstore(a.V + off, z);
      acc_dot<T, CPLX, VEC>(&acc[0][k * VEC], r, r);
      acc_dot<T, CPLX, VEC>(&acc[1][k * VEC], r, r);
    }
  }
  if (dot_reduce<T, TPR, NVPT, 2>(acc, a.nvec * VEC, a.dots))
    kfinalize(FIN_INIT, a.dots.out, a.nvec * VEC, CPLX, a.st, a.hdr, a.tol2);
}

// p = r + beta (p - omega v);  ph = Dinv p
template <class T, int TPR, int NVPT, bool CPLX, bool PREC>
__global__ void __launch_bounds__(kBlock) k_bicg_p(KArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int NC = CPLX ? VEC / 2 : VEC;
  RowIter<TPR> it;
  cd beta[NVPT][NC], omega[NVPT][NC];
  bool act[NVPT][NC];
#pragma unroll
  for (int k = 0; k < NVPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int v = it.lane_v + k * TPR;
      const int j = v * NC + c;
      act[k][c] = false;
      if (v < a.nvec) {
        const KState& q = a.st[j];
        act[k][c] = q.flag == 0;
        beta[k][c] = cd{q.beta_re, q.beta_im};
        omega[k][c] = cd{q.omega_re, q.omega_im};
      }
    }
  for (long row = it.row; row < a.n; row += it.stride) {
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v >= a.nvec) continue;
      const size_t off = (size_t)row * a.ld + v * VEC;
      T r[VEC], p[VEC], vv[VEC], t1[VEC], t2[VEC];
      vload(a.R + off, r);
      vload(a.P + off, p);
      vload(a.V + off, vv);
      scal_mul<T, CPLX, VEC>(t1, omega[k], vv);
#pragma unroll
      for (int q = 0; q < VEC; ++q) t1[q] = p[q] - t1[q];
      scal_mul<T, CPLX, VEC>(t2, beta[k], t1);
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const int c = CPLX ? q / 2 : q;
        if (act[k][c]) p[q] = r[q] + t2[q];
      }
      vstore(a.P + off, p);
      if constexpr (PREC) {
        T ph[VEC];
        apply_dinv<T, CPLX, VEC>(ph, a.Dinv, row, p);
        vstore(a.Ph + off, ph);
      }
    }
  }
}

// s = r - alpha v;  sh = Dinv s
template <class T, int TPR, int NVPT, bool CPLX, bool PREC>
__global__ void __launch_bounds__(kBlock) k_bicg_s(KArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int NC = CPLX ? VEC / 2 : VEC;
  RowIter<TPR> it;
  cd alpha[NVPT][NC];
  bool act[NVPT][NC];
#pragma unroll
  for (int k = 0; k < NVPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int v = it.lane_v + k * TPR;
      act[k][c] = false;
      if (v < a.nvec) {
        const KState& q = a.st[v * NC + c];
        act[k][c] = q.flag == 0;
        alpha[k][c] = act[k][c] ? cd{q.alpha_re, q.alpha_im} : cd{0.0, 0.0};
      }
    }
  for (long row = it.row; row < a.n; row += it.stride) {
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v >= a.nvec) continue;
      const size_t off = (size_t)row * a.ld + v * VEC;
      T r[VEC], vv[VEC], t1[VEC];
      vload(a.R + off, r);
      vload(a.V + off, vv);
      scal_mul<T, CPLX, VEC>(t1, alpha[k], vv);
#pragma unroll
      for (int q = 0; q < VEC; ++q) r[q] = r[q] - t1[q];
      vstore(a.S + off, r);
      if constexpr (PREC) {
        T sh[VEC];
        apply_dinv<T, CPLX, VEC>(sh, a.Dinv, row, r);
        vstore(a.Sh + off, sh);
      }
    }
  }
}

// x += alpha ph + omega sh;  r = s - omega t;  dots <rhat, r>, <r, r>
template <class T, int TPR, int NVPT, bool CPLX, bool PREC>
__global__ void __launch_bounds__(kBlock) k_bicg_xr(KArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T), NS = NVPT * VEC;
  constexpr int NC = CPLX ? VEC / 2 : VEC;
  RowIter<TPR> it;
  cd alpha[NVPT][NC], omega[NVPT][NC];
  bool act[NVPT][NC];
#pragma unroll
  for (int k = 0; k < NVPT; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int v = it.lane_v + k * TPR;
      act[k][c] = false;
      alpha[k][c] = cd{0.0, 0.0};
      omega[k][c] = cd{0.0, 0.0};
      if (v < a.nvec) {
        const KState& q = a.st[v * NC + c];
        act[k][c] = q.flag == 0;
        if (act[k][c]) {
          alpha[k][c] = cd{q.alpha_re, q.alpha_im};
          omega[k][c] = cd{q.omega_re, q.omega_im};
        }
      }
    }
  T acc[2][NS];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) acc[q][e] = T(0);
  for (long row = it.row; row < a.n; row += it.stride) {
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v >= a.nvec) continue;
      const size_t off = (size_t)row * a.ld + v * VEC;
      T x[VEC], ph[VEC], sh[VEC], s[VEC], t[VEC], rh[VEC], t1[VEC], t2[VEC], r[VEC];
      vload(a.X + off, x);
      vload((PREC ? a.Ph : a.P) + off, ph);
      vload(a.S + off, s);
      if constexpr (PREC) vload(a.Sh + off, sh);
      else
#pragma unroll
        for (int q = 0; q < VEC; ++q) sh[q] = s[q];
      vload(a.Tt + off, t);
      vload(a.Rh + off, rh);
      scal_mul<T, CPLX, VEC>(t1, alpha[k], ph);
      scal_mul<T, CPLX, VEC>(t2, omega[k], sh);
#pragma unroll
      for (int q = 0; q < VEC; ++q) x[q] = x[q] + t1[q] + t2[q];
      scal_mul<T, CPLX, VEC>(t1, omega[k], t);
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        const int c = CPLX ? q / 2 : q;
        r[q] = act[k][c] ? s[q] - t1[q] : T(0);
      }
      vstore(a.X + off, x);
      bool any = false;
#pragma unroll
      for (int c = 0; c < NC; ++c) any |= act[k][c];
      if (any) {
        // inactive columns keep their last residual (r is not re-read for them)
        T rold[VEC];
        vload(a.R + off, rold);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          const int c = CPLX ? q / 2 : q;
          if (!act[k][c]) r[q] = rold[q];
        }
        vstore(a.R + off, r);
      }
      acc_dot<T, CPLX, VEC>(&acc[0][k * VEC], rh, r);
      acc_dot<T, CPLX, VEC>(&acc[1][k * VEC], r, r);
    }
  }
  if (dot_reduce<T, TPR, NVPT, 2>(acc, a.nvec * VEC, a.dots))
    kfinalize(FIN_RHO, a.dots.out, a.nvec * VEC, CPLX, a.st, a.hdr, a.tol2);
}

// sol = x (valid columns only)
template <class T>
__global__ void k_copy_out(KArgs<T> a) {
  const long total = a.n * (long)a.cols;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
    const long row = i / a.cols;
    const int c = (int)(i % a.cols);
    a.sol[(size_t)row * a.ld_sol + c] = a.X[(size_t)row * a.ld + c];
  }
}

// Dinv[row] = 1 / (a_ii + sigma)  (complex when sigma is complex)
template <class T>
__global__ void k_dinv(long n, const T* diag, double sre, double sim, bool cplx, T* dinv) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double dr = (double)diag[i] + sre;
    if (cplx) {
      const cd z = cdivz(cd{1.0, 0.0}, cd{dr, sim});
      dinv[2 * i] = (T)z.re;
      dinv[2 * i + 1] = (T)z.im;
    } else {
      dinv[i] = (T)(1.0 / dr);
    }
  }
}

template <class T>
KrylovWork<T> krylov_alloc(Arena& ar, int n, bool jacobi) {
  KrylovWork<T> w;
  const size_t blk = (size_t)n * kMaxRealCols;
  w.n = n;
  w.X = ar.get<T>(blk); w.R = ar.get<T>(blk); w.Rh = ar.get<T>(blk); w.P = ar.get<T>(blk);
  w.V = ar.get<T>(blk); w.S = ar.get<T>(blk); w.Tt = ar.get<T>(blk);
  if (jacobi) {
    w.Ph = ar.get<T>(blk); w.Sh = ar.get<T>(blk); w.Dinv = ar.get<T>((size_t)2 * n);
  }
  w.st = ar.get<KState>(kMaxRealCols);
  w.hdr = ar.get<KHeader>(1);
  w.partial = ar.get<double>((size_t)device_sms() * 8 * 2 * kMaxRealCols);
  w.out = ar.get<double>(2 * kMaxRealCols);
  return w;
}
template KrylovWork<float> krylov_alloc<float>(Arena&, int, bool);
template KrylovWork<double> krylov_alloc<double>(Arena&, int, bool);

template <class T, int TPR, int NVPT, bool CPLX, bool PREC>
static KrylovResult run_bicg(const OpT<T>& op, cd sigma, KArgs<T> a, int maxit, int grid,
                             cudaStream_t s) {
  KrylovResult res;
  SpmmArgs<T> sp{};
  sp.n = op.n; sp.rp = op.rp; sp.ci = op.ci; sp.av = op.val; sp.ldx = a.ld; sp.ldy = a.ld;
  sp.nvec = a.nvec; sp.sre = sigma.re; sp.sim = sigma.im; sp.dots = a.dots; sp.st = a.st;
  sp.hdr = a.hdr; sp.tol2 = a.tol2;
  k_bicg_init<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  const int poll = 4;
  KHeader h{};
  int it = 0;
  CARE_CUDA(cudaMemcpyAsync(&h, a.hdr, sizeof(KHeader), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  if (h.n_active == 0) return res;
  for (it = 0; it < maxit; ++it) {
    k_bicg_p<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
    CARE_LAUNCH();
    sp.X = PREC ? a.Ph : a.P; sp.Y = a.V; sp.w0 = a.Rh; sp.w1 = nullptr; sp.mode = FIN_ALPHA;
    k_spmm<T, TPR, NVPT, CPLX, 1><<<grid, kBlock, 0, s>>>(sp);
    CARE_LAUNCH();
    k_bicg_s<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
    CARE_LAUNCH();
    sp.X = PREC ? a.Sh : a.S; sp.Y = a.Tt; sp.w0 = a.S; sp.w1 = nullptr; sp.mode = FIN_OMEGA;
    k_spmm<T, TPR, NVPT, CPLX, 2><<<grid, kBlock, 0, s>>>(sp);
    CARE_LAUNCH();
    k_bicg_xr<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
    CARE_LAUNCH();
    res.spmm += 2;
    if ((it + 1) % poll == 0 || it + 1 == maxit) {
      CARE_CUDA(cudaMemcpyAsync(&h, a.hdr, sizeof(KHeader), cudaMemcpyDeviceToHost, s));
      CARE_CUDA(cudaStreamSynchronize(s));
      if (h.n_active == 0) {
        ++it;
        break;
      }
    }
  }
  res.iters = it;
  return res;
}

template <class T>
KrylovResult krylov_bicgstab(const OpT<T>& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol,
                             int ld_sol, int cols, double tol, int maxit, bool jacobi,
                             KrylovWork<T>& w, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T);
  CARE_REQUIRE(cols <= kMaxRealCols && cols > 0, CARE_ERR_INVALID_ARG, "krylov: bad width");
  CARE_REQUIRE(!cplx || cols % 2 == 0, CARE_ERR_INVALID_ARG, "krylov: odd complex width");
  const bool prec = jacobi && !op.diag_const && w.Ph != nullptr;
  KArgs<T> a{};
  a.n = op.n;
  a.ld = pad_ld<T>(cols);
  a.nvec = a.ld / VEC;
  a.X = w.X; a.R = w.R; a.Rh = w.Rh; a.P = w.P; a.V = w.V; a.S = w.S; a.Tt = w.Tt;
  a.Ph = w.Ph; a.Sh = w.Sh; a.Dinv = w.Dinv;
  a.rhs = rhs; a.ld_rhs = ld_rhs; a.sol = sol; a.ld_sol = ld_sol; a.cols = cols;
  a.st = w.st; a.hdr = w.hdr;
  a.dots = DotOut{w.partial, w.out, &w.hdr->counter};
  a.tol2 = tol * tol;
  const int tpr = tpr_for(a.nvec);
  const int nvpt = (a.nvec + 31) / 32;
  const int grid = grid_rows(op.n, tpr);
  CARE_REQUIRE(grid <= device_sms() * 8, CARE_ERR_INVALID_ARG, "krylov: grid exceeds partial buffer");
  // reduction counter and flags start from zero for every solve
  CARE_CUDA(cudaMemsetAsync(w.hdr, 0, sizeof(KHeader), s));
  if (prec) {
    k_dinv<T><<<device_sms() * 4, kBlock, 0, s>>>(op.n, op.diag, sigma.re, sigma.im, cplx, w.Dinv);
    CARE_LAUNCH();
  }
  KrylovResult r;
#define CARE_BICG_CASE(TP, NV)                                                               \
  if (tpr == TP && nvpt == NV) {                                                             \
    if (cplx) r = prec ? run_bicg<T, TP, NV, true, true>(op, sigma, a, maxit, grid, s)       \
                       : run_bicg<T, TP, NV, true, false>(op, sigma, a, maxit, grid, s);     \
    else r = prec ? run_bicg<T, TP, NV, false, true>(op, sigma, a, maxit, grid, s)           \
                  : run_bicg<T, TP, NV, false, false>(op, sigma, a, maxit, grid, s);         \
    goto done;                                                                               \
  }
  CARE_BICG_CASE(1, 1) CARE_BICG_CASE(2, 1) CARE_BICG_CASE(4, 1) CARE_BICG_CASE(8, 1)
  CARE_BICG_CASE(16, 1) CARE_BICG_CASE(32, 1) CARE_BICG_CASE(32, 2)
#undef CARE_BICG_CASE
  CARE_THROW(CARE_ERR_INVALID_ARG, "krylov: unsupported width");
done:
  k_copy_out<T><<<device_sms() * 4, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  {
    // count unconverged columns (flag != 1 among the valid state entries)
    const int nst = cplx ? cols / 2 : cols;
    std::vector<KState> hs(nst);
    CARE_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(KState) * nst, cudaMemcpyDeviceToHost, s));
    CARE_CUDA(cudaStreamSynchronize(s));
    for (int j = 0; j < nst; ++j)
      if (hs[j].flag != 1) ++r.unconverged;
  }
  return r;
}
template KrylovResult krylov_bicgstab<float>(const OpT<float>&, cd, bool, const float*, int, float*, int,
                                             int, double, int, bool, KrylovWork<float>&, cudaStream_t);
template KrylovResult krylov_bicgstab<double>(const OpT<double>&, cd, bool, const double*, int, double*,
                                              int, int, double, int, bool, KrylovWork<double>&,
                                              cudaStream_t);

}  // namespace care
