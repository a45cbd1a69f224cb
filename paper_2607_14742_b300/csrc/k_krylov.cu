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

#include "dense.cuh"
#include "krylov.cuh"

namespace care {

OpT<double> op64(const care_op& o) {
  OpT<double> r;
  r.n = o.n; r.nnz = o.nnz; r.rp = o.rowptr_t; r.ci = o.colind_t; r.val = o.val64_t; r.diag = o.diag64;
  r.diag_const = o.diag_const != 0;
  r.full_diag = o.full_diag != 0 && o.max_row_nnz <= 32;
  return r;
}
OpT<float> op32(const care_op& o) {
  OpT<float> r;
  r.n = o.n; r.nnz = o.nnz; r.rp = o.rowptr_t; r.ci = o.colind_t; r.val = o.val32_t; r.diag = o.diag32;
  r.rowsum = o.rowsum32_t;
  r.diag_const = o.diag_const != 0;
  r.full_diag = o.full_diag != 0 && o.max_row_nnz <= 32;
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
  constexpr int NWARP = kBlock / 32;
  __shared__ double sm[NWARP * NDOT * TPR * NVPT * VEC];
  __shared__ bool s_last;
  // 1. within each warp, lanes that own the same vector slot are those with equal
  //    lane % TPR: combine them with a fixed xor-shuffle tree (in FP64)
  double v[NDOT][NS];
#pragma unroll
  for (int q = 0; q < NDOT; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) {
      double x = (double)acc[q][e];
#pragma unroll
      for (int off = TPR; off < 32; off <<= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      v[q][e] = x;
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // lanes 0..TPR-1 hold the warp totals for slots (lane + k*TPR)*VEC + e
  if (lane < TPR) {
#pragma unroll
    for (int q = 0; q < NDOT; ++q)
#pragma unroll
      for (int k2 = 0; k2 < NVPT; ++k2)
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const int slot = (lane + k2 * TPR) * VEC + e;
          sm[(warp * NDOT + q) * (TPR * NVPT * VEC) + slot] = v[q][k2 * VEC + e];
        }
  }
  __syncthreads();
  // 2. the CTA total of each item: fixed-order sum over the warps
  const int items = NDOT * w;
  constexpr int SPAN = TPR * NVPT * VEC;  // slots per dot held in shared memory
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int q = it / w, slot = it % w;
    double sum = 0.0;
    if (slot < SPAN)
#pragma unroll
      for (int wp = 0; wp < NWARP; ++wp) sum += sm[(wp * NDOT + q) * SPAN + slot];
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
  // last CTA: TPI threads per item sum strided subsets of the G partials, then a
  // fixed-order tree in shared memory (deterministic for a given grid)
  const int G = gridDim.x;
  int TPI = 1;
  while (TPI * 2 * items <= (int)blockDim.x) TPI *= 2;
  __shared__ double red[kBlock];
  {
    const int t = threadIdx.x;
    const int item = t / TPI, tl = t % TPI;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (item < items) {
      int g = tl;
      for (; g + 3 * TPI < G; g += 4 * TPI) {
        s0 += __ldcg(d.partial + (size_t)g * items + item);
        s1 += __ldcg(d.partial + (size_t)(g + TPI) * items + item);
        s2 += __ldcg(d.partial + (size_t)(g + 2 * TPI) * items + item);
        s3 += __ldcg(d.partial + (size_t)(g + 3 * TPI) * items + item);
      }
      for (; g < G; g += TPI) s0 += __ldcg(d.partial + (size_t)g * items + item);
    }
    red[t] = (s0 + s1) + (s2 + s3);
    __syncthreads();
    for (int w2 = TPI / 2; w2 > 0; w2 >>= 1) {
      if (tl < w2) red[t] += red[t + w2];
      __syncthreads();
    }
    if (item < items && tl == 0) d.out[item] = red[t];
  }
  // items beyond one pass of the block (items > blockDim.x) use one thread each
  for (int it = blockDim.x; it < items; it += blockDim.x) {
    const int item = it + threadIdx.x;
    if (item >= items) continue;
    double s0 = 0.0;
    for (int g = 0; g < G; ++g) s0 += __ldcg(d.partial + (size_t)g * items + item);
    d.out[item] = s0;
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
  const T* rs;  // row sums: difference form  y_i = sum_j a_ij (x_j - x_i) + (s_i + p) x_i
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
  // rows per CTA when > 0: CTA b takes the contiguous rows [b chunk, (b+1) chunk)
  // (its warps interleaved inside), so the neighbours a stencil row gathers were
  // mostly loaded by the same SM moments before; 0: rows grid-stride over warps
  long chunk;
};

// (register budget: the plain FP32 product with one vector per thread keeps 8 CTAs
// per SM resident; the other variants take what they need without spilling)
template <class T, int TPR, int NVPT, bool CPLX, int NDOT>
__global__ void __launch_bounds__(kBlock, (NVPT == 1 && NDOT == 0 && sizeof(T) == 4) ? 8 : 1)
    k_spmm(SpmmArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T), NS = NVPT * VEC;
  constexpr int ND = NDOT > 0 ? NDOT : 1;
  RowIter<TPR> it;
  long row_end = a.n;
  if (a.chunk > 0) {
    constexpr int RPW = 32 / TPR;
    const long r0 = (long)blockIdx.x * a.chunk;
    it.row = r0 + (long)(threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / TPR;
    it.stride = (long)(blockDim.x >> 5) * RPW;
    row_end = r0 + a.chunk < a.n ? r0 + a.chunk : a.n;
  }
  T acc[ND][NS];
#pragma unroll
  for (int q = 0; q < ND; ++q)
#pragma unroll
    for (int e = 0; e < NS; ++e) acc[q][e] = T(0);
  const T sim = (T)a.sim;
  const bool diff = a.rs != nullptr;
  for (long row = it.row; row < row_end; row += it.stride) {
    const int s = __ldg(a.rp + row), e = __ldg(a.rp + row + 1);
    T y[NVPT][VEC], xi[NVPT][VEC];
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
#pragma unroll
      for (int q = 0; q < VEC; ++q) {
        y[k][q] = T(0);
        xi[k][q] = T(0);
      }
      if (v < a.nvec && diff) vload_ro(a.X + (size_t)row * a.ldx + v * VEC, xi[k]);
    }
    // four independent gathers in flight per thread (stencil rows have 5-7 entries),
    // then the remainder one by one; 32 registers keep every warp slot resident
    int j = s;
    for (; j + 3 < e; j += 4) {
      int c[4];
      T av[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = __ldg(a.ci + j + u);
        av[u] = __ldg(a.av + j + u);
      }
#pragma unroll
      for (int k = 0; k < NVPT; ++k) {
        const int v = it.lane_v + k * TPR;
        if (v < a.nvec) {
          T x[4][VEC];
#pragma unroll
          for (int u = 0; u < 4; ++u) vload_ro(a.X + (size_t)c[u] * a.ldx + v * VEC, x[u]);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < VEC; ++q) y[k][q] = fma(av[u], x[u][q] - xi[k][q], y[k][q]);
        }
      }
    }
    for (; j < e; ++j) {
      const int c = __ldg(a.ci + j);
      const T av = __ldg(a.av + j);
      const T* xr = a.X + (size_t)c * a.ldx;
#pragma unroll
      for (int k = 0; k < NVPT; ++k) {
        const int v = it.lane_v + k * TPR;
        if (v < a.nvec) {
          T x[VEC];
          vload_ro(xr + v * VEC, x);
#pragma unroll
          for (int q = 0; q < VEC; ++q) y[k][q] = fma(av, x[q] - xi[k][q], y[k][q]);
        }
      }
    }
    // diagonal term: (s_i + p) in the difference form, p otherwise
    const T dre = (T)a.sre + (diff ? __ldg(a.rs + row) : T(0));
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v < a.nvec) {
        if (!diff) vload_ro(a.X + (size_t)row * a.ldx + v * VEC, xi[k]);
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            const T yr = y[k][q] + dre * xi[k][q] - sim * xi[k][q + 1];
            const T yi = y[k][q + 1] + dre * xi[k][q + 1] + sim * xi[k][q];
            y[k][q] = yr;
            y[k][q + 1] = yi;
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) y[k][q] = fma(dre, xi[k][q], y[k][q]);
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

// Every SpMM launch (standalone and inside the Krylov iterations) takes the thread
// shape of the tuned vectors-per-thread count, with its own grid.
template <class T, int NDOT, bool CPLX>
static void launch_spmm(const SpmmArgs<T>& a, cudaStream_t s) {
  int tpr = 1, nvpt = 1;
  spmm_shape(a.nvec, tuned_spmm_vpt(a.nvec), &tpr, &nvpt);
  const int grid = grid_rows(a.n, tpr);
  SpmmArgs<T> b = a;
  b.chunk = 0;
  if (tuned_spmm_blocked()) {
    const long step = (long)(kBlock / 32) * (32 / tpr);  // rows per pass of a CTA
    b.chunk = ((a.n + grid - 1) / grid + step - 1) / step * step;
  }
#define CARE_SPMM_CASE(TP, NV)                                                          \
  if (tpr == TP && nvpt == NV) {                                                        \
    k_spmm<T, TP, NV, CPLX, NDOT><<<grid, kBlock, 0, s>>>(b);                           \
    CARE_LAUNCH();                                                                      \
    return;                                                                             \
  }
  CARE_SPMM_CASE(1, 1) CARE_SPMM_CASE(2, 1) CARE_SPMM_CASE(4, 1) CARE_SPMM_CASE(8, 1)
  CARE_SPMM_CASE(16, 1) CARE_SPMM_CASE(32, 1) CARE_SPMM_CASE(32, 2)
  CARE_SPMM_CASE(1, 2) CARE_SPMM_CASE(2, 2) CARE_SPMM_CASE(4, 2) CARE_SPMM_CASE(8, 2) CARE_SPMM_CASE(16, 2)
  CARE_SPMM_CASE(1, 3) CARE_SPMM_CASE(2, 3) CARE_SPMM_CASE(4, 3) CARE_SPMM_CASE(8, 3) CARE_SPMM_CASE(16, 3)
  CARE_SPMM_CASE(1, 4) CARE_SPMM_CASE(2, 4) CARE_SPMM_CASE(4, 4) CARE_SPMM_CASE(8, 4) CARE_SPMM_CASE(16, 4)
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
    a.n = op.n; a.rp = op.rp; a.ci = op.ci; a.av = op.val; a.rs = op.rowsum;
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
  // ILU(0) preconditioner
  const int* rp;
  const int* ci;
  const int* dpos;
  const T* F;
  T *Y1, *Y2, *Y3;
  int tri_sweeps;
  // exact ILU(0) application (precond CARE_PRECOND_ILU0_EXACT)
  int exact;
  int *iflags, *iticket, *ierr;
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
template <class T, int TPR, int NVPT, bool CPLX, int PREC>
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
template <class T, int TPR, int NVPT, bool CPLX, int PREC>
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
      if constexpr (PREC == 1) {
        T ph[VEC];
        apply_dinv<T, CPLX, VEC>(ph, a.Dinv, row, p);
        vstore(a.Ph + off, ph);
      }
    }
  }
}

// s = r - alpha v;  sh = Dinv s
template <class T, int TPR, int NVPT, bool CPLX, int PREC>
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
      if constexpr (PREC == 1) {
        T sh[VEC];
        apply_dinv<T, CPLX, VEC>(sh, a.Dinv, row, r);
        vstore(a.Sh + off, sh);
      }
    }
  }
}

// x += alpha ph + omega sh;  r = s - omega t;  dots <rhat, r>, <r, r>
template <class T, int TPR, int NVPT, bool CPLX, int PREC>
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
      if constexpr (PREC != 0) vload(a.Sh + off, sh);
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

// ------------------------------------------------------------ ILU(0) ----
// Incomplete LU of M_p = A^T + p I on the pattern of A^T, computed by
// fixed-point sweeps (Chow & Patel, SIAM J. Sci. Comput. 37(2), 2015): every
// entry is updated in parallel from the previous iterate,
//   i > j: l_ij = (m_ij - sum_{k<j} l_ik u_kj) / u_jj,
//   i <= j: u_ij =  m_ij - sum_{k<i} l_ik u_kj,
// with L unit lower and U upper stored in one array F on the pattern.  The
// triangular solves of the preconditioner are approximated by Jacobi sweeps
// (Anzt, Chow & Dongarra 2015): y <- r - (L - I) y, x <- D^{-1}(y - (U - D) x).
// Complex shifts give complex factors (interleaved re, im).

__global__ void k_diagpos(int n, const int* __restrict__ rp, const int* __restrict__ ci, int* __restrict__ dpos) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    int lo = rp[i], hi = rp[i + 1] - 1, pos = -1;
    while (lo <= hi) {
      const int mid = (lo + hi) >> 1;
      const int c = ci[mid];
      if (c == i) { pos = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    dpos[i] = pos;
  }
}

template <class T, bool CPLX>
__device__ __forceinline__ cd fload(const T* F, int e) {
  if constexpr (CPLX) return cd{(double)F[2 * e], (double)F[2 * e + 1]};
  else return cd{(double)F[e], 0.0};
}
template <class T, bool CPLX>
__device__ __forceinline__ void fstore(T* F, int e, cd v) {
  if constexpr (CPLX) { F[2 * e] = (T)v.re; F[2 * e + 1] = (T)v.im; }
  else F[e] = (T)v.re;
}

// m_e = (A^T)_e + p [i == j]
template <class T, bool CPLX>
__device__ __forceinline__ cd mval(const T* av, int e, int i, int j, double pre, double pim) {
  cd m{(double)av[e], 0.0};
  if (i == j) { m.re += pre; m.im += pim; }
  return m;
}

// initial guess: l_ij = m_ij / m_jj, u_ij = m_ij
template <class T, bool CPLX>
__global__ void k_ilu_init(int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ av,
                           const int* __restrict__ dpos, double pre, double pim, T* __restrict__ F) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      const int j = ci[e];
      cd m = mval<T, CPLX>(av, e, (int)i, j, pre, pim);
      if (j < i) {
        const int dj = dpos[j];
        const cd mjj = mval<T, CPLX>(av, dj, j, j, pre, pim);
        m = cdivz(m, mjj);
      }
      fstore<T, CPLX>(F, e, m);
    }
  }
}

// one synchronous fixed-point sweep Fnew <- G(Fold)
template <class T, bool CPLX>
__global__ void k_ilu_sweep(int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ av,
                            const int* __restrict__ dpos, double pre, double pim, const T* __restrict__ Fo,
                            T* __restrict__ Fn) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int b = rp[i], e_end = rp[i + 1];
    for (int e = b; e < e_end; ++e) {
      const int j = ci[e];
      const int lim = j < i ? j : (int)i;  // k < min(i, j)
      cd s = mval<T, CPLX>(av, e, (int)i, j, pre, pim);
      for (int kk = b; kk < e_end; ++kk) {
        const int k = ci[kk];
        if (k >= lim) break;  // columns sorted
        // find (k, j) in row k
        int lo = rp[k], hi = rp[k + 1] - 1, pos = -1;
        while (lo <= hi) {
          const int mid = (lo + hi) >> 1;
          const int c = ci[mid];
          if (c == j) { pos = mid; break; }
          if (c < j) lo = mid + 1; else hi = mid - 1;
        }
        if (pos >= 0) {
          const cd t = cmul(fload<T, CPLX>(Fo, kk), fload<T, CPLX>(Fo, pos));
          s.re -= t.re;
          s.im -= t.im;
        }
      }
      if (j < i) s = cdivz(s, fload<T, CPLX>(Fo, dpos[j]));
      fstore<T, CPLX>(Fn, e, s);
    }
  }
}

// Dinv[i] = 1 / u_ii
template <class T, bool CPLX>
__global__ void k_ilu_dinv(int n, const int* __restrict__ dpos, const T* __restrict__ F, T* __restrict__ dinv) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const cd z = cdivz(cd{1.0, 0.0}, fload<T, CPLX>(F, dpos[i]));
    if constexpr (CPLX) { dinv[2 * i] = (T)z.re; dinv[2 * i + 1] = (T)z.im; }
    else dinv[i] = (T)z.re;
  }
}

// Jacobi sweep of a triangular factor on an n x w block:
//   LOWER:  out = r - (L - I) xin          (xin == nullptr: out = r)
//   UPPER:  out = D^{-1} (r - (U - D) xin)  (xin == nullptr: out = D^{-1} r)
// SCALE_OUT (LOWER only): also write out2 = D^{-1} out (the first U iterate).
template <class T>
struct TriArgs {
  long n;
  const int* rp;
  const int* ci;
  const int* dpos;
  const T* F;
  const T* dinv;
  const T* r;
  const T* xin;
  T* out;
  T* out2;
  int ld;
  int nvec;
};

template <class T, int TPR, int NVPT, bool CPLX, bool LOWER, bool SCALE_OUT>
__global__ void __launch_bounds__(kBlock) k_trisweep(TriArgs<T> a) {
  constexpr int VEC = 16 / sizeof(T);
  RowIter<TPR> it;
  for (long row = it.row; row < a.n; row += it.stride) {
    const int dp = __ldg(a.dpos + row);
    const int e0 = LOWER ? __ldg(a.rp + row) : dp + 1;
    const int e1 = LOWER ? dp : __ldg(a.rp + row + 1);
    T acc[NVPT][VEC];
#pragma unroll
    for (int k = 0; k < NVPT; ++k)
#pragma unroll
      for (int q = 0; q < VEC; ++q) acc[k][q] = T(0);
    if (a.xin) {
      // triangles of stencil rows hold <= 3 entries: predicated chunks of 4
      for (int e = e0; e < e1; e += 4) {
        int c[4];
        T fr[4], fi[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = e + u < e1;
          c[u] = in ? __ldg(a.ci + e + u) : (int)row;
          if constexpr (CPLX) {
            fr[u] = in ? a.F[2 * (e + u)] : T(0);
            fi[u] = in ? a.F[2 * (e + u) + 1] : T(0);
          } else {
            fr[u] = in ? a.F[e + u] : T(0);
            fi[u] = T(0);
          }
        }
#pragma unroll
        for (int k = 0; k < NVPT; ++k) {
          const int v = it.lane_v + k * TPR;
          if (v < a.nvec) {
            T x[4][VEC];
#pragma unroll
            for (int u = 0; u < 4; ++u) vload(a.xin + (size_t)c[u] * a.ld + v * VEC, x[u]);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if constexpr (CPLX) {
#pragma unroll
                for (int q = 0; q < VEC; q += 2) {
                  acc[k][q] += fr[u] * x[u][q] - fi[u] * x[u][q + 1];
                  acc[k][q + 1] += fr[u] * x[u][q + 1] + fi[u] * x[u][q];
                }
              } else {
#pragma unroll
                for (int q = 0; q < VEC; ++q) acc[k][q] = fma(fr[u], x[u][q], acc[k][q]);
              }
            }
          }
        }
      }
    }
    T dr = T(1), di = T(0);
    if constexpr (CPLX) { dr = a.dinv[2 * row]; di = a.dinv[2 * row + 1]; }
    else dr = a.dinv[row];
#pragma unroll
    for (int k = 0; k < NVPT; ++k) {
      const int v = it.lane_v + k * TPR;
      if (v >= a.nvec) continue;
      const size_t off = (size_t)row * a.ld + v * VEC;
      T r[VEC], o[VEC];
      vload(a.r + off, r);
#pragma unroll
      for (int q = 0; q < VEC; ++q) o[q] = r[q] - acc[k][q];
      if constexpr (!LOWER) {
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            const T yr = dr * o[q] - di * o[q + 1], yi = dr * o[q + 1] + di * o[q];
            o[q] = yr;
            o[q + 1] = yi;
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) o[q] *= dr;
        }
      }
      vstore(a.out + off, o);
      if constexpr (LOWER && SCALE_OUT) {
        T o2[VEC];
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            o2[q] = dr * o[q] - di * o[q + 1];
            o2[q + 1] = dr * o[q + 1] + di * o[q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) o2[q] = dr * o[q];
        }
        vstore(a.out2 + off, o2);
      }
    }
  }
}

// GMRES per-column state (doubles): H ((m+1) x m complex, column-major), Givens
// cosines cs (m) and sines sn (m, complex), the rotated right-hand side g (m+1,
// complex), then beta0 = ||r_0||, the converged flag, the inner step count, ||b||.
__host__ __device__ inline size_t gm_state_stride(int m) { return (size_t)2 * (m + 1) * m + m + 2 * m + 2 * (m + 1) + 4; }
inline int gm_dot_ctas() { return device_sms() * 2; }

// ------------------------------------------------------- exact ILU(0) -----
// ILU(0) of M_p = A^T + p I on the pattern of A^T computed exactly (the IKJ
// elimination restricted to the pattern, Saad, Iterative Methods, Alg. 10.4), and
// exact triangular solves with it, without level sets: one warp per row, rows
// claimed in elimination order from an atomic ticket, each row waiting (bounded)
// for the rows it depends on to publish their results (a ready flag per row,
// release/acquire; the data are read past L1).  A warp only ever waits for rows
// claimed before its own, by warps already running, so progress is guaranteed.
// A wait that exceeds its bound sets the error word and the kernel finishes
// without further waits; the host reports CARE_TIMEOUT.
constexpr long long ILU_WAIT_NS = 2000000000LL;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ long long ilu_clock() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// lane 0 waits until flags[k] != 0; warp-uniform result (false: gave up)
__device__ __forceinline__ bool ilu_wait(const int* flags, int k, int* err) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if (ld_acquire(flags + k) == 0) {
      const long long t0 = ilu_clock();
      while (ld_acquire(flags + k) == 0) {
        if (*(volatile int*)err != 0 || ilu_clock() - t0 > ILU_WAIT_NS) {
          atomicCAS(err, 0, 5);
          ok = 0;
          break;
        }
      }
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();  // the other lanes' reads of the awaited row come after lane 0's acquire
  return ok != 0;
}

template <class T, bool CPLX>
__device__ __forceinline__ cd fld_cg(const T* F, int e) {
  if constexpr (CPLX) return cd{(double)__ldcg(F + 2 * e), (double)__ldcg(F + 2 * e + 1)};
  else return cd{(double)__ldcg(F + e), 0.0};
}

// F (values on the pattern; complex interleaved) = M_p, then eliminated in place:
// strictly lower part L (unit diagonal implied), the rest U.  flags, ticket zeroed.
template <class T, bool CPLX>
__global__ void k_ilu_exact(int n, const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ dpos,
                            T* F, int* flags, int* ticket, int* err) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    int row = 0;
    if (lane == 0) row = atomicAdd(ticket, 1);
    row = __shfl_sync(0xffffffffu, row, 0);
    if (row >= n) break;
    const int b = rp[row], e_end = rp[row + 1], dp = dpos[row];
    // entry e of the row belongs to lane (e - b) % 32 for the whole row: it is read
    // and written by that lane only, so no value of this row passes between lanes
    // through memory (the multiplier is broadcast by shuffle)
    bool alive = __shfl_sync(0xffffffffu, *(volatile int*)err == 0 ? 1 : 0, 0) != 0;
    for (int e = b; e < dp && alive; ++e) {
      const int k = ci[e];
      if (!ilu_wait(flags, k, err)) {
        alive = false;
        break;
      }
      // l_ik = a_ik / u_kk, then a_ij -= l_ik u_kj for the pattern entries j > k of row i
      const int owner = (e - b) & 31;
      cd lik{0.0, 0.0};
      if (lane == owner) {
        lik = cdivz(fld_cg<T, CPLX>(F, e), fld_cg<T, CPLX>(F, dpos[k]));
        fstore<T, CPLX>(F, e, lik);
      }
      lik.re = __shfl_sync(0xffffffffu, lik.re, owner);
      lik.im = __shfl_sync(0xffffffffu, lik.im, owner);
      const int kb = dpos[k] + 1, ke = rp[k + 1];
      for (int e2 = b + lane; e2 < e_end; e2 += 32) {
        if (e2 <= e) continue;
        const int j = ci[e2];
        int lo = kb, hi = ke - 1, pos = -1;
        while (lo <= hi) {
          const int mid = (lo + hi) >> 1;
          const int c = ci[mid];
          if (c == j) { pos = mid; break; }
          if (c < j) lo = mid + 1; else hi = mid - 1;
        }
        if (pos >= 0) {
          const cd t = cmul(lik, fld_cg<T, CPLX>(F, pos));
          cd a = fld_cg<T, CPLX>(F, e2);
          a.re -= t.re;
          a.im -= t.im;
          fstore<T, CPLX>(F, e2, a);
        }
      }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + row, 1);
  }
}

// Exact triangular solve on an n x (nvec vectors) block, one warp per row:
// LOWER: y_i = r_i - sum_{k<i} l_ik y_k (rows in increasing order);
// UPPER: x_i = (r_i - sum_{k>i} u_ik x_k) / u_ii (rows in decreasing order).
template <class T, bool CPLX, bool LOWER>
__global__ void k_tri_exact(long n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const int* __restrict__ dpos, const T* __restrict__ F, const T* __restrict__ r, T* out,
                            int ld, int nvec, int* flags, int* ticket, int* err) {
  constexpr int VEC = 16 / sizeof(T);
  const int lane = threadIdx.x & 31;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= n) break;
    const long row = LOWER ? t : n - 1 - t;
    const int dp = dpos[row];
    const int e0 = LOWER ? rp[row] : dp + 1, e1 = LOWER ? dp : rp[row + 1];
    T acc[2][VEC];
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int v = lane + 32 * k2;
      if (v < nvec) vload(r + (size_t)row * ld + v * VEC, acc[k2]);
    }
    bool alive = __shfl_sync(0xffffffffu, *(volatile int*)err == 0 ? 1 : 0, 0) != 0;
    for (int e = e0; e < e1 && alive; ++e) {
      const int k = ci[e];
      if (!ilu_wait(flags, k, err)) {
        alive = false;
        break;
      }
      const cd f = fld_cg<T, CPLX>(F, e);
#pragma unroll
      for (int k2 = 0; k2 < 2; ++k2) {
        const int v = lane + 32 * k2;
        if (v >= nvec) continue;
        const T* xr = out + (size_t)k * ld + v * VEC;
        T x[VEC];
#pragma unroll
        for (int q = 0; q < VEC; ++q) x[q] = __ldcg(xr + q);
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            acc[k2][q] -= (T)f.re * x[q] - (T)f.im * x[q + 1];
            acc[k2][q + 1] -= (T)f.re * x[q + 1] + (T)f.im * x[q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[k2][q] -= (T)f.re * x[q];
        }
      }
    }
    if (!LOWER) {
      const cd dinv = cdivz(cd{1.0, 0.0}, fld_cg<T, CPLX>(F, dp));
#pragma unroll
      for (int k2 = 0; k2 < 2; ++k2) {
        if constexpr (CPLX) {
#pragma unroll
          for (int q = 0; q < VEC; q += 2) {
            const T yr = (T)dinv.re * acc[k2][q] - (T)dinv.im * acc[k2][q + 1];
            const T yi = (T)dinv.re * acc[k2][q + 1] + (T)dinv.im * acc[k2][q];
            acc[k2][q] = yr;
            acc[k2][q + 1] = yi;
          }
        } else {
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[k2][q] *= (T)dinv.re;
        }
      }
    }
#pragma unroll
    for (int k2 = 0; k2 < 2; ++k2) {
      const int v = lane + 32 * k2;
      if (v < nvec) vstore(out + (size_t)row * ld + v * VEC, acc[k2]);
    }
    __threadfence();
    __syncwarp();
    if (lane == 0) st_release(flags + row, 1);
  }
}

template <class T>
KrylovWork<T> krylov_alloc(Arena& ar, int n, bool jacobi, long nnz_ilu, int gmres_restart) {
  KrylovWork<T> w;
  const size_t blk = (size_t)n * kMaxRealCols;
  w.n = n;
  w.X = ar.get<T>(blk); w.R = ar.get<T>(blk); w.Rh = ar.get<T>(blk); w.P = ar.get<T>(blk);
  w.V = ar.get<T>(blk); w.S = ar.get<T>(blk); w.Tt = ar.get<T>(blk);
  if (jacobi) {
    w.Ph = ar.get<T>(blk); w.Sh = ar.get<T>(blk); w.Dinv = ar.get<T>((size_t)2 * n);
  }
  if (nnz_ilu >= 0) {
    w.ilu = true;
    w.F0 = ar.get<T>((size_t)2 * nnz_ilu);
    w.F1 = ar.get<T>((size_t)2 * nnz_ilu);
    w.dpos = ar.get<int>((size_t)n);
    w.Y1 = ar.get<T>(blk); w.Y2 = ar.get<T>(blk); w.Y3 = ar.get<T>(blk);
    w.iflags = ar.get<int>((size_t)n + 64);
    w.iticket = ar.get<int>(64);
    w.ierr = ar.get<int>(64);
  }
  w.st = ar.get<KState>(kMaxRealCols);
  w.hdr = ar.get<KHeader>(1);
  w.partial = ar.get<double>((size_t)device_sms() * 8 * 2 * kMaxRealCols);
  w.out = ar.get<double>(2 * kMaxRealCols);
  if (gmres_restart > 0) {
    const int m = gmres_restart;
    w.gm_restart = m;
    w.GV = ar.get<T>(blk * (size_t)(m + 1));
    w.GZ = ar.get<T>(blk);
    w.GS = ar.get<double>((size_t)kMaxRealCols * gm_state_stride(m));
    w.GH = ar.get<double>((size_t)2 * (m + 1) * kMaxRealCols);
    w.GP = ar.get<double>((size_t)gm_dot_ctas() * 2 * (m + 1) * kMaxRealCols);
  }
  return w;
}
template KrylovWork<float> krylov_alloc<float>(Arena&, int, bool, long, int);
template KrylovWork<double> krylov_alloc<double>(Arena&, int, bool, long, int);

// out = P^{-1} r with P = L U the ILU(0) factor: tri_sweeps Jacobi sweeps on L
// then on U (see the ILU(0) notes above).
template <class T, int TPR, int NVPT, bool CPLX>
static void ilu_apply(const KArgs<T>& a, const T* r, T* out, int grid, cudaStream_t s) {
  if (a.exact) {
    // exact forward (unit L) then backward (U) substitution, sync-free by rows
    const int g = device_sms() * 4;
    CARE_CUDA(cudaMemsetAsync(a.iflags, 0, sizeof(int) * (size_t)a.n, s));
    CARE_CUDA(cudaMemsetAsync(a.iticket, 0, sizeof(int), s));
    k_tri_exact<T, CPLX, true><<<g, kBlock, 0, s>>>(a.n, a.rp, a.ci, a.dpos, a.F, r, a.Y1, a.ld, a.nvec, a.iflags,
                                                    a.iticket, a.ierr);
    CARE_LAUNCH();
    CARE_CUDA(cudaMemsetAsync(a.iflags, 0, sizeof(int) * (size_t)a.n, s));
    CARE_CUDA(cudaMemsetAsync(a.iticket, 0, sizeof(int), s));
    k_tri_exact<T, CPLX, false><<<g, kBlock, 0, s>>>(a.n, a.rp, a.ci, a.dpos, a.F, a.Y1, out, a.ld, a.nvec, a.iflags,
                                                     a.iticket, a.ierr);
    CARE_LAUNCH();
    return;
  }
  TriArgs<T> t{};
  t.n = a.n; t.rp = a.rp; t.ci = a.ci; t.dpos = a.dpos; t.F = a.F; t.dinv = a.Dinv; t.ld = a.ld; t.nvec = a.nvec;
  const int sT = a.tri_sweeps;
  T* yb[2] = {a.Y1, a.Y2};
  int yi = 0;
  const T* yprev = r;
  for (int q = 1; q <= sT; ++q) {
    t.r = r; t.xin = yprev; t.out = yb[yi];
    if (q == sT) {
      t.out2 = a.Y3;
      k_trisweep<T, TPR, NVPT, CPLX, true, true><<<grid, kBlock, 0, s>>>(t);
    } else {
      k_trisweep<T, TPR, NVPT, CPLX, true, false><<<grid, kBlock, 0, s>>>(t);
    }
    CARE_LAUNCH();
    yprev = yb[yi];
    yi ^= 1;
  }
  // y = yprev (yb[yi ^ 1]); first U iterate x0 = D^{-1} y is in Y3
  const T* xprev = a.Y3;
  for (int q = 1; q <= sT; ++q) {
    T* dst = (q == sT) ? out : (xprev == a.Y3 ? yb[yi] : a.Y3);
    t.r = yprev; t.xin = xprev; t.out = dst; t.out2 = nullptr;
    k_trisweep<T, TPR, NVPT, CPLX, false, false><<<grid, kBlock, 0, s>>>(t);
    CARE_LAUNCH();
    xprev = dst;
  }
}

// One BiCGStab iteration: p-update, [ILU apply], SpMM + <rhat, v>, s-update,
// [ILU apply], SpMM + <s, t>, <t, t>, x/r-update + <rhat, r>, <r, r>.
template <class T, int TPR, int NVPT, bool CPLX, int PREC>
static void bicg_iteration(const KArgs<T>& a, SpmmArgs<T>& sp, int grid, cudaStream_t s) {
  k_bicg_p<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  if constexpr (PREC == 2) ilu_apply<T, TPR, NVPT, CPLX>(a, a.P, a.Ph, grid, s);
  sp.X = PREC ? a.Ph : a.P; sp.Y = a.V; sp.w0 = a.Rh; sp.w1 = nullptr; sp.mode = FIN_ALPHA;
  launch_spmm<T, 1, CPLX>(sp, s);
  k_bicg_s<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  if constexpr (PREC == 2) ilu_apply<T, TPR, NVPT, CPLX>(a, a.S, a.Sh, grid, s);
  sp.X = PREC ? a.Sh : a.S; sp.Y = a.Tt; sp.w0 = a.S; sp.w1 = nullptr; sp.mode = FIN_OMEGA;
  launch_spmm<T, 2, CPLX>(sp, s);
  k_bicg_xr<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
}

// Per-thread, per-device capture stream and fork/join events (created once,
// destroyed when the thread exits: the batched solver's worker threads are
// short-lived, and every launch on these streams has been synchronised by then).
struct CaptureRes {
  cudaStream_t cs = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  CaptureRes() = default;
  CaptureRes(const CaptureRes&) = delete;
  CaptureRes& operator=(const CaptureRes&) = delete;
  ~CaptureRes() {
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    if (cs) cudaStreamDestroy(cs);
  }
};
// Per-thread, per-device executable graphs of one BiCGStab instantiation,
// destroyed with the thread for the same reason.
struct GraphExecCache {
  cudaGraphExec_t e[64] = {nullptr};
  GraphExecCache() = default;
  GraphExecCache(const GraphExecCache&) = delete;
  GraphExecCache& operator=(const GraphExecCache&) = delete;
  ~GraphExecCache() {
    for (cudaGraphExec_t x : e)
      if (x) cudaGraphExecDestroy(x);
  }
};
static CaptureRes& capture_res() {
  thread_local CaptureRes r[64];
  int dev = 0;
  CARE_CUDA(cudaGetDevice(&dev));
  CaptureRes& c = r[dev & 63];
  if (!c.cs) {
    CARE_CUDA(cudaStreamCreateWithFlags(&c.cs, cudaStreamNonBlocking));
    CARE_CUDA(cudaEventCreateWithFlags(&c.ev[0], cudaEventDisableTiming));
    CARE_CUDA(cudaEventCreateWithFlags(&c.ev[1], cudaEventDisableTiming));
  }
  return c;
}

template <class T, int TPR, int NVPT, bool CPLX, int PREC>
static KrylovResult run_bicg(const OpT<T>& op, cd sigma, KArgs<T> a, int maxit, int grid,
                             cudaStream_t s) {
  KrylovResult res;
  SpmmArgs<T> sp{};
  sp.n = op.n; sp.rp = op.rp; sp.ci = op.ci; sp.av = op.val; sp.rs = op.rowsum; sp.ldx = a.ld; sp.ldy = a.ld;
  sp.nvec = a.nvec; sp.sre = sigma.re; sp.sim = sigma.im; sp.dots = a.dots; sp.st = a.st;
  sp.hdr = a.hdr; sp.tol2 = a.tol2;
  k_bicg_init<T, TPR, NVPT, CPLX, PREC><<<grid, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  constexpr int poll = 4;
  KHeader h{};
  int it = 0;
  CARE_CUDA(cudaMemcpyAsync(&h, a.hdr, sizeof(KHeader), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  if (h.n_active == 0) return res;
  // Capture `poll` iterations once and replay the graph; the executable graph is
  // kept per thread and updated in place when only kernel parameters change.
  const long per_iter = 5 + (PREC == 2 ? (a.exact ? 4L : 4L * a.tri_sweeps) : 0);
  thread_local GraphExecCache exec_cache;
  int dev = 0;
  CARE_CUDA(cudaGetDevice(&dev));
  cudaGraphExec_t& exec = exec_cache.e[dev & 63];
  CaptureRes& cr = capture_res();
  bool graphs = maxit >= poll;
  if (graphs) {
    cudaGraph_t g = nullptr;
    CARE_CUDA(cudaStreamBeginCapture(cr.cs, cudaStreamCaptureModeThreadLocal));
    for (int q = 0; q < poll; ++q) bicg_iteration<T, TPR, NVPT, CPLX, PREC>(a, sp, grid, cr.cs);
    CARE_CUDA(cudaStreamEndCapture(cr.cs, &g));
    count_launch_n(-per_iter * poll);  // captured, not executed
    bool ok = false;
    if (exec) {
      cudaGraphExecUpdateResultInfo info{};
      ok = cudaGraphExecUpdate(exec, g, &info) == cudaSuccess;
      if (!ok) {
        cudaGetLastError();
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
    }
    if (!ok) CARE_CUDA(cudaGraphInstantiate(&exec, g, 0));
    cudaGraphDestroy(g);
    // fork onto the capture stream after the caller's stream
    CARE_CUDA(cudaEventRecord(cr.ev[0], s));
    CARE_CUDA(cudaStreamWaitEvent(cr.cs, cr.ev[0], 0));
  }
  while (it < maxit) {
    if (graphs && it + poll <= maxit) {
      CARE_CUDA(cudaGraphLaunch(exec, cr.cs));
      count_launch_n(per_iter * poll);
      it += poll;
      res.spmm += 2 * poll;
      CARE_CUDA(cudaMemcpyAsync(&h, a.hdr, sizeof(KHeader), cudaMemcpyDeviceToHost, cr.cs));
      CARE_CUDA(cudaStreamSynchronize(cr.cs));
    } else {
      cudaStream_t ss = graphs ? cr.cs : s;
      bicg_iteration<T, TPR, NVPT, CPLX, PREC>(a, sp, grid, ss);
      ++it;
      res.spmm += 2;
      if (it % poll == 0 || it == maxit) {
        CARE_CUDA(cudaMemcpyAsync(&h, a.hdr, sizeof(KHeader), cudaMemcpyDeviceToHost, ss));
        CARE_CUDA(cudaStreamSynchronize(ss));
      } else {
        continue;
      }
    }
    if (h.n_active == 0) break;
  }
  if (graphs) {
    // join back: the caller's stream waits for the capture stream
    CARE_CUDA(cudaEventRecord(cr.ev[1], cr.cs));
    CARE_CUDA(cudaStreamWaitEvent(s, cr.ev[1], 0));
  }
  res.iters = it;
  return res;
}

// F = M_p = A^T + sigma I on the pattern (complex interleaved when CPLX)
template <class T, bool CPLX>
__global__ void k_ilu_copy(int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ av,
                           double pre, double pim, T* __restrict__ F) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    for (int e = rp[i]; e < rp[i + 1]; ++e) fstore<T, CPLX>(F, e, mval<T, CPLX>(av, e, (int)i, ci[e], pre, pim));
}

// exact ILU(0) of M_p into w.F0 (w.ierr is cleared first and read by the caller)
template <class T>
static const T* ilu_exact_setup(const OpT<T>& op, cd sigma, bool cplx, KrylovWork<T>& w, cudaStream_t s) {
  const int g = device_sms() * 4;
  k_diagpos<<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, w.dpos);
  CARE_LAUNCH();
  if (cplx) k_ilu_copy<T, true><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, sigma.re, sigma.im, w.F0);
  else k_ilu_copy<T, false><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, sigma.re, sigma.im, w.F0);
  CARE_LAUNCH();
  CARE_CUDA(cudaMemsetAsync(w.iflags, 0, sizeof(int) * (size_t)op.n, s));
  CARE_CUDA(cudaMemsetAsync(w.iticket, 0, sizeof(int), s));
  CARE_CUDA(cudaMemsetAsync(w.ierr, 0, sizeof(int), s));
  if (cplx) k_ilu_exact<T, true><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, w.dpos, w.F0, w.iflags, w.iticket, w.ierr);
  else k_ilu_exact<T, false><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, w.dpos, w.F0, w.iflags, w.iticket, w.ierr);
  CARE_LAUNCH();
  return w.F0;
}

// ILU(0) of M_p = A^T + sigma I into w.F0 / w.F1; returns the final factor.
template <class T>
static const T* ilu_setup(const OpT<T>& op, cd sigma, bool cplx, KrylovWork<T>& w, cudaStream_t s) {
  const int g = device_sms() * 4;
  k_diagpos<<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, w.dpos);
  CARE_LAUNCH();
  T* Fa = w.F0;
  T* Fb = w.F1;
  if (cplx) k_ilu_init<T, true><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, w.dpos, sigma.re, sigma.im, Fa);
  else k_ilu_init<T, false><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, w.dpos, sigma.re, sigma.im, Fa);
  CARE_LAUNCH();
  for (int q = 0; q < w.ilu_sweeps; ++q) {
    if (cplx) k_ilu_sweep<T, true><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, w.dpos, sigma.re, sigma.im, Fa, Fb);
    else k_ilu_sweep<T, false><<<g, kBlock, 0, s>>>(op.n, op.rp, op.ci, op.val, w.dpos, sigma.re, sigma.im, Fa, Fb);
    CARE_LAUNCH();
    std::swap(Fa, Fb);
  }
  if (cplx) k_ilu_dinv<T, true><<<g, kBlock, 0, s>>>(op.n, w.dpos, Fa, w.Dinv);
  else k_ilu_dinv<T, false><<<g, kBlock, 0, s>>>(op.n, w.dpos, Fa, w.Dinv);
  CARE_LAUNCH();
  return Fa;
}

template <class T>
KrylovResult krylov_bicgstab(const OpT<T>& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol,
                             int ld_sol, int cols, double tol, int maxit, int precond,
                             KrylovWork<T>& w, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T);
  CARE_REQUIRE(cols <= kMaxRealCols && cols > 0, CARE_ERR_INVALID_ARG, "krylov: bad width");
  CARE_REQUIRE(!cplx || cols % 2 == 0, CARE_ERR_INVALID_ARG, "krylov: odd complex width");
  int pmode = 0;
  const bool ilu_req = precond == CARE_PRECOND_ILU0 || precond == CARE_PRECOND_ILU0_EXACT;
  if (ilu_req && w.ilu && op.full_diag) pmode = 2;
  else if ((precond == CARE_PRECOND_JACOBI || ilu_req) && !op.diag_const && w.Ph != nullptr)
    pmode = 1;  // ILU(0) needs every diagonal entry and sparse rows; Jacobi otherwise
  const bool exact = pmode == 2 && precond == CARE_PRECOND_ILU0_EXACT;
  KArgs<T> a{};
  a.exact = exact ? 1 : 0;
  a.iflags = w.iflags; a.iticket = w.iticket; a.ierr = w.ierr;
  a.n = op.n;
  a.ld = pad_ld<T>(cols);
  a.nvec = a.ld / VEC;
  a.X = w.X; a.R = w.R; a.Rh = w.Rh; a.P = w.P; a.V = w.V; a.S = w.S; a.Tt = w.Tt;
  a.Ph = w.Ph; a.Sh = w.Sh; a.Dinv = w.Dinv;
  a.rhs = rhs; a.ld_rhs = ld_rhs; a.sol = sol; a.ld_sol = ld_sol; a.cols = cols;
  a.st = w.st; a.hdr = w.hdr;
  a.dots = DotOut{w.partial, w.out, &w.hdr->counter};
  a.tol2 = tol * tol;
  a.rp = op.rp; a.ci = op.ci; a.dpos = w.dpos; a.Y1 = w.Y1; a.Y2 = w.Y2; a.Y3 = w.Y3;
  a.tri_sweeps = w.tri_sweeps < 1 ? 1 : w.tri_sweeps;
  const int tpr = tpr_for(a.nvec);
  const int nvpt = (a.nvec + 31) / 32;
  const int grid = grid_rows(op.n, tpr);
  CARE_REQUIRE(grid <= device_sms() * 8, CARE_ERR_INVALID_ARG, "krylov: grid exceeds partial buffer");
  // reduction counter and flags start from zero for every solve
  CARE_CUDA(cudaMemsetAsync(w.hdr, 0, sizeof(KHeader), s));
  if (pmode == 1) {
    k_dinv<T><<<device_sms() * 4, kBlock, 0, s>>>(op.n, op.diag, sigma.re, sigma.im, cplx, w.Dinv);
    CARE_LAUNCH();
  } else if (pmode == 2) {
    a.F = exact ? ilu_exact_setup<T>(op, sigma, cplx, w, s) : ilu_setup<T>(op, sigma, cplx, w, s);
  }
  KrylovResult r;
#define CARE_BICG_CASE(TP, NV)                                                                        \
  if (tpr == TP && nvpt == NV) {                                                                      \
    if (cplx) r = pmode == 2 ? run_bicg<T, TP, NV, true, 2>(op, sigma, a, maxit, grid, s)             \
                 : pmode == 1 ? run_bicg<T, TP, NV, true, 1>(op, sigma, a, maxit, grid, s)            \
                              : run_bicg<T, TP, NV, true, 0>(op, sigma, a, maxit, grid, s);           \
    else r = pmode == 2 ? run_bicg<T, TP, NV, false, 2>(op, sigma, a, maxit, grid, s)                 \
            : pmode == 1 ? run_bicg<T, TP, NV, false, 1>(op, sigma, a, maxit, grid, s)                \
                         : run_bicg<T, TP, NV, false, 0>(op, sigma, a, maxit, grid, s);               \
    goto done;                                                                                        \
  }
  CARE_BICG_CASE(1, 1) CARE_BICG_CASE(2, 1) CARE_BICG_CASE(4, 1) CARE_BICG_CASE(8, 1)
  CARE_BICG_CASE(16, 1) CARE_BICG_CASE(32, 1) CARE_BICG_CASE(32, 2)
#undef CARE_BICG_CASE
  CARE_THROW(CARE_ERR_INVALID_ARG, "krylov: unsupported width");
done:
  k_copy_out<T><<<device_sms() * 4, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  {
    // Algorithmic bytes (what the iteration must move, each block once per pass):
    // a block pass is n * ld reals; the operator pass reads A^T's values and
    // indices, row pointers and row sums; a triangular ILU(0) sweep reads about
    // half of the factor with its indices.  Per iteration: p-update 4 passes
    // (+1 Jacobi), two SpMMs of 3 passes + the operator, s-update 3 (+1), x/r
    // update 8 (+2 Jacobi / ILU), and for ILU(0) two applications of 2T triangular
    // sweeps of 3 passes (+1) each; init 6 passes; ILU(0) setup 1 + sweeps passes
    // over the factor.
    const double sv = sizeof(T), sf = sv * (cplx ? 2 : 1);
    const double blk = (double)op.n * a.ld * sv;
    const double amat = (double)op.nnz * (sv + 4) + 4.0 * (op.n + 1) + (op.rowsum ? sv * op.n : 0.0);
    const double trisw = 0.5 * op.nnz * (sf + 4) + 8.0 * op.n;
    const int T_ = a.exact ? 1 : a.tri_sweeps;  // exact triangular solves: one pass each
    double per = 2 * amat;
    if (pmode == 0) per += 21 * blk;
    else if (pmode == 1) per += 25 * blk + 2 * sf * op.n;
    else per += (24 + 12.0 * T_) * blk + 4.0 * T_ * trisw;
    double setup = 6 * blk;
    if (pmode == 2) setup += (1 + (a.exact ? 1 : w.ilu_sweeps)) * ((double)op.nnz * (2 * sf + 4) + 8.0 * op.n);
    r.bytes = setup + per * r.iters;
  }
  {
    // count unconverged columns (flag != 1 among the valid state entries)
    const int nst = cplx ? cols / 2 : cols;
    std::vector<KState> hs(nst);
    CARE_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(KState) * nst, cudaMemcpyDeviceToHost, s));
    int ierr = 0;
    if (exact) CARE_CUDA(cudaMemcpyAsync(&ierr, w.ierr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CARE_CUDA(cudaStreamSynchronize(s));
    CARE_REQUIRE(ierr == 0, CARE_TIMEOUT, "exact ILU(0): a bounded wait expired");
    for (int j = 0; j < nst; ++j)
      if (hs[j].flag != 1) ++r.unconverged;
  }
  return r;
}
// ------------------------------------------------------------------ GMRES ---

struct GmView {
  double *H, *cs, *sn, *g, *misc;
  __host__ __device__ GmView(double* base, int m) {
    H = base;
    cs = H + 2 * (m + 1) * m;
    sn = cs + m;
    g = sn + 2 * m;
    misc = g + 2 * (m + 1);  // beta0, flag, steps
  }
};

// part[cta][q][c] (complex: 2 doubles) = sum over the CTA's row slab of conj(V_q) W,
// c over the (complex) columns; V_q = V + q * blk
template <class T, bool CPLX>
__global__ void k_gm_dots(long n, int ld, int ncol, const T* __restrict__ V, long blk, int nq,
                          const T* __restrict__ W, double* __restrict__ part) {
  const long per = (n + gridDim.x - 1) / gridDim.x;
  const long r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  const int items = nq * ncol;
  for (int t = threadIdx.x; t < items; t += blockDim.x) {
    const int q = t / ncol, c = t % ncol;
    const T* vq = V + (size_t)q * blk;
    double re = 0.0, im = 0.0;
    for (long r = r0; r < r1; ++r) {
      if constexpr (CPLX) {
        const double vr = vq[(size_t)r * ld + 2 * c], vi = vq[(size_t)r * ld + 2 * c + 1];
        const double wr = W[(size_t)r * ld + 2 * c], wi = W[(size_t)r * ld + 2 * c + 1];
        re += vr * wr + vi * wi;
        im += vr * wi - vi * wr;
      } else {
        re += (double)vq[(size_t)r * ld + c] * (double)W[(size_t)r * ld + c];
      }
    }
    double* o = part + ((size_t)blockIdx.x * nq * ncol + t) * 2;
    o[0] = re;
    o[1] = im;
  }
}
// out[q][c] (2 doubles) = fixed-order sum over the CTAs
__global__ void k_gm_dots_reduce(int ctas, int items, const double* __restrict__ part, double* __restrict__ out) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < items; t += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < ctas; ++b) {
      re += part[((size_t)b * items + t) * 2];
      im += part[((size_t)b * items + t) * 2 + 1];
    }
    out[2 * t] = re;
    out[2 * t + 1] = im;
  }
}

// W[r][c] = beta_w W[r][c] + sum_q coef[q][c] V_q[r][c]  (complex coefficients in
// complex mode; coef as produced by k_gm_dots_reduce, scaled by cscale)
template <class T, bool CPLX>
__global__ void k_gm_combine(long n, int ld, int ncol, T* __restrict__ W, double beta_w, const T* __restrict__ V,
                             long blk, int nq, const double* __restrict__ coef, double cscale) {
  const long total = n * (long)ncol;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / ncol;
    const int c = (int)(e % ncol);
    if constexpr (CPLX) {
      double ar = beta_w * (double)W[(size_t)r * ld + 2 * c], ai = beta_w * (double)W[(size_t)r * ld + 2 * c + 1];
      for (int q = 0; q < nq; ++q) {
        const double hr = cscale * coef[2 * (q * ncol + c)], hi = cscale * coef[2 * (q * ncol + c) + 1];
        const double vr = V[(size_t)q * blk + (size_t)r * ld + 2 * c], vi = V[(size_t)q * blk + (size_t)r * ld + 2 * c + 1];
        ar += hr * vr - hi * vi;
        ai += hr * vi + hi * vr;
      }
      W[(size_t)r * ld + 2 * c] = (T)ar;
      W[(size_t)r * ld + 2 * c + 1] = (T)ai;
    } else {
      double a = beta_w * (double)W[(size_t)r * ld + c];
      for (int q = 0; q < nq; ++q) a += cscale * coef[2 * (q * ncol + c)] * (double)V[(size_t)q * blk + (size_t)r * ld + c];
      W[(size_t)r * ld + c] = (T)a;
    }
  }
}

// dst[r][c] = src[r][c] * s[c] (complex columns share s[c]); the padding columns of
// dst (beyond the valid ones, up to ld) are set to zero
template <class T, bool CPLX>
__global__ void k_gm_scale(long n, int ld, int ncol, const T* __restrict__ src, const double* __restrict__ sc,
                           T* __restrict__ dst) {
  const long total = n * (long)ld;
  const int valid = CPLX ? 2 * ncol : ncol;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / ld;
    const int c = (int)(e % ld);
    const int cc = CPLX ? c / 2 : c;
    dst[(size_t)r * ld + c] = c < valid ? (T)(sc[cc] * (double)src[(size_t)r * ld + c]) : T(0);
  }
}

// dst = right-hand side in the padded block layout (zeros beyond the valid columns)
template <class T>
__global__ void k_gm_copy_in(KArgs<T> a, T* __restrict__ dst) {
  const long total = a.n * (long)a.ld;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / a.ld;
    const int c = (int)(e % a.ld);
    dst[e] = c < a.cols ? a.rhs[(size_t)r * a.ld_rhs + c] : T(0);
  }
}

// Start of a cycle: from nr = ||r||^2 (dots output, re part) set beta0, g = (beta, 0..),
// scale[c] = 1 / beta (0 for converged / zero columns), steps = 0.  At the first
// cycle bnorm[c] = ||b_c|| is recorded; a column whose ||r|| <= tol ||b|| is done.
__global__ void k_gm_start(int ncol, int m, const double* __restrict__ nr, double* __restrict__ GS,
                           double* __restrict__ bnorm, int first, double tol, double* __restrict__ scale,
                           int* __restrict__ active) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    GmView v(GS + (size_t)c * gm_state_stride(m), m);
    const double beta = sqrt(fmax(nr[2 * c], 0.0));
    if (first) bnorm[c] = beta;
    const bool done = !(beta > tol * bnorm[c]) || !isfinite(beta);
    for (int i = 0; i < 2 * (m + 1); ++i) v.g[i] = 0.0;
    v.g[0] = beta;
    v.misc[0] = beta;
    v.misc[1] = done ? 1.0 : 0.0;
    v.misc[2] = 0.0;
    scale[c] = done ? 0.0 : 1.0 / beta;
    if (!done) atomicAdd(active, 1);
  }
}

// Arnoldi step k for every column: h (k+1 complex coefficients, CGS2 sum) and
// hn = ||w||^2 give H(:, k); earlier rotations applied, a new one computed; g
// rotated; scale[c] = 1 / ||w|| for the next basis vector.  Converged columns keep
// their state (their basis vectors are scaled by 0).
__global__ void k_gm_arnoldi(int ncol, int m, int k, const double* __restrict__ h1, const double* __restrict__ h2,
                             const double* __restrict__ nw, double* __restrict__ GS, double tol,
                             double* __restrict__ scale, int* __restrict__ active) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    GmView v(GS + (size_t)c * gm_state_stride(m), m);
    if (v.misc[1] != 0.0) {
      scale[c] = 0.0;
      continue;
    }
    double* Hk = v.H + (size_t)2 * (m + 1) * k;  // column k: m+1 complex entries
    for (int i = 0; i <= k; ++i) {
      Hk[2 * i] = h1[2 * (i * ncol + c)] + h2[2 * (i * ncol + c)];
      Hk[2 * i + 1] = h1[2 * (i * ncol + c) + 1] + h2[2 * (i * ncol + c) + 1];
    }
    const double hn = sqrt(fmax(nw[2 * c], 0.0));
    Hk[2 * (k + 1)] = hn;
    Hk[2 * (k + 1) + 1] = 0.0;
    // earlier rotations: [a; b] <- [c a + s b; -conj(s) a + c b]
    for (int i = 0; i < k; ++i) {
      const cd a{Hk[2 * i], Hk[2 * i + 1]}, b{Hk[2 * i + 2], Hk[2 * i + 3]};
      const double cc = v.cs[i];
      const cd s{v.sn[2 * i], v.sn[2 * i + 1]};
      const cd sb = cmul(s, b), sa = cmul(cconj(s), a);
      Hk[2 * i] = cc * a.re + sb.re;
      Hk[2 * i + 1] = cc * a.im + sb.im;
      Hk[2 * i + 2] = cc * b.re - sa.re;
      Hk[2 * i + 3] = cc * b.im - sa.im;
    }
    // new rotation zeroing H(k+1, k): c = |a| / r, s = (a / |a|) conj(b) / r
    const cd a{Hk[2 * k], Hk[2 * k + 1]}, b{Hk[2 * k + 2], Hk[2 * k + 3]};
    const double aa = hypot(a.re, a.im), bb = hypot(b.re, b.im), rr = hypot(aa, bb);
    double cc = 1.0;
    cd s{0.0, 0.0};
    if (rr > 0.0) {
      if (aa == 0.0) {
        cc = 0.0;
        s = cconj(cd{b.re / bb, b.im / bb});
      } else {
        cc = aa / rr;
        const cd ph{a.re / aa, a.im / aa};
        s = cmul(ph, cd{b.re / rr, -b.im / rr});
      }
    }
    v.cs[k] = cc;
    v.sn[2 * k] = s.re;
    v.sn[2 * k + 1] = s.im;
    const cd sb = cmul(s, b);
    Hk[2 * k] = cc * a.re + sb.re;
    Hk[2 * k + 1] = cc * a.im + sb.im;
    Hk[2 * k + 2] = 0.0;
    Hk[2 * k + 3] = 0.0;
    // g(k..k+1) rotated
    const cd gk{v.g[2 * k], v.g[2 * k + 1]};
    const cd sg = cmul(cconj(s), gk);
    v.g[2 * k] = cc * gk.re;
    v.g[2 * k + 1] = cc * gk.im;
    v.g[2 * k + 2] = -sg.re;
    v.g[2 * k + 3] = -sg.im;
    v.misc[2] = k + 1;
    const double res = hypot(v.g[2 * k + 2], v.g[2 * k + 3]);
    scale[c] = hn > 0.0 ? 1.0 / hn : 0.0;
    if (res <= tol * v.misc[3] || hn == 0.0 || !isfinite(res)) {
      v.misc[1] = 1.0;  // converged (or breakdown: the Krylov space is invariant)
      atomicSub(active, 1);
    }
  }
}

// y = H(0:s, 0:s)^{-1} g(0:s) (upper triangular, s = steps of the cycle), into
// coef[q][c] for the correction sum_q y_q V_q
__global__ void k_gm_solve(int ncol, int m, const double* __restrict__ GS, double* __restrict__ coef) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x) {
    GmView v(const_cast<double*>(GS) + (size_t)c * gm_state_stride(m), m);
    const int st = (int)v.misc[2];
    for (int q = 0; q < m; ++q) {
      coef[2 * (q * ncol + c)] = 0.0;
      coef[2 * (q * ncol + c) + 1] = 0.0;
    }
    for (int i = st - 1; i >= 0; --i) {
      cd acc{v.g[2 * i], v.g[2 * i + 1]};
      for (int j = i + 1; j < st; ++j) {
        const double* Hj = v.H + (size_t)2 * (m + 1) * j;
        const cd t = cmul(cd{Hj[2 * i], Hj[2 * i + 1]}, cd{coef[2 * (j * ncol + c)], coef[2 * (j * ncol + c) + 1]});
        acc.re -= t.re;
        acc.im -= t.im;
      }
      const double* Hi = v.H + (size_t)2 * (m + 1) * i;
      const cd y = cdivz(acc, cd{Hi[2 * i], Hi[2 * i + 1]});
      coef[2 * (i * ncol + c)] = y.re;
      coef[2 * (i * ncol + c) + 1] = y.im;
    }
  }
}

__global__ void k_gm_set_bnorm(int ncol, int m, double* __restrict__ GS, const double* __restrict__ bn) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncol; c += gridDim.x * blockDim.x)
    GS[(size_t)c * gm_state_stride(m) + gm_state_stride(m) - 1] = bn[c];
}

// Jacobi preconditioner apply for GMRES: out = Dinv x
template <class T, bool CPLX>
__global__ void k_gm_jacobi(long n, int ld, int ncol, const T* __restrict__ dinv, const T* __restrict__ x,
                            T* __restrict__ out) {
  const long total = n * (long)ncol;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / ncol;
    const int c = (int)(e % ncol);
    if constexpr (CPLX) {
      const T dr = dinv[2 * r], di = dinv[2 * r + 1];
      const T xr = x[(size_t)r * ld + 2 * c], xi = x[(size_t)r * ld + 2 * c + 1];
      out[(size_t)r * ld + 2 * c] = dr * xr - di * xi;
      out[(size_t)r * ld + 2 * c + 1] = dr * xi + di * xr;
    } else {
      out[(size_t)r * ld + c] = dinv[r] * x[(size_t)r * ld + c];
    }
  }
}

template <class T, bool CPLX, int TPR, int NVPT>
static KrylovResult run_gmres(const OpT<T>& op, cd sigma, const KArgs<T>& a, int pmode, double tol, int maxit,
                              KrylovWork<T>& w, int grid, cudaStream_t s) {
  KrylovResult res;
  const long n = op.n;
  const int ld = a.ld, m = w.gm_restart;
  const int ncol = CPLX ? a.cols / 2 : a.cols;
  const long blk = n * (long)ld;
  const int dctas = gm_dot_ctas();
  const int eg = device_sms() * 4;
  double* bn = w.out;                   // ||b|| per column
  double* scale = w.out + kMaxRealCols; // per-column scale factors
  double* h1 = w.GH;                    // (m+1) x ncol complex
  double* h2 = w.GH + (size_t)(m + 1) * kMaxRealCols;
  double* nw = w.partial;               // norm^2 per column (complex layout)
  int* active = &w.hdr->n_active;
  T* R = w.R;    // residual / new Arnoldi vector
  T* X = w.X;    // solution
  T* Zb = w.GZ;  // preconditioned vector
  auto dots = [&](const T* Vq, int nq, const T* Wv, double* out) {
    k_gm_dots<T, CPLX><<<dctas, 256, 0, s>>>(n, ld, ncol, Vq, blk, nq, Wv, w.GP);
    CARE_LAUNCH();
    k_gm_dots_reduce<<<(nq * ncol + 127) / 128, 128, 0, s>>>(dctas, nq * ncol, w.GP, out);
    CARE_LAUNCH();
  };
  auto precond = [&](const T* x, T* out) {
    if (pmode == 2) {
      ilu_apply<T, TPR, NVPT, CPLX>(a, x, out, grid, s);
    } else if (pmode == 1) {
      k_gm_jacobi<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, a.Dinv, x, out);
      CARE_LAUNCH();
    } else {
      CARE_CUDA(cudaMemcpyAsync(out, x, sizeof(T) * blk, cudaMemcpyDeviceToDevice, s));
    }
  };
  SpmmArgs<T> sp{};
  sp.n = n; sp.rp = op.rp; sp.ci = op.ci; sp.av = op.val; sp.rs = op.rowsum; sp.ldx = ld; sp.ldy = ld;
  sp.nvec = a.nvec; sp.sre = sigma.re; sp.sim = sigma.im;
  auto matvec = [&](const T* x, T* y) {
    sp.X = x; sp.Y = y;
    launch_spmm<T, 0, CPLX>(sp, s);
  };
  // x = 0, r = b (padded block copy of the right-hand side)
  CARE_CUDA(cudaMemsetAsync(X, 0, sizeof(T) * blk, s));
  k_gm_copy_in<T><<<eg, 256, 0, s>>>(a, R);
  CARE_LAUNCH();
  int steps_total = 0;
  bool first = true;
  for (;;) {
    // cycle start: beta = ||r||, v_0 = r / beta
    dots(R, 1, R, nw);
    CARE_CUDA(cudaMemsetAsync(active, 0, sizeof(int), s));
    k_gm_start<<<1, 128, 0, s>>>(ncol, m, nw, w.GS, bn, first ? 1 : 0, tol, scale, active);
    CARE_LAUNCH();
    if (first) {
      k_gm_set_bnorm<<<1, 128, 0, s>>>(ncol, m, w.GS, bn);
      CARE_LAUNCH();
    }
    first = false;
    int act = 0;
    CARE_CUDA(cudaMemcpyAsync(&act, active, sizeof(int), cudaMemcpyDeviceToHost, s));
    CARE_CUDA(cudaStreamSynchronize(s));
    if (act == 0 || steps_total >= maxit) break;
    k_gm_scale<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, R, scale, w.GV);
    CARE_LAUNCH();
    int k = 0;
    for (; k < m && steps_total < maxit; ++k) {
      T* vk = w.GV + (size_t)k * blk;
      precond(vk, Zb);
      matvec(Zb, R);  // w = A M^{-1} v_k
      ++res.spmm;
      // classical Gram-Schmidt, twice
      dots(w.GV, k + 1, R, h1);
      k_gm_combine<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, R, 1.0, w.GV, blk, k + 1, h1, -1.0);
      CARE_LAUNCH();
      dots(w.GV, k + 1, R, h2);
      k_gm_combine<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, R, 1.0, w.GV, blk, k + 1, h2, -1.0);
      CARE_LAUNCH();
      dots(R, 1, R, nw);
      k_gm_arnoldi<<<1, 128, 0, s>>>(ncol, m, k, h1, h2, nw, w.GS, tol, scale, active);
      CARE_LAUNCH();
      k_gm_scale<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, R, scale, w.GV + (size_t)(k + 1) * blk);
      CARE_LAUNCH();
      ++steps_total;
      if ((k + 1) % 4 == 0) {
        CARE_CUDA(cudaMemcpyAsync(&act, active, sizeof(int), cudaMemcpyDeviceToHost, s));
        CARE_CUDA(cudaStreamSynchronize(s));
        if (act == 0) {
          ++k;
          break;
        }
      }
    }
    // x += M^{-1} (V y), then the true residual r = b - A x for the restart test.
    // Only the k basis blocks built in this cycle take part: later blocks hold an
    // earlier cycle's vectors or never-written memory, and a zero coefficient times
    // a non-finite stale entry would still poison the sum
    if (k == 0) break;
    k_gm_solve<<<1, 128, 0, s>>>(ncol, m, w.GS, h1);
    CARE_LAUNCH();
    CARE_CUDA(cudaMemsetAsync(R, 0, sizeof(T) * blk, s));
    k_gm_combine<T, CPLX><<<eg, 256, 0, s>>>(n, ld, ncol, R, 0.0, w.GV, blk, k, h1, 1.0);
    CARE_LAUNCH();
    precond(R, Zb);
    axpby<T>(n, ld, 1.0, Zb, ld, 1.0, X, ld, s);
    matvec(X, Zb);
    ++res.spmm;
    k_gm_copy_in<T><<<eg, 256, 0, s>>>(a, R);
    CARE_LAUNCH();
    axpby<T>(n, ld, -1.0, Zb, ld, 1.0, R, ld, s);
  }
  res.iters = steps_total;
  return res;
}

template <class T>
KrylovResult krylov_gmres(const OpT<T>& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol, int ld_sol,
                          int cols, double tol, int maxit, int precond, KrylovWork<T>& w, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T);
  CARE_REQUIRE(w.gm_restart > 0 && w.GV, CARE_ERR_INVALID_ARG, "gmres: workspace has no basis");
  CARE_REQUIRE(cols <= kMaxRealCols && cols > 0, CARE_ERR_INVALID_ARG, "gmres: bad width");
  CARE_REQUIRE(!cplx || cols % 2 == 0, CARE_ERR_INVALID_ARG, "gmres: odd complex width");
  int pmode = 0;
  const bool ilu_req = precond == CARE_PRECOND_ILU0 || precond == CARE_PRECOND_ILU0_EXACT;
  if (ilu_req && w.ilu && op.full_diag) pmode = 2;
  else if ((precond == CARE_PRECOND_JACOBI || ilu_req) && !op.diag_const && w.Ph != nullptr)
    pmode = 1;
  const bool exact = pmode == 2 && precond == CARE_PRECOND_ILU0_EXACT;
  KArgs<T> a{};
  a.exact = exact ? 1 : 0;
  a.iflags = w.iflags; a.iticket = w.iticket; a.ierr = w.ierr;
  a.n = op.n;
  a.ld = pad_ld<T>(cols);
  a.nvec = a.ld / VEC;
  a.X = w.X; a.R = w.R;
  a.Dinv = w.Dinv;
  a.rhs = rhs; a.ld_rhs = ld_rhs; a.sol = sol; a.ld_sol = ld_sol; a.cols = cols;
  a.st = w.st; a.hdr = w.hdr;
  a.rp = op.rp; a.ci = op.ci; a.dpos = w.dpos; a.Y1 = w.Y1; a.Y2 = w.Y2; a.Y3 = w.Y3;
  a.tri_sweeps = w.tri_sweeps < 1 ? 1 : w.tri_sweeps;
  const int tpr = tpr_for(a.nvec);
  const int nvpt = (a.nvec + 31) / 32;
  const int grid = grid_rows(op.n, tpr);
  CARE_CUDA(cudaMemsetAsync(w.hdr, 0, sizeof(KHeader), s));
  if (pmode == 1) {
    k_dinv<T><<<device_sms() * 4, kBlock, 0, s>>>(op.n, op.diag, sigma.re, sigma.im, cplx, w.Dinv);
    CARE_LAUNCH();
  } else if (pmode == 2) {
    a.F = exact ? ilu_exact_setup<T>(op, sigma, cplx, w, s) : ilu_setup<T>(op, sigma, cplx, w, s);
  }
  // the tolerance is applied to the true residual at every restart and to the
  // Givens estimate within a cycle; the per-column ||b|| sits in the last state slot
  KrylovResult r;
#define CARE_GM_CASE(TP, NV)                                                               \
  if (tpr == TP && nvpt == NV) {                                                           \
    r = cplx ? run_gmres<T, true, TP, NV>(op, sigma, a, pmode, tol, maxit, w, grid, s)     \
             : run_gmres<T, false, TP, NV>(op, sigma, a, pmode, tol, maxit, w, grid, s);   \
    goto gm_done;                                                                          \
  }
  CARE_GM_CASE(1, 1) CARE_GM_CASE(2, 1) CARE_GM_CASE(4, 1) CARE_GM_CASE(8, 1)
  CARE_GM_CASE(16, 1) CARE_GM_CASE(32, 1) CARE_GM_CASE(32, 2)
#undef CARE_GM_CASE
  CARE_THROW(CARE_ERR_INVALID_ARG, "gmres: unsupported width");
gm_done:
  k_copy_out<T><<<device_sms() * 4, kBlock, 0, s>>>(a);
  CARE_LAUNCH();
  {
    // unconverged columns: the flag of the last cycle's start test
    const int ncol = cplx ? cols / 2 : cols;
    std::vector<double> st(gm_state_stride(w.gm_restart) * ncol);
    CARE_CUDA(cudaMemcpyAsync(st.data(), w.GS, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, s));
    int ierr = 0;
    if (exact) CARE_CUDA(cudaMemcpyAsync(&ierr, w.ierr, sizeof(int), cudaMemcpyDeviceToHost, s));
    CARE_CUDA(cudaStreamSynchronize(s));
    CARE_REQUIRE(ierr == 0, CARE_TIMEOUT, "exact ILU(0): a bounded wait expired");
    for (int c = 0; c < ncol; ++c)
      if (st[(size_t)c * gm_state_stride(w.gm_restart) + 2 * (w.gm_restart + 1) * w.gm_restart + w.gm_restart +
             2 * w.gm_restart + 2 * (w.gm_restart + 1) + 1] == 0.0)
        ++r.unconverged;
    const double sv = sizeof(T), sf = sv * (cplx ? 2 : 1);
    const double blkb = (double)op.n * a.ld * sv;
    const double amat = (double)op.nnz * (sv + 4) + 4.0 * (op.n + 1) + (op.rowsum ? sv * op.n : 0.0);
    // per Arnoldi step k: matvec (2 passes + operator), preconditioner, two CGS
    // passes of (k+2) + (k+2) block passes, the norm and the scaling (3 passes)
    const double avgk = 0.5 * std::min(w.gm_restart, std::max(r.iters, 1));
    double per = amat + 2 * blkb + 4 * (avgk + 2) * blkb + 3 * blkb;
    if (pmode == 2) per += 2.0 * a.tri_sweeps * (3 * blkb + 0.5 * op.nnz * (sf + 4));
    r.bytes = per * r.iters;
  }
  return r;
}
template KrylovResult krylov_gmres<float>(const OpT<float>&, cd, bool, const float*, int, float*, int, int, double,
                                          int, int, KrylovWork<float>&, cudaStream_t);
template KrylovResult krylov_gmres<double>(const OpT<double>&, cd, bool, const double*, int, double*, int, int,
                                           double, int, int, KrylovWork<double>&, cudaStream_t);

template <class T>
void ilu0_factor(const OpT<T>& op, cd sigma, bool cplx, bool exact, KrylovWork<T>& w, T* F, cudaStream_t s) {
  CARE_REQUIRE(w.ilu && op.full_diag, CARE_ERR_INVALID_ARG, "ilu0: needs the ILU workspace and a full diagonal");
  const T* f = exact ? ilu_exact_setup<T>(op, sigma, cplx, w, s) : ilu_setup<T>(op, sigma, cplx, w, s);
  CARE_CUDA(cudaMemcpyAsync(F, f, sizeof(T) * (size_t)op.nnz * (cplx ? 2 : 1), cudaMemcpyDeviceToDevice, s));
  int ierr = 0;
  if (exact) CARE_CUDA(cudaMemcpyAsync(&ierr, w.ierr, sizeof(int), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  CARE_REQUIRE(ierr == 0, CARE_TIMEOUT, "exact ILU(0): a bounded wait expired");
}
template void ilu0_factor<float>(const OpT<float>&, cd, bool, bool, KrylovWork<float>&, float*, cudaStream_t);
template void ilu0_factor<double>(const OpT<double>&, cd, bool, bool, KrylovWork<double>&, double*, cudaStream_t);

template KrylovResult krylov_bicgstab<float>(const OpT<float>&, cd, bool, const float*, int, float*, int,
                                             int, double, int, int, KrylovWork<float>&, cudaStream_t);
template KrylovResult krylov_bicgstab<double>(const OpT<double>&, cd, bool, const double*, int, double*,
                                              int, int, double, int, int, KrylovWork<double>&,
                                              cudaStream_t);

}  // namespace care
