// Batched shifted solves for many independent CAREs: one persistent cooperative
// launch runs block BiCGStab (per-column scalars, right Jacobi preconditioning) on
// the shifted systems M_p X = W of every instance that has one pending, over a
// work list of row tiles of all of them (Section 4: the shifted solves are the
// dominant work of NLR-ADI and LR-ADI; batching them over instances is this
// library's serving mode, the paper solves one CARE at a time).
//
//  * Work list: request r has its rows cut into tiles of 256 / nv2 rows (nv2 = the
//    power of two >= its 16-byte vectors per row), one (row, vector) element per
//    thread; tiles of all requests are numbered consecutively and CTAs take them
//    grid-stride, so small and large instances share the SMs.
//  * Phases of one iteration (p update | v = M p^ | alpha | s update | t = M s^ |
//    omega | x, r update | rho, convergence) are separated by grid barriers;
//    dot products are accumulated per thread across a CTA's tiles of a request,
//    combined per CTA in a fixed order into per-(request, CTA) partials, and
//    summed over CTAs in a fixed order by one warp per column: the results are
//    bitwise reproducible for a given batch.
//  * Converged columns (||r|| <= tol ||b||), broken-down ones and requests at their
//    iteration limit are frozen (alpha = omega = beta = 0); the launch ends when no
//    column is active.  The FP32 operator uses the difference form (row sums) as
//    the single-instance SpMM does.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <vector>

#include "batch.cuh"

namespace cg = cooperative_groups;

namespace care {
namespace {

constexpr int BT = 256;  // threads per CTA (one tile)

// Loads of data that other CTAs wrote earlier in the same launch bypass L1 (whose
// lines are not kept coherent across SMs): every block and scalar the phases
// exchange is read this way.
template <class T>
__device__ __forceinline__ void vload_cg(const T* p, T (&v)[16 / sizeof(T)]) {
  using V = typename Vec<T>::type;
  const V x = __ldcg(reinterpret_cast<const V*>(p));
  if constexpr (sizeof(T) == 4) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    v[0] = x.x; v[1] = x.y;
  }
}

struct Cx {
  double re, im;
};
__device__ __forceinline__ Cx cxmul(Cx a, Cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ Cx cxdiv(Cx a, Cx b) {
  // Smith's algorithm for a / b (b != 0)
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.im + b.re * r;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}

// request of tile t (tile0 ascending; nreq <= kBatchMaxReq)
template <class T>
__device__ __forceinline__ int req_of(const BatchArgs<T>& g, int t) {
  int lo = 0, hi = g.nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (g.req[mid].tile0 <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// element (row, vector v) of tile t of request q for this thread; false if idle
template <class T>
__device__ __forceinline__ bool elem_of(const BatchReq<T>& q, int t, long* row, int* v) {
  const int rr = threadIdx.x / q.nv2;
  *v = threadIdx.x % q.nv2;
  *row = (long)(t - q.tile0) * q.rpt + rr;
  return *row < q.n && *v < q.nvec;
}

// scalars of the real column c of request q (complex: the slot of its pair)
template <class T>
__device__ __forceinline__ BatchSlot& slot_of(const BatchArgs<T>& g, const BatchReq<T>& q, int c) {
  return g.slots[q.slot0 + (q.cplx ? c / 2 : c)];
}

// per-thread dot accumulators: acc[d][e] for the thread's VEC real columns
template <class T>
struct DotAcc {
  static constexpr int VEC = 16 / sizeof(T);
  double a[2][VEC];
  __device__ void zero() {
#pragma unroll
    for (int d = 0; d < 2; ++d)
#pragma unroll
      for (int e = 0; e < VEC; ++e) a[d][e] = 0.0;
  }
  // conj(x) y per complex pair (re at even, im at odd), x y per real column
  __device__ void add(int d, bool cplx, const T (&x)[VEC], const T (&y)[VEC]) {
    if (cplx) {
#pragma unroll
      for (int e = 0; e < VEC; e += 2) {
        a[d][e] += (double)x[e] * y[e] + (double)x[e + 1] * y[e + 1];
        a[d][e + 1] += (double)x[e] * y[e + 1] - (double)x[e + 1] * y[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < VEC; ++e) a[d][e] += (double)x[e] * y[e];
    }
  }
};

// Combine the CTA's accumulators for request r (rows of the tile in a fixed order)
// into partial[(pbase_r + b * cols_r + c) * 2 + d].  All threads of the CTA call it.
template <class T>
__device__ void flush_dots(const BatchArgs<T>& g, int r, DotAcc<T>& acc, int ndot, double* sm) {
  constexpr int VEC = 16 / sizeof(T);
  const BatchReq<T>& q = g.req[r];
  __syncthreads();
  for (int d = 0; d < ndot; ++d)
#pragma unroll
    for (int e = 0; e < VEC; ++e) sm[(threadIdx.x * 2 + d) * VEC + e] = acc.a[d][e];
  __syncthreads();
  const int rpt = q.rpt, nv2 = q.nv2;
  for (int k = threadIdx.x; k < ndot * q.cols; k += blockDim.x) {
    const int d = k / q.cols, c = k % q.cols;
    const int v = c / VEC, e = c % VEC;
    double s = 0.0;
    for (int rr = 0; rr < rpt; ++rr) s += sm[((rr * nv2 + v) * 2 + d) * VEC + e];
    g.partial[((size_t)q.pbase + (size_t)blockIdx.x * q.cols + c) * 2 + d] = s;
  }
  acc.zero();
}

// Sum of the partials of column c, dot d, over the CTAs that own tiles of request
// q (fixed order: lanes over CTAs, then a fixed xor tree); valid in every lane.
template <class T>
__device__ double sum_partials(const BatchArgs<T>& g, const BatchReq<T>& q, int c, int d) {
  const int G = gridDim.x;
  const int nb = q.ntiles < G ? q.ntiles : G;
  double s = 0.0;
  for (int k = threadIdx.x & 31; k < nb; k += 32) {
    const int b = (q.tile0 + k) % G;
    s += __ldcg(g.partial + ((size_t)q.pbase + (size_t)b * q.cols + c) * 2 + d);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// complex dot of slot j of request q (d = dot index): (re, im) of sum conj(x) y
template <class T>
__device__ Cx slot_dot(const BatchArgs<T>& g, const BatchReq<T>& q, int j, int d) {
  if (q.cplx) return {sum_partials(g, q, 2 * j, d), sum_partials(g, q, 2 * j + 1, d)};
  return {sum_partials(g, q, j, d), 0.0};
}

enum { PH_INIT = 0, PH_ALPHA = 1, PH_OMEGA = 2, PH_RHO = 3 };

// One warp per slot: the reduction of phase `ph` and the scalar update.
template <class T>
__device__ void reduce_phase(const BatchArgs<T>& g, int ph, int it) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int sidx = gw; sidx < g.nslot; sidx += nw) {
    // request of the slot (slot0 ascending)
    int lo = 0, hi = g.nreq - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (g.req[mid].slot0 <= sidx) lo = mid;
      else hi = mid - 1;
    }
    const BatchReq<T>& q = g.req[lo];
    const int j = sidx - q.slot0;
    BatchSlot& S = g.slots[sidx];
    const Cx d0 = slot_dot(g, q, j, 0);
    Cx d1{0.0, 0.0};
    if (ph != PH_ALPHA) d1 = slot_dot(g, q, j, 1);
    if (lane != 0) continue;
    if (ph == PH_INIT) {
      S.bnorm2 = d1.re;
      S.rnorm2 = d1.re;
      S.rho_re = d0.re;
      S.rho_im = d0.im;
      S.alpha_re = S.alpha_im = S.omega_re = S.omega_im = S.beta_re = S.beta_im = 0.0;
      S.iters = 0;
      S.flag = d1.re > 0.0 ? 0 : 1;  // a zero right-hand side is solved by x = 0
    } else if (S.flag != 0) {
      S.alpha_re = S.alpha_im = S.omega_re = S.omega_im = S.beta_re = S.beta_im = 0.0;
    } else if (ph == PH_ALPHA) {
      if (d0.re == 0.0 && d0.im == 0.0) {
        S.flag = 2;
        S.alpha_re = S.alpha_im = 0.0;
      } else {
        const Cx a = cxdiv(Cx{S.rho_re, S.rho_im}, d0);
        S.alpha_re = a.re;
        S.alpha_im = a.im;
      }
    } else if (ph == PH_OMEGA) {
      // d0 = <t, s>, d1 = <t, t>
      if (d1.re > 0.0) {
        S.omega_re = d0.re / d1.re;
        S.omega_im = d0.im / d1.re;
      } else {
        S.omega_re = S.omega_im = 0.0;
      }
    } else {
      // d0 = <rhat, r>, d1 = <r, r>
      S.rnorm2 = d1.re;
      S.iters = it + 1;
      if (!(d1.re > q.tol2 * S.bnorm2)) {
        S.flag = d1.re <= q.tol2 * S.bnorm2 ? 1 : 2;  // NaN: breakdown
      } else if (it + 1 >= q.maxit) {
        S.flag = 3;
      } else if ((S.omega_re == 0.0 && S.omega_im == 0.0) || (S.rho_re == 0.0 && S.rho_im == 0.0)) {
        S.flag = 2;
      } else {
        const Cx b = cxmul(cxdiv(d0, Cx{S.rho_re, S.rho_im}), cxdiv(Cx{S.alpha_re, S.alpha_im},
                                                                     Cx{S.omega_re, S.omega_im}));
        S.beta_re = b.re;
        S.beta_im = b.im;
      }
      S.rho_re = d0.re;
      S.rho_im = d0.im;
      if (S.flag != 0) S.alpha_re = S.alpha_im = S.omega_re = S.omega_im = S.beta_re = S.beta_im = 0.0;
    }
    if ((ph == PH_INIT || ph == PH_RHO) && S.flag == 0) {
      atomicAdd(g.active, 1);
      atomicAdd(g.ractive_next + lo, 1);
    }
  }
}

// y (VEC reals) = M_p x at element (row, v) of request q
template <class T>
__device__ __forceinline__ void spmv_elem(const BatchReq<T>& q, const T* X, long row, int v, T (&y)[16 / sizeof(T)]) {
  constexpr int VEC = 16 / sizeof(T);
  T xi[VEC], acc[VEC];
  vload_cg(X + (size_t)row * q.ld + v * VEC, xi);
#pragma unroll
  for (int e = 0; e < VEC; ++e) acc[e] = T(0);
  const bool diff = q.rs != nullptr;
  const int s = __ldg(q.rp + row), en = __ldg(q.rp + row + 1);
  for (int j0 = s; j0 < en; j0 += 8) {
    int c[8];
    T a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const bool in = j0 + u < en;
      c[u] = in ? __ldg(q.ci + j0 + u) : (int)row;
      a[u] = in ? __ldg(q.av + j0 + u) : T(0);
    }
    T x[8][VEC];
#pragma unroll
    for (int u = 0; u < 8; ++u) vload_cg(X + (size_t)c[u] * q.ld + v * VEC, x[u]);
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int e = 0; e < VEC; ++e) acc[e] = fma(a[u], diff ? x[u][e] - xi[e] : x[u][e], acc[e]);
  }
  const T dre = (T)q.sre + (diff ? __ldg(q.rs + row) : T(0));
  const T dim = (T)q.sim;
  if (q.cplx) {
#pragma unroll
    for (int e = 0; e < VEC; e += 2) {
      y[e] = acc[e] + dre * xi[e] - dim * xi[e + 1];
      y[e + 1] = acc[e + 1] + dre * xi[e + 1] + dim * xi[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) y[e] = fma(dre, xi[e], acc[e]);
  }
}

// z = Dinv x (complex per pair when cplx)
template <class T>
__device__ __forceinline__ void jacobi_elem(const BatchReq<T>& q, long row, const T (&x)[16 / sizeof(T)],
                                            T (&z)[16 / sizeof(T)]) {
  constexpr int VEC = 16 / sizeof(T);
  if (!q.Dinv) {
#pragma unroll
    for (int e = 0; e < VEC; ++e) z[e] = x[e];
    return;
  }
  if (q.cplx) {
    const T dr = __ldcg(q.Dinv + 2 * row), di = __ldcg(q.Dinv + 2 * row + 1);
#pragma unroll
    for (int e = 0; e < VEC; e += 2) {
      z[e] = dr * x[e] - di * x[e + 1];
      z[e + 1] = dr * x[e + 1] + di * x[e];
    }
  } else {
    const T d = __ldcg(q.Dinv + row);
#pragma unroll
    for (int e = 0; e < VEC; ++e) z[e] = d * x[e];
  }
}

// scalar of the real column c (complex pairs share their slot's complex value)
template <class T>
struct ColScal {
  static constexpr int VEC = 16 / sizeof(T);
  double re[VEC], im[VEC];
};
template <class T>
__device__ __forceinline__ void col_scal(const BatchArgs<T>& g, const BatchReq<T>& q, int v, int which,
                                         ColScal<T>& o) {
  constexpr int VEC = 16 / sizeof(T);
#pragma unroll
  for (int e = 0; e < VEC; ++e) {
    const int c = v * VEC + e;
    if (c >= q.cols) {
      o.re[e] = o.im[e] = 0.0;
      continue;
    }
    const BatchSlot& S = slot_of(g, q, c);
    const double r = __ldcg(which == 0 ? &S.alpha_re : (which == 1 ? &S.omega_re : &S.beta_re));
    const double i = __ldcg(which == 0 ? &S.alpha_im : (which == 1 ? &S.omega_im : &S.beta_im));
    o.re[e] = r;
    o.im[e] = i;
  }
}
// y += s x (complex scalar per pair when cplx)
template <class T>
__device__ __forceinline__ void axpy_elem(bool cplx, const ColScal<T>& s, const T (&x)[16 / sizeof(T)],
                                          T (&y)[16 / sizeof(T)], double sign) {
  constexpr int VEC = 16 / sizeof(T);
  if (cplx) {
#pragma unroll
    for (int e = 0; e < VEC; e += 2) {
      const double sr = sign * s.re[e], si = sign * s.im[e];
      const double yr = y[e] + sr * x[e] - si * x[e + 1];
      const double yi = y[e + 1] + sr * x[e + 1] + si * x[e];
      y[e] = (T)yr;
      y[e + 1] = (T)yi;
    }
  } else {
#pragma unroll
    for (int e = 0; e < VEC; ++e) y[e] = (T)(y[e] + sign * s.re[e] * x[e]);
  }
}

// ractive = the per-request active-column counts of the last reduction; the
// counters for the next one start from zero
template <class T>
__device__ void publish_active(const BatchArgs<T>& g) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < g.nreq; r += gridDim.x * blockDim.x) {
    g.ractive[r] = __ldcg(g.ractive_next + r);
    g.ractive_next[r] = 0;
  }
}

template <class T>
__global__ void __launch_bounds__(BT) k_batch_bicgstab(BatchArgs<T> g) {
  constexpr int VEC = 16 / sizeof(T);
  cg::grid_group grid = cg::this_grid();
  __shared__ double sm[BT * 2 * VEC];
  DotAcc<T> acc;
  acc.zero();
  // Every phase below loops over the tiles of this CTA; `ndot` dot products are
  // flushed whenever the request changes and after the last tile.
  auto tiles = [&](int ndot, auto&& body) {
    int cur = -1;
    for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
      const int r = req_of(g, t);
      // a request whose columns are all frozen is skipped (its scalars ignore the dots)
      if (__ldcg(g.ractive + r) == 0) continue;
      if (r != cur) {
        if (cur >= 0 && ndot) flush_dots(g, cur, acc, ndot, sm);
        cur = r;
      }
      const BatchReq<T>& q = g.req[r];
      long row;
      int v;
      if (elem_of(q, t, &row, &v)) body(q, row, v);
    }
    if (cur >= 0 && ndot) flush_dots(g, cur, acc, ndot, sm);
  };
  // init: Dinv, x = 0, r = rhat = b, p = v = 0; <rhat, r>, <r, r>
  tiles(2, [&](const BatchReq<T>& q, long row, int v) {
    const size_t o = (size_t)row * q.ld + v * VEC;
    T b[VEC], z[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int c = v * VEC + e;
      b[e] = c < q.cols ? q.rhs[(size_t)row * q.ld_rhs + c] : T(0);
      z[e] = T(0);
    }
    if (v == 0 && q.Dinv) {
      const double dre = (double)q.diag[row] + q.sre, dim = q.sim;
      if (q.cplx) {
        const double den = dre * dre + dim * dim;
        q.Dinv[2 * row] = (T)(den > 0.0 ? dre / den : 1.0);
        q.Dinv[2 * row + 1] = (T)(den > 0.0 ? -dim / den : 0.0);
      } else {
        q.Dinv[row] = (T)(dre != 0.0 ? 1.0 / dre : 1.0);
      }
    }
    vstore(q.X + o, z);
    vstore(q.P + o, z);
    vstore(q.V + o, z);
    vstore(q.R + o, b);
    vstore(q.Rh + o, b);
    acc.add(0, q.cplx, b, b);
    acc.add(1, q.cplx, b, b);
  });
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.active = 0;
  grid.sync();
  reduce_phase(g, PH_INIT, 0);
  grid.sync();
  publish_active(g);
  grid.sync();
  int it = 0;
  while (*(volatile int*)g.active > 0 && it < g.maxit) {
    // p = r + beta (p - omega v);  p^ = Dinv p
    tiles(0, [&](const BatchReq<T>& q, long row, int v) {
      const size_t o = (size_t)row * q.ld + v * VEC;
      ColScal<T> be, om;
      col_scal(g, q, v, 2, be);
      col_scal(g, q, v, 1, om);
      T p[VEC], vv[VEC], r[VEC], ph[VEC];
      vload_cg(q.P + o, p);
      vload_cg(q.V + o, vv);
      vload_cg(q.R + o, r);
      axpy_elem<T>(q.cplx, om, vv, p, -1.0);  // p - omega v
      T t[VEC];
#pragma unroll
      for (int e = 0; e < VEC; ++e) t[e] = r[e];
      axpy_elem<T>(q.cplx, be, p, t, 1.0);    // r + beta (p - omega v)
      vstore(q.P + o, t);
      jacobi_elem(q, row, t, ph);
      vstore(q.Ph + o, ph);
    });
    grid.sync();
    // v = M p^;  <rhat, v>
    tiles(1, [&](const BatchReq<T>& q, long row, int v) {
      const size_t o = (size_t)row * q.ld + v * VEC;
      T y[VEC], rh[VEC];
      spmv_elem(q, q.Ph, row, v, y);
      vstore(q.V + o, y);
      vload_cg(q.Rh + o, rh);
      acc.add(0, q.cplx, rh, y);
    });
    if (blockIdx.x == 0 && threadIdx.x == 0) *g.active = 0;
    grid.sync();
    reduce_phase(g, PH_ALPHA, it);
    grid.sync();
    // s = r - alpha v;  s^ = Dinv s
    tiles(0, [&](const BatchReq<T>& q, long row, int v) {
      const size_t o = (size_t)row * q.ld + v * VEC;
      ColScal<T> al;
      col_scal(g, q, v, 0, al);
      T r[VEC], vv[VEC], sh[VEC];
      vload_cg(q.R + o, r);
      vload_cg(q.V + o, vv);
      axpy_elem<T>(q.cplx, al, vv, r, -1.0);
      vstore(q.S + o, r);
      jacobi_elem(q, row, r, sh);
      vstore(q.Sh + o, sh);
    });
    grid.sync();
    // t = M s^;  <t, s>, <t, t>
    tiles(2, [&](const BatchReq<T>& q, long row, int v) {
      const size_t o = (size_t)row * q.ld + v * VEC;
      T y[VEC], s[VEC];
      spmv_elem(q, q.Sh, row, v, y);
      vstore(q.Tt + o, y);
      vload_cg(q.S + o, s);
      acc.add(0, q.cplx, y, s);
      acc.add(1, q.cplx, y, y);
    });
    grid.sync();
    reduce_phase(g, PH_OMEGA, it);
    grid.sync();
    // x += alpha p^ + omega s^;  r = s - omega t;  <rhat, r>, <r, r>
    tiles(2, [&](const BatchReq<T>& q, long row, int v) {
      const size_t o = (size_t)row * q.ld + v * VEC;
      ColScal<T> al, om;
      col_scal(g, q, v, 0, al);
      col_scal(g, q, v, 1, om);
      T x[VEC], ph[VEC], sh[VEC], s[VEC], tt[VEC], rh[VEC];
      vload_cg(q.X + o, x);
      vload_cg(q.Ph + o, ph);
      vload_cg(q.Sh + o, sh);
      axpy_elem<T>(q.cplx, al, ph, x, 1.0);
      axpy_elem<T>(q.cplx, om, sh, x, 1.0);
      vstore(q.X + o, x);
      vload_cg(q.S + o, s);
      vload_cg(q.Tt + o, tt);
      axpy_elem<T>(q.cplx, om, tt, s, -1.0);
      vstore(q.R + o, s);
      vload_cg(q.Rh + o, rh);
      acc.add(0, q.cplx, rh, s);
      acc.add(1, q.cplx, s, s);
    });
    grid.sync();
    reduce_phase(g, PH_RHO, it);
    grid.sync();
    publish_active(g);
    grid.sync();
    ++it;
  }
  // sol = x (valid columns) for every request
  for (int r = 0; r < g.nreq && threadIdx.x == 0 && blockIdx.x == 0; ++r) g.ractive[r] = 1;
  grid.sync();
  tiles(0, [&](const BatchReq<T>& q, long row, int v) {
    const size_t o = (size_t)row * q.ld + v * VEC;
    T x[VEC];
    vload_cg(q.X + o, x);
#pragma unroll
    for (int e = 0; e < VEC; ++e) {
      const int c = v * VEC + e;
      if (c < q.cols) q.sol[(size_t)row * q.ld_sol + c] = x[e];
    }
  });
  if (blockIdx.x == 0 && threadIdx.x == 0) *g.iters = it;
}

}  // namespace

size_t batch_scratch_bytes(int max_req) {
  Arena a;
  a.get<BatchReq<double>>((size_t)max_req);
  a.get<BatchSlot>((size_t)max_req * kMaxRealCols);
  a.get<int>(64);
  a.get<int>((size_t)2 * max_req);
  a.get<double>((size_t)max_req * (size_t)device_sms() * 8 * kMaxRealCols * 2);
  return a.off + 256;
}

template <class T>
int batch_launch(std::vector<BatchReq<T>>& reqs, char* scratch, size_t scratch_bytes, cudaStream_t s,
                 std::vector<BatchSlot>* slots_out) {
  constexpr int VEC = 16 / sizeof(T);
  const int nreq = (int)reqs.size();
  CARE_REQUIRE(nreq > 0 && nreq <= kBatchMaxReq, CARE_ERR_INVALID_ARG, "batch: request count");
  int per_sm = 0;
  CARE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_bicgstab<T>, BT, 0));
  CARE_REQUIRE(per_sm >= 1, CARE_ERR_CUDA, "batch: kernel cannot be resident");
  const int G = device_sms() * std::min(per_sm, 8);
  // tiles, slots and partial offsets
  int tiles = 0, nslot = 0;
  size_t pb = 0;
  int maxit = 0;
  for (auto& q : reqs) {
    CARE_REQUIRE(q.cols > 0 && q.cols <= kMaxRealCols && (!q.cplx || q.cols % 2 == 0), CARE_ERR_INVALID_ARG,
                 "batch: request width");
    q.ld = pad_ld<T>(q.cols);
    q.nvec = q.ld / VEC;
    int nv2 = 1;
    while (nv2 < q.nvec) nv2 <<= 1;
    q.nv2 = nv2;
    q.rpt = BT / nv2;
    q.tile0 = tiles;
    q.ntiles = (int)((q.n + q.rpt - 1) / q.rpt);
    tiles += q.ntiles;
    q.slot0 = nslot;
    nslot += q.cplx ? q.cols / 2 : q.cols;
    q.pbase = pb;
    pb += (size_t)G * q.cols;
    maxit = std::max(maxit, q.maxit);
  }
  Arena a;
  a.base = scratch;
  a.cap = scratch_bytes;
  BatchReq<T>* dreq = a.get<BatchReq<T>>((size_t)nreq);
  BatchSlot* dslot = a.get<BatchSlot>((size_t)std::max(nslot, 1));
  int* misc = a.get<int>(64);
  int* ract = a.get<int>((size_t)2 * nreq);
  double* partial = a.get<double>(pb * 2);
  CARE_CUDA(cudaMemcpyAsync(dreq, reqs.data(), sizeof(BatchReq<T>) * nreq, cudaMemcpyHostToDevice, s));
  {
    std::vector<int> init(2 * (size_t)nreq, 0);
    for (int r = 0; r < nreq; ++r) init[r] = 1;  // every request takes part in the first phase
    CARE_CUDA(cudaMemcpyAsync(ract, init.data(), sizeof(int) * 2 * nreq, cudaMemcpyHostToDevice, s));
    CARE_CUDA(cudaStreamSynchronize(s));  // the host vector goes out of scope
  }
  BatchArgs<T> g{};
  g.req = dreq;
  g.nreq = nreq;
  g.ntiles = tiles;
  g.slots = dslot;
  g.nslot = nslot;
  g.partial = partial;
  g.active = misc;
  g.iters = misc + 1;
  g.ractive = ract;
  g.ractive_next = ract + nreq;
  g.maxit = maxit;
  void* args[] = {(void*)&g};
  CARE_CUDA(cudaLaunchCooperativeKernel((const void*)k_batch_bicgstab<T>, dim3(G), dim3(BT), args, 0, s));
  count_launch();
  int it = 0;
  CARE_CUDA(cudaMemcpyAsync(&it, g.iters, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (slots_out) {
    slots_out->resize(nslot);
    CARE_CUDA(cudaMemcpyAsync(slots_out->data(), dslot, sizeof(BatchSlot) * nslot, cudaMemcpyDeviceToHost, s));
  }
  CARE_CUDA(cudaStreamSynchronize(s));
  return it;
}
template int batch_launch<float>(std::vector<BatchReq<float>>&, char*, size_t, cudaStream_t,
                                 std::vector<BatchSlot>*);
template int batch_launch<double>(std::vector<BatchReq<double>>&, char*, size_t, cudaStream_t,
                                  std::vector<BatchSlot>*);

// ------------------------------------------------------------ broker -------
struct BatchBroker::Impl {
  std::mutex mu;
  std::condition_variable cv;
  int active = 0;      // instances still solving
  bool leader = false;  // a batch is being assembled or run
  struct Pending {
    void* req;  // BatchReq<T>*
    int instance;
    bool done = false, failed = false;
    int iters = 0, unconverged = 0;
  };
  std::vector<Pending*> pending;
  char* scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaStream_t stream = nullptr;
  int elem = 8;
  double wait_ms = 2.0;
  long long launches = 0, requests = 0;
};

BatchBroker::BatchBroker(int instances, int elem_bytes, char* scratch, size_t scratch_bytes) : p(new Impl) {
  p->active = instances;
  p->elem = elem_bytes;
  p->scratch = scratch;
  p->scratch_bytes = scratch_bytes;
  CARE_CUDA(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
}
BatchBroker::~BatchBroker() {
  if (p->stream) cudaStreamDestroy(p->stream);
  delete p;
}
void BatchBroker::instance_done() {
  std::lock_guard<std::mutex> lk(p->mu);
  p->active--;
  p->cv.notify_all();
}
long long BatchBroker::launches() const { return p->launches; }
long long BatchBroker::requests() const { return p->requests; }

template <class T>
KrylovResult BatchBroker::solve(BatchReq<T> q, cudaStream_t caller) {
  // the request's inputs were produced on the caller's stream
  cudaEvent_t ready;
  CARE_CUDA(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  CARE_CUDA(cudaEventRecord(ready, caller));
  CARE_CUDA(cudaEventSynchronize(ready));
  CARE_CUDA(cudaEventDestroy(ready));
  Impl::Pending me;
  me.req = &q;
  std::unique_lock<std::mutex> lk(p->mu);
  p->pending.push_back(&me);
  p->cv.notify_all();
  while (!me.done) {
    if (p->leader) {
      p->cv.wait(lk);
      continue;
    }
    // lead: wait (briefly) until every active instance has a request pending
    p->leader = true;
    const auto t0 = std::chrono::steady_clock::now();
    p->cv.wait_until(lk, t0 + std::chrono::microseconds((long)(p->wait_ms * 1000)),
                     [&] { return (int)p->pending.size() >= p->active; });
    std::vector<Impl::Pending*> batch;
    const size_t take = std::min(p->pending.size(), (size_t)kBatchMaxReq);
    batch.assign(p->pending.begin(), p->pending.begin() + take);
    p->pending.erase(p->pending.begin(), p->pending.begin() + take);
    lk.unlock();
    std::vector<BatchReq<T>> reqs;
    reqs.reserve(batch.size());
    for (auto* b : batch) reqs.push_back(*static_cast<BatchReq<T>*>(b->req));
    std::vector<BatchSlot> slots;
    int it = 0;
    bool ok = true;
    try {
      it = batch_launch<T>(reqs, p->scratch, p->scratch_bytes, p->stream, &slots);
    } catch (...) {
      ok = false;
    }
    lk.lock();
    for (size_t k = 0; k < batch.size(); ++k) {
      Impl::Pending* b = batch[k];
      b->iters = it;
      int unc = 0;
      if (ok) {
        const BatchReq<T>& r = reqs[k];
        const int ns = r.cplx ? r.cols / 2 : r.cols;
        int mx = 0;
        for (int j = 0; j < ns; ++j) {
          const BatchSlot& S = slots[r.slot0 + j];
          mx = std::max(mx, S.iters);
          if (S.flag != 1) unc += r.cplx ? 2 : 1;
        }
        b->iters = mx;
      } else {
        unc = reqs[k].cols;
      }
      b->unconverged = unc;
      b->failed = !ok;
      b->done = true;
    }
    p->launches++;
    p->requests += (long long)batch.size();
    p->leader = false;
    p->cv.notify_all();
  }
  lk.unlock();
  CARE_REQUIRE(!me.failed, CARE_ERR_CUDA, "batched shifted solve: launch failed");
  KrylovResult r;
  r.iters = me.iters;
  r.unconverged = me.unconverged;
  r.spmm = 2LL * me.iters;
  return r;
}
template KrylovResult BatchBroker::solve<float>(BatchReq<float>, cudaStream_t);
template KrylovResult BatchBroker::solve<double>(BatchReq<double>, cudaStream_t);

}  // namespace care
