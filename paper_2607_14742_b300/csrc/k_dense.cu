// Tall-skinny dense kernels on the CUDA cores (FP32 / FP64 FMA).
//
// gram:    G = X^T Y, a, b up to a few thousand, n up to 1e6.  Output tiles
//          of 64 x 64 per CTA, rows split across CTAs (split-K, the split chosen
//          to balance the CTAs over the SMs); each CTA stages 32-row slabs of X
//          and Y in shared memory, accumulates a 4 x 4 register tile per thread,
//          and writes an FP64 partial; a second kernel sums the partials in a
//          fixed order (deterministic).  X^T X computes only the upper tiles.
// gemm_ts: Y = alpha X S + beta Y with S small (a x b): 64-row x 64-column
//          output tiles, the contraction over a staged 32 columns at a time.
#include "dense.cuh"

namespace care {

constexpr int GT = 64;   // output tile
constexpr int GK = 32;   // rows (gram) / inner columns (gemm_ts) per stage

// Row slices (split-K) of a Gram product.  Each CTA owns one 64 x 64 output
// tile and one slice of rows; the CUDA-core FMA pipe is the bound, so the
// time goes with the CTAs queued on the busiest SM times the rows per CTA:
// ceil(tiles * split / SMs) / split, minimised over split (ties to the
// smaller split) with at least 4 staging slabs per CTA and split * a * b
// partials within cap_elems.  A symmetric product (X^T X) has only the
// ta (ta + 1) / 2 tiles on and above the diagonal.
constexpr size_t GRAM_SCRATCH_TARGET = size_t(1) << 24;  // doubles (128 MB)

static long gram_split(long n, int a, int b, bool sym, size_t cap_elems) {
  const long ta = (a + GT - 1) / GT, tb = (b + GT - 1) / GT;
  const long tiles = sym ? ta * (ta + 1) / 2 : ta * tb;
  const long sms = device_sms();
  long smax = (n + 4 * GK - 1) / (4 * GK);
  const long by_cap = (long)(std::min(cap_elems, GRAM_SCRATCH_TARGET) / ((size_t)a * b));
  smax = std::min(smax, std::min(by_cap, 8 * sms));
  if (smax < 1) return 1;
  long best = 1;
  double best_cost = (double)((tiles + sms - 1) / sms);
  for (long sp = 2; sp <= smax; ++sp) {
    const double cost = (double)((tiles * sp + sms - 1) / sms) / (double)sp;
    if (cost < best_cost * 0.995) {
      best_cost = cost;
      best = sp;
    }
  }
  return best;
}

size_t gram_work_elems(long n, int a, int b) {
  long split = gram_split(n, a, b, false, GRAM_SCRATCH_TARGET);
  if (a == b) split = std::max(split, gram_split(n, a, b, true, GRAM_SCRATCH_TARGET));
  return (size_t)split * a * b;
}

// X^T Y is computed as a symmetric product when Y is X itself
template <class T>
static bool gram_is_sym(int a, int b, const T* X, int ldx, const T* Y, int ldy) {
  return a == b && X == Y && ldx == ldy;
}

template <class T>
__global__ void __launch_bounds__(256) k_gram(long n, int a, int b, const T* __restrict__ X, int ldx,
                                              const T* __restrict__ Y, int ldy, long rows_per,
                                              double* __restrict__ part, bool sym) {
  __shared__ T xs[GK][GT];
  __shared__ T ys[GK][GT];
  const int ta = blockIdx.y, tb = blockIdx.z;
  if (sym && tb < ta) return;  // strictly lower tile of a symmetric product (whole CTA)
  const int i0 = ta * GT, j0 = tb * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  T acc[4][4];
  double accd[4][4];  // FP32 inputs: FP64 accumulation of 32-row FP32 partial sums
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      acc[u][v] = T(0);
      accd[u][v] = 0.0;
    }
  const long r_begin = (long)blockIdx.x * rows_per;
  long r_end = r_begin + rows_per;
  if (r_end > n) r_end = n;
  for (long r0 = r_begin; r0 < r_end; r0 += GK) {
    // stage GK rows x GT columns of X and Y (zero outside)
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int k = e / GT, c = e % GT;
      const long r = r0 + k;
      const bool rin = r < r_end;
      xs[k][c] = (rin && i0 + c < a) ? X[(size_t)r * ldx + i0 + c] : T(0);
      ys[k][c] = (rin && j0 + c < b) ? Y[(size_t)r * ldy + j0 + c] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      T xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = xs[k][ty * 4 + u];
#pragma unroll
      for (int v = 0; v < 4; ++v) yv[v] = ys[k][tx * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xv[u], yv[v], acc[u][v]);
    }
    if constexpr (sizeof(T) == 4) {
      // each 32-row FP32 partial sum is flushed into FP64 (keeps the FP32
      // rounding to 32-term sums; the inner solves are sensitive to it)
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          accd[u][v] += (double)acc[u][v];
          acc[u][v] = T(0);
        }
    }
    __syncthreads();
  }
  // compact partial layout [split][a][b]: only valid entries are written
  double* out = part + (size_t)blockIdx.x * a * b;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u;
    if (i >= a) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int j = j0 + tx * 4 + v;
      if (j < b) out[(size_t)i * b + j] = sizeof(T) == 4 ? accd[u][v] : (double)acc[u][v];
    }
  }
}

// one warp per output: lanes sum strided partials, then a fixed xor-shuffle tree;
// a symmetric product reads the strictly lower tiles from their mirror image
__global__ void k_gram_reduce(int a, int b, long split, const double* __restrict__ part, double* __restrict__ G,
                              int ldg, bool sym) {
  const long total = (long)a * b;
  const int lane = threadIdx.x & 31;
  const long warps = (long)gridDim.x * (blockDim.x / 32);
  for (long e = (blockIdx.x * (long)blockDim.x + threadIdx.x) / 32; e < total; e += warps) {
    const int i = (int)(e / b), j = (int)(e % b);
    const long src = (sym && j / GT < i / GT) ? (long)j * b + i : e;
    double s0 = 0.0, s1 = 0.0;
    long g = lane;
    for (; g + 32 < split; g += 64) {
      s0 += part[(size_t)g * total + src];
      s1 += part[(size_t)(g + 32) * total + src];
    }
    if (g < split) s0 += part[(size_t)g * total + src];
    double v = s0 + s1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) G[(size_t)i * ldg + j] = v;
  }
}

template <class T>
void gram(long n, int a, int b, const T* X, int ldx, const T* Y, int ldy, double* G, int ldg,
          double* work, size_t work_elems, cudaStream_t s) {
  if (a == 0 || b == 0) return;
  const int ta = (a + GT - 1) / GT, tb = (b + GT - 1) / GT;
  const bool sym = gram_is_sym(a, b, X, ldx, Y, ldy);
  CARE_REQUIRE((size_t)a * b <= work_elems, CARE_ERR_WORKSPACE, "gram: scratch too small");
  const long split = gram_split(n, a, b, sym, work_elems);
  const size_t need = (size_t)split * a * b;
  const long rows_per = ((n + split - 1) / split + GK - 1) / GK * GK;
  if (n == 0) {
    CARE_CUDA(cudaMemsetAsync(work, 0, need * sizeof(double), s));
  } else {
    dim3 grid((unsigned)split, ta, tb);
    k_gram<T><<<grid, 256, 0, s>>>(n, a, b, X, ldx, Y, ldy, rows_per, work, sym);
    CARE_LAUNCH();
  }
  const long tot = (long)a * b;
  int g = (int)((tot + 7) / 8);  // 8 warps per CTA, one output per warp
  if (g > device_sms() * 8) g = device_sms() * 8;
  k_gram_reduce<<<g, 256, 0, s>>>(a, b, n == 0 ? 1 : split, work, G, ldg, sym);
  CARE_LAUNCH();
}
template void gram<float>(long, int, int, const float*, int, const float*, int, double*, int, double*,
                          size_t, cudaStream_t);
template void gram<double>(long, int, int, const double*, int, const double*, int, double*, int, double*,
                           size_t, cudaStream_t);

template <class Ti, class To>
__global__ void __launch_bounds__(256) k_gemm_ts(long n, int a, int b, double alpha,
                                                 const Ti* __restrict__ X, int ldx,
                                                 const double* __restrict__ S, int lds, double beta,
                                                 To* __restrict__ Y, int ldy) {
  __shared__ Ti xs[GT][GK + 1];
  __shared__ Ti ss[GK][GT];
  const long r0 = (long)blockIdx.x * GT;
  const int j0 = blockIdx.y * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  Ti acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = Ti(0);
  for (int k0 = 0; k0 < a; k0 += GK) {
    for (int e = threadIdx.x; e < GT * GK; e += 256) {
      const int r = e / GK, k = e % GK;
      const long rr = r0 + r;
      xs[r][k] = (rr < n && k0 + k < a) ? X[(size_t)rr * ldx + k0 + k] : Ti(0);
    }
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int k = e / GT, c = e % GT;
      ss[k][c] = (k0 + k < a && j0 + c < b) ? (Ti)S[(size_t)(k0 + k) * lds + j0 + c] : Ti(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < GK; ++k) {
      Ti xv[4], sv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = xs[ty * 4 + u][k];
#pragma unroll
      for (int v = 0; v < 4; ++v) sv[v] = ss[k][tx * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xv[u], sv[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long r = r0 + ty * 4 + u;
    if (r >= n) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = j0 + tx * 4 + v;
      if (c >= b) continue;
      const size_t o = (size_t)r * ldy + c;
      double y = alpha * (double)acc[u][v];
      if (beta != 0.0) y += beta * (double)Y[o];
      Y[o] = (To)y;
    }
  }
}

template <class Ti, class To>
void gemm_ts(long n, int a, int b, double alpha, const Ti* X, int ldx, const double* S, int lds,
             double beta, To* Y, int ldy, cudaStream_t s) {
  if (n == 0 || b == 0) return;
  if (a == 0) {
    // Y = beta Y
    if (beta == 1.0) return;
    copy2d<To, To>(n, b, Y, ldy, 1, Y, ldy, 1, beta, s);
    return;
  }
  dim3 grid((unsigned)((n + GT - 1) / GT), (b + GT - 1) / GT);
  k_gemm_ts<Ti, To><<<grid, 256, 0, s>>>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy);
  CARE_LAUNCH();
}
template void gemm_ts<float, float>(long, int, int, double, const float*, int, const double*, int, double,
                                    float*, int, cudaStream_t);
template void gemm_ts<double, double>(long, int, int, double, const double*, int, const double*, int,
                                      double, double*, int, cudaStream_t);
template void gemm_ts<double, float>(long, int, int, double, const double*, int, const double*, int,
                                     double, float*, int, cudaStream_t);
template void gemm_ts<float, double>(long, int, int, double, const float*, int, const double*, int,
                                     double, double*, int, cudaStream_t);

// ---------------------------------------------------------------- copies --
template <class Ti, class To>
__global__ void k_copy2d(long rows, int cols, const Ti* __restrict__ src, long srs, long scs,
                         To* __restrict__ dst, long drs, long dcs, double scale) {
  // 32 x 32 tile: read with threadIdx.x along the source's contiguous index,
  // write with threadIdx.x along the destination's contiguous index.
  __shared__ double tile[32][33];
  const long bi = (long)blockIdx.x * 32;
  const int bj = blockIdx.y * 32;
  const bool src_rowmajor = (scs == 1);
  const bool dst_rowmajor = (dcs == 1);
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    long i;
    int j;
    if (src_rowmajor) { i = bi + t; j = bj + threadIdx.x; }
    else { i = bi + threadIdx.x; j = bj + t; }
    double v = 0.0;
    if (i < rows && j < cols) v = (double)src[i * srs + (long)j * scs];
    tile[i - bi][j - bj] = v;
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    long i;
    int j;
    if (dst_rowmajor) { i = bi + t; j = bj + threadIdx.x; }
    else { i = bi + threadIdx.x; j = bj + t; }
    if (i < rows && j < cols) dst[i * drs + (long)j * dcs] = (To)(scale * tile[i - bi][j - bj]);
  }
}

template <class Ti, class To>
void copy2d(long rows, int cols, const Ti* src, long src_rs, long src_cs, To* dst, long dst_rs,
            long dst_cs, double scale, cudaStream_t s) {
  if (rows == 0 || cols == 0) return;
  dim3 grid((unsigned)((rows + 31) / 32), (cols + 31) / 32);
  dim3 block(32, 8);
  k_copy2d<Ti, To><<<grid, block, 0, s>>>(rows, cols, src, src_rs, src_cs, dst, dst_rs, dst_cs, scale);
  CARE_LAUNCH();
}
template void copy2d<float, float>(long, int, const float*, long, long, float*, long, long, double,
                                   cudaStream_t);
template void copy2d<double, double>(long, int, const double*, long, long, double*, long, long, double,
                                     cudaStream_t);
template void copy2d<double, float>(long, int, const double*, long, long, float*, long, long, double,
                                    cudaStream_t);
template void copy2d<float, double>(long, int, const float*, long, long, double*, long, long, double,
                                    cudaStream_t);

template <class T>
__global__ void k_axpby(long n, int cols, double alpha, const T* __restrict__ X, int ldx, double beta,
                        T* __restrict__ Y, int ldy) {
  const long total = n * (long)cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / cols;
    const int c = (int)(e % cols);
    T& y = Y[(size_t)r * ldy + c];
    const double v = alpha * (double)X[(size_t)r * ldx + c] + (beta != 0.0 ? beta * (double)y : 0.0);
    y = (T)v;
  }
}
template <class T>
void axpby(long n, int cols, double alpha, const T* X, int ldx, double beta, T* Y, int ldy,
           cudaStream_t s) {
  if (n == 0 || cols == 0) return;
  k_axpby<T><<<device_sms() * 4, 256, 0, s>>>(n, cols, alpha, X, ldx, beta, Y, ldy);
  CARE_LAUNCH();
}
template void axpby<float>(long, int, double, const float*, int, double, float*, int, cudaStream_t);
template void axpby<double>(long, int, double, const double*, int, double, double*, int, cudaStream_t);

// LR-ADI update for a complex pair (p, conj p) in real arithmetic, elementwise:
// with V = SOL (complex interleaved, column q at 2q, 2q+1) and u = Re V + d Im V,
//   W(:, q) += g^2 u_q;
//   q < rp:  Zp(:, q) = g u_q,          Zp(:, rp + q) = gi Im V_q;
//   q >= rp: Zm(:, q - rp) = g u_q,     Zm(:, rm + q - rp) = gi Im V_q   (rm = b - rp).
template <class T>
__global__ void k_cpair_update(long n, int b, int rp, const T* __restrict__ sol, int ldr, double g, double d,
                               double gi, T* __restrict__ W, int ldw, T* __restrict__ Zp, T* __restrict__ Zm,
                               int ldz) {
  const long total = n * (long)b;
  const int rm = b - rp;
  const T tg = (T)g, td = (T)d, tgi = (T)gi, tg2 = (T)(g * g);
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / b;
    const int q = (int)(e % b);
    const T re = sol[(size_t)r * ldr + 2 * q], im = sol[(size_t)r * ldr + 2 * q + 1];
    const T u = re + td * im;
    W[(size_t)r * ldw + q] += tg2 * u;
    if (q < rp) {
      Zp[(size_t)r * ldz + q] = tg * u;
      Zp[(size_t)r * ldz + rp + q] = tgi * im;
    } else {
      Zm[(size_t)r * ldz + (q - rp)] = tg * u;
      Zm[(size_t)r * ldz + rm + (q - rp)] = tgi * im;
    }
  }
}
template <class T>
void cpair_update(long n, int b, int rp, const T* sol, int ldr, double g, double d, double gi, T* W, int ldw, T* Zp,
                  T* Zm, int ldz, cudaStream_t s) {
  if (n == 0 || b == 0) return;
  k_cpair_update<T><<<device_sms() * 4, 256, 0, s>>>(n, b, rp, sol, ldr, g, d, gi, W, ldw, Zp, Zm, ldz);
  CARE_LAUNCH();
}
template void cpair_update<float>(long, int, int, const float*, int, double, double, double, float*, int, float*,
                                  float*, int, cudaStream_t);
template void cpair_update<double>(long, int, int, const double*, int, double, double, double, double*, int,
                                   double*, double*, int, cudaStream_t);

template <class T>
__global__ void k_scale_cols(long n, int cols, T* __restrict__ Y, int ldy, const double* __restrict__ d) {
  const long total = n * (long)cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / cols;
    const int c = (int)(e % cols);
    Y[(size_t)r * ldy + c] = (T)((double)Y[(size_t)r * ldy + c] * d[c]);
  }
}
template <class T>
void scale_cols(long n, int cols, T* Y, int ldy, const double* d, cudaStream_t s) {
  if (n == 0 || cols == 0) return;
  k_scale_cols<T><<<device_sms() * 4, 256, 0, s>>>(n, cols, Y, ldy, d);
  CARE_LAUNCH();
}
template void scale_cols<float>(long, int, float*, int, const double*, cudaStream_t);
template void scale_cols<double>(long, int, double*, int, const double*, cudaStream_t);

// ------------------------------------------------- allocation-free Gram ----
// Scratch for care_gram_noalloc: a fixed file-scope device array, so the entry
// point never allocates.  The CUDA driver reserves it when it loads this module on a
// device (with lazy loading: at the first call into the library there), and
// that device holds it until the process exits.  Host code must not pass the symbol itself to a kernel
// (in host code it names a host-side stand-in); its device address is looked
// up once per device with cudaGetSymbolAddress.
static __device__ __align__(256) double g_gram_noalloc_scratch[CARE_GRAM_NOALLOC_SCRATCH_DOUBLES];

}  // namespace care

#include <mutex>

namespace care {

static double* gram_noalloc_scratch_ptr(int dev) {
  static std::mutex mu;
  static double* ptrs[64] = {nullptr};
  CARE_REQUIRE(dev >= 0 && dev < 64, CARE_ERR_INVALID_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    CARE_CUDA(cudaGetSymbolAddress(&p, g_gram_noalloc_scratch));
    ptrs[dev] = static_cast<double*>(p);
  }
  return ptrs[dev];
}

template <class T>
void gram_noalloc(long n, int a, int b, const T* X, int ldx, const T* Y, int ldy, double* G, int ldg,
                  cudaStream_t s) {
  if (a == 0 || b == 0) return;
  const long cap = CARE_GRAM_NOALLOC_SCRATCH_DOUBLES;
  CARE_REQUIRE((long)a * b <= cap, CARE_ERR_INVALID_ARG,
               "gram_noalloc: a*b exceeds the fixed scratch (CARE_GRAM_NOALLOC_SCRATCH_DOUBLES)");
  int dev = 0;
  CARE_CUDA(cudaGetDevice(&dev));
  double* work = gram_noalloc_scratch_ptr(dev);
  const int ta = (a + GT - 1) / GT, tb = (b + GT - 1) / GT;
  const bool sym = gram_is_sym(a, b, X, ldx, Y, ldy);
  const long split = gram_split(n, a, b, sym, (size_t)cap);
  const long rows_per = ((n + split - 1) / split + GK - 1) / GK * GK;
  if (n == 0) {
    CARE_CUDA(cudaMemsetAsync(work, 0, (size_t)a * b * sizeof(double), s));
  } else {
    dim3 grid((unsigned)split, ta, tb);
    k_gram<T><<<grid, 256, 0, s>>>(n, a, b, X, ldx, Y, ldy, rows_per, work, sym);
    CARE_LAUNCH();
  }
  const long tot = (long)a * b;
  int g = (int)((tot + 7) / 8);
  if (g > device_sms() * 8) g = device_sms() * 8;
  k_gram_reduce<<<g, 256, 0, s>>>(a, b, n == 0 ? 1 : split, work, G, ldg, sym);
  CARE_LAUNCH();
}
template void gram_noalloc<float>(long, int, int, const float*, int, const float*, int, double*, int, cudaStream_t);
template void gram_noalloc<double>(long, int, int, const double*, int, const double*, int, double*, int,
                                   cudaStream_t);

}  // namespace care

namespace care {

// FP64 FMA throughput of the CUDA cores (roofline denominator of the FP64
// products): 8 independent dependent-FMA chains per thread, full occupancy.
__global__ void __launch_bounds__(256) k_fp64_fma_peak(int iters, double a, double b, double* out) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 12345.678) out[0] = s;  // keeps the chains live
}

double fp64_fma_peak_tflops(cudaStream_t s) {
  const int grid = device_sms() * 8, block = 256, iters = 4096;
  cudaEvent_t e0, e1;
  CARE_CUDA(cudaEventCreate(&e0));
  CARE_CUDA(cudaEventCreate(&e1));
  double best = 0.0;
  for (int rep = 0; rep < 4; ++rep) {
    CARE_CUDA(cudaEventRecord(e0, s));
    k_fp64_fma_peak<<<grid, block, 0, s>>>(iters, 0.9999999, 1e-7, nullptr);
    CARE_LAUNCH();
    CARE_CUDA(cudaEventRecord(e1, s));
    CARE_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    CARE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double fl = 2.0 * 8.0 * iters * (double)grid * block;
    if (rep > 0) best = std::max(best, fl / (ms * 1e-3) * 1e-12);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace care
