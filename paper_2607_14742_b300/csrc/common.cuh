// Shared utilities of the CARE library: error handling, workspace arena,
// small complex helpers and the launch geometry of the row-block kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "care_b300.h"

namespace care {

// ---------------------------------------------------------------- errors --
struct CudaError {
  cudaError_t err;
  const char* what;
  int line;
};
struct StatusError {
  care_status status;
  const char* what;
};

#define CARE_CUDA(x)                                                         \
  do {                                                                       \
    cudaError_t care_e_ = (x);                                               \
    if (care_e_ != cudaSuccess) throw ::care::CudaError{care_e_, #x, __LINE__}; \
  } while (0)
// every kernel launch site ends with CARE_LAUNCH(): it checks the launch and
// counts it (care_kernel_launches)
void count_launch();
void count_launch_n(long delta);
#define CARE_LAUNCH()               \
  do {                              \
    ::care::count_launch();         \
    CARE_CUDA(cudaGetLastError());  \
  } while (0)
#define CARE_THROW(st, msg) throw ::care::StatusError{st, msg}
#define CARE_REQUIRE(cond, st, msg) \
  do {                              \
    if (!(cond)) CARE_THROW(st, msg); \
  } while (0)

int device_sms();          // SM count of the current device (cached per device)
int verbose_level();       // set per call from care_opts.verbose
void set_verbose(int v);

// --------------------------------------------------------------- arena ----
// Bump allocator over caller-provided device memory.  With base == nullptr it
// only counts, which is how the workspace queries are answered: the query runs
// the same allocation sequence as the solver.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  size_t peak = 0;
  bool counting() const { return base == nullptr; }
  template <class T>
  T* get(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (!counting() && off + bytes > cap) CARE_THROW(CARE_ERR_WORKSPACE, "workspace too small");
    T* p = counting() ? nullptr : reinterpret_cast<T*>(base + off);
    off += bytes;
    if (off > peak) peak = off;
    return p;
  }
  size_t mark() const { return off; }
  void release(size_t m) { off = m; }
};

// -------------------------------------------------------------- complex ---
struct cd {
  double re, im;
};
__host__ __device__ inline cd cmul(cd a, cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ inline cd cdivz(cd a, cd b) {
  // Smith's algorithm (Smith 1962) for a / b.
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  double r = b.re / b.im, d = b.im + b.re * r;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
__host__ __device__ inline cd cconj(cd a) { return {a.re, -a.im}; }

// ------------------------------------------------------------ vectors -----
template <class T>
struct Vec;
template <>
struct Vec<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <class T>
__device__ __forceinline__ void vload(const T* p, T (&v)[16 / sizeof(T)]) {
  using V = typename Vec<T>::type;
  V x = *reinterpret_cast<const V*>(p);
  if constexpr (sizeof(T) == 4) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    v[0] = x.x; v[1] = x.y;
  }
}
// the same through the read-only (non-coherent) data path, for blocks that no
// thread of the running kernel writes
template <class T>
__device__ __forceinline__ void vload_ro(const T* p, T (&v)[16 / sizeof(T)]) {
  using V = typename Vec<T>::type;
  const V x = __ldg(reinterpret_cast<const V*>(p));
  if constexpr (sizeof(T) == 4) {
    v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
  } else {
    v[0] = x.x; v[1] = x.y;
  }
}
template <class T>
__device__ __forceinline__ void vstore(T* p, const T (&v)[16 / sizeof(T)]) {
  using V = typename Vec<T>::type;
  V x;
  if constexpr (sizeof(T) == 4) {
    x.x = v[0]; x.y = v[1]; x.z = v[2]; x.w = v[3];
  } else {
    x.x = v[0]; x.y = v[1];
  }
  *reinterpret_cast<V*>(p) = x;
}

// Leading dimension (in reals) of a row-major block with `cols` real columns:
// padded to a whole number of 16-byte vectors.
template <class T>
inline int pad_ld(int cols) {
  const int v = 16 / sizeof(T);
  return ((cols + v - 1) / v) * v;
}

// Threads per row for a row of `nvec` 16-byte vectors: the smallest power of two
// >= nvec, at most 32; rows wider than 32 vectors loop (NVPT vectors per thread).
inline int tpr_for(int nvec) {
  int t = 1;
  while (t < nvec && t < 32) t <<= 1;
  return t;
}

constexpr int kBlock = 256;    // threads per CTA of the row-block kernels
constexpr int kMaxRealCols = 128;  // widest row-block handled by the fused kernels

// CTAs per SM of the row-block kernels (set by care_autotune; default 8)
int tuned_ctas_per_sm();
void set_tuned_ctas_per_sm(int v);
// 16-byte vectors per thread of the SpMM (1, 2 or 4): fewer threads per row,
// more independent gathers in flight each.  One value per width class of the
// block (vectors per row <= 2, <= 4, <= 8, <= 16, more), set by care_autotune,
// default 1.
constexpr int kSpmmBuckets = 5;
inline int spmm_bucket(int nvec) { return nvec <= 2 ? 0 : nvec <= 4 ? 1 : nvec <= 8 ? 2 : nvec <= 16 ? 3 : 4; }
int tuned_spmm_vpt(int nvec);
void set_tuned_spmm_vpt(int v);                 // every width class
void set_tuned_spmm_vpt_bucket(int bucket, int v);
// SpMM row order: 1 = contiguous row blocks per CTA, 0 = grid-stride (set by care_autotune)
int tuned_spmm_blocked();
void set_tuned_spmm_blocked(int v);
// SpMM thread shape for a row of nvec vectors: tpr threads of nvpt vectors each
// (tpr a power of two <= 32, nvpt <= vpt; every pair this returns for nvec <= 64
// has a kernel instance)
inline void spmm_shape(int nvec, int vpt, int* tpr, int* nvpt) {
  if (vpt < 1) vpt = 1;
  int t = tpr_for((nvec + vpt - 1) / vpt);
  int v = (nvec + t - 1) / t;
  if (v > 4) {
    t = 32;
    v = (nvec + 31) / 32;
  }
  *tpr = t;
  *nvpt = v < 1 ? 1 : v;
}

inline int grid_rows(long rows, int tpr, int ctas_per_sm = 0) {
  if (ctas_per_sm <= 0) ctas_per_sm = tuned_ctas_per_sm();
  long rows_per_cta = (kBlock / 32) * (32 / tpr);
  long need = (rows + rows_per_cta - 1) / rows_per_cta;
  long cap = (long)device_sms() * ctas_per_sm;
  long g = need < cap ? need : cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace care
