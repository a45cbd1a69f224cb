// Tensor-core (tcgen05 + TMA) products of the tall-skinny contractions.
//
// Two arithmetic modes share one kernel:
//  * FP64-accurate (slices): every FP64 operand row is scaled by a power of two
//    2^-e (its largest entry below 1), rounded to a 56-bit fixed-point integer and
//    split exactly into 8 signed 7-bit slices (round-to-nearest digits, |s_0| <= 128,
//    |s_a| <= 64 for a >= 1), each stored in BF16 as s_a 2^-7(a+1) (exact: at most
//    8 significant bits).  The slice products s_a t_b 2^-7(a+b+2) are exact in the
//    tensor core; the 43 pairs with a + b <= 8 are accumulated in FP32 in TMEM.
//    Pairs with a + b <= 4 go to one accumulator per a + b ("exact groups"): over a
//    chunk of 128 K-rows their sums are integers below 2^22 in units of
//    2^-7(a+b+2), so FP32 holds them exactly in any summation order; after every
//    chunk they are read back, converted to integers and added into one int64
//    fixed-point accumulator per output entry (exact).  Pairs with a + b >= 5 carry
//    weights below 2^-35 of the leading term and go to a single FP32 tail
//    accumulator.  The result (int64 * 2^-42 + tail) * 2^(e_i + f_j) differs from
//    the exact product of the FP64 inputs by the 56-bit input rounding (2^-57
//    relative to each row's largest entry), the dropped pairs (below 2^-63 of it)
//    and the tail's FP32 rounding, while the leading sums are exact: no larger than
//    the accumulation error of an FP64 dot product.  This is the splitting idea of
//    Ozaki et al. (Numer. Algorithms 59, 2012), realised with exact integer chunk
//    sums because B300 has neither a fast FP64 nor INT8 tensor path.
//  * TF32 / BF16 (plain): FP32 inputs rounded by the tensor core (kind::tf32) or
//    converted to BF16 (kind::f16), FP32 accumulation in TMEM.
//
// Operands are K-major (row i of A holds A(i, k) for consecutive k), staged by TMA
// (3-D tensor maps: k, row, slice; 64-byte rows with the 64-byte swizzle, zero
// fill outside the valid range) into a shared-memory ring; one thread issues
// tcgen05.mma with a 128 x 64 FP32 tile per accumulator in TMEM; eight epilogue
// warps read TMEM with tcgen05.ld.  Every wait on an mbarrier is bounded in time;
// on expiry the kernel records an error code and returns after its copies and
// products have drained.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace care {

// Device scratch of the tensor-core products (inside a caller workspace).
struct TcScratch {
  uint16_t* slices = nullptr;  // BF16 slice storage (or FP32 staging in the plain modes)
  size_t slice_bytes = 0;
  int* expo = nullptr;         // per-row exponents of both operands
  size_t expo_elems = 0;
  double* part = nullptr;      // split-K partial tiles
  size_t part_elems = 0;
  int* err = nullptr;          // device error word (0 = ok)
  bool ok() const { return slices != nullptr && part != nullptr && err != nullptr; }
};

// Bytes of scratch that tc_alloc carves from an arena for products whose operand
// widths add up to at most `maxdim` (a + b for X^T Y, a + b for X S).
size_t tc_scratch_bytes(int maxdim);
TcScratch tc_alloc(Arena& ar, int maxdim);

// True if the tensor-core path is compiled in and the device supports it.
bool tc_available();
// Process-wide switch: 0 = off, 1 = on where profitable (default), 2 = every FP64
// product of the solver (tests).
void tc_set_enabled(int on);
int tc_enabled();

// Whether the FP64-accurate tensor-core path takes a product of this shape
// (a, b: output sizes; k: contraction length).
bool tc_f64_profitable(long k, int a, int b);

// G (a x b, FP64, ldg) = X^T Y, X (n x a, ldx) and Y (n x b, ldy) row-major FP64,
// FP64-accurate slices on the tensor cores.  X == Y (same pointer and ld, a == b)
// computes the upper tiles only and mirrors them.
void tc_gram_f64(long n, int a, int b, const double* X, int ldx, const double* Y, int ldy, double* G, int ldg,
                 const TcScratch& sc, int maxdim, cudaStream_t s);

// Y (n x b, ldy) = alpha X S + beta Y with X (n x a, ldx) row-major FP64 and S
// (a x b, lds) row-major FP64 on the device; FP64-accurate slices.  To = float or
// double.
template <class To>
void tc_gemm_ts_f64(long n, int a, int b, double alpha, const double* X, int ldx, const double* S, int lds,
                    double beta, To* Y, int ldy, const TcScratch& sc, int maxdim, cudaStream_t s);

// FP32-accurate counterparts for FP32 operands: 4 slices (28-bit fixed point per
// row), the 10 pairs with a + b <= 3, all accumulated exactly (the dropped pairs
// are below 2^-28 of the leading term, under the FP32 unit roundoff).
void tc_gram_f32acc(long n, int a, int b, const float* X, int ldx, const float* Y, int ldy, double* G, int ldg,
                    const TcScratch& sc, int maxdim, cudaStream_t s);
template <class To>
void tc_gemm_ts_f32acc(long n, int a, int b, double alpha, const float* X, int ldx, const double* S, int lds,
                       double beta, To* Y, int ldy, const TcScratch& sc, int maxdim, cudaStream_t s);

// G (a x b, FP64, ldg) = X^T Y for FP32 X, Y (row-major) with TF32 (kind = 1)
// or BF16 (kind = 2) inputs and FP32 accumulation on the tensor cores.
void tc_gram_lowp(int kind, long n, int a, int b, const float* X, int ldx, const float* Y, int ldy, double* G,
                  int ldg, const TcScratch& sc, int maxdim, cudaStream_t s);

// Test hook: while on, the product kernels issue no operand copies, so their first
// bounded wait expires and they return through the error path.
void tc_set_test_starve(int on);

// Reads and clears the device error word (synchronises s).  Returns the code.
int tc_check(const TcScratch& sc, cudaStream_t s);

}  // namespace care
