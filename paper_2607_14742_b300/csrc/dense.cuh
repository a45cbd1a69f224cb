// Tall-skinny dense kernels: Gram matrices X^T Y, block products X S, layout
// conversions, and the host small-dense routines.
#pragma once

#include <functional>

#include "common.cuh"

namespace care {

// G (a x b, row-major, FP64, ldg) = X^T Y for row-major X (n x a) and Y (n x b).
size_t gram_work_elems(long n, int a, int b);
template <class T>
void gram(long n, int a, int b, const T* X, int ldx, const T* Y, int ldy, double* G, int ldg,
          double* work, size_t work_elems, cudaStream_t s);

// Same product with the split-K scratch in a fixed file-scope device array
// (no allocation, no workspace argument); a * b <= CARE_GRAM_NOALLOC_SCRATCH_DOUBLES.
template <class T>
void gram_noalloc(long n, int a, int b, const T* X, int ldx, const T* Y, int ldy, double* G, int ldg,
                  cudaStream_t s);

// Y (n x b, row-major To, ldy) = alpha X S + beta Y,  X row-major Ti (n x a, ldx),
// S device FP64 row-major (a x b, lds).
template <class Ti, class To>
void gemm_ts(long n, int a, int b, double alpha, const Ti* X, int ldx, const double* S, int lds,
             double beta, To* Y, int ldy, cudaStream_t s);

// dst(i, j) = scale * src(i, j) for i < rows, j < cols with independent row
// and column strides (any layout; a 32x32 shared-memory tile makes both sides
// coalesced when one is row-major and the other column-major).
template <class Ti, class To>
void copy2d(long rows, int cols, const Ti* src, long src_rs, long src_cs, To* dst, long dst_rs,
            long dst_cs, double scale, cudaStream_t s);

// Y = alpha X + beta Y (row-major, same shape)
template <class T>
void axpby(long n, int cols, double alpha, const T* X, int ldx, double beta, T* Y, int ldy,
           cudaStream_t s);

// LR-ADI complex-pair update (elementwise, see k_dense.cu): W += g^2 (Re V + d Im V);
// the new X_+ columns g (Re V + d Im V), gi Im V of the first rp columns go to Zp,
// those of the other b - rp columns to Zm.  V complex interleaved (ldr reals).
template <class T>
void cpair_update(long n, int b, int rp, const T* sol, int ldr, double g, double d, double gi, T* W, int ldw, T* Zp,
                  T* Zm, int ldz, cudaStream_t s);

// Y(:, j) *= d[j] (row-major; d on device, FP64)
template <class T>
void scale_cols(long n, int cols, T* Y, int ldy, const double* d, cudaStream_t s);

// Symmetric eigendecomposition on the device (k_syev.cu): all eigenvalues of the
// n x n matrix S (device, row-major, lds; returned ascending in w on the host) and
// the eigenvectors of those for which want(w_i, max|w|) holds, written as rows of
// V (device, length n each, in ascending eigenvalue order); returns their indices.
// work: dev_symeig_work_elems(n) doubles of device scratch.
// weighted = false: the vectors are orthonormal to working accuracy (clusters of
// eigenvalues closer than 1e-6 ||T|| orthogonalised explicitly).  weighted = true:
// for callers that only use the vectors weighted by their eigenvalues (V diag(f(w))
// with |f(w)| <= |w|^(1/2)...|w|): clusters are also split where the gap exceeds 1e-3
// of the eigenvalues' magnitude, which keeps the weighted loss of orthogonality
// below about 1e3 eps ||S|| but not V's own orthogonality among tiny eigenvalues.
size_t dev_symeig_work_elems(int n);
std::vector<int> dev_symeig_select(int n, const double* S, int lds, std::vector<double>& w, double* V,
                                   const std::function<bool(double, double)>& want, double* work,
                                   size_t work_elems, cudaStream_t s, bool weighted = false);

// measured FP64 FMA throughput of the CUDA cores (TFLOP/s)
double fp64_fma_peak_tflops(cudaStream_t s);

// ---- host small dense (column-major) ---------------------------------------
// symmetric eigendecomposition, ascending eigenvalues; V may be null
bool host_symeig(int n, const double* A, double* w, double* V);
// the same with only the eigenvectors t for which want(w[t], max_i |w[i]|) holds
// (the other columns of V are zero); all eigenvalues are returned
bool host_symeig_select(int n, const double* A, double* w, double* V,
                        const std::function<bool(double, double)>& want);
// largest eigenvalue of a symmetric matrix (Lanczos; full eig for small n)
double host_sym_lmax(int n, const double* G);
// eigenvalues of a general real matrix
bool host_eigvals(int n, const double* A, double* wr, double* wi);
// upper Cholesky factor of SPD G = R^T R (column-major); false if not SPD
bool host_cholesky_upper(int n, const double* G, double* R);
// rank-revealing Cholesky with complete (diagonal) pivoting of the positive
// semidefinite c x c matrix G (row-major), stopping when the largest remaining
// pivot is <= tol or after max_rank (> 0) pivots; returns the rank r, the pivot
// order and R (r x c, row-major, original column order) with G ~= R^T R
int host_pivoted_cholesky(int c, const double* G, double tol, int max_rank, std::vector<int>& piv,
                          std::vector<double>& R);
// inverse of an upper triangular r x r matrix (row-major in and out)
void host_upper_inverse(int r, const double* U, double* Ui);
// C = A diag(dk) B^T (dk may be null) for row-major A (m x k), B (n x k), C (m x n);
// sym: B is A and only the upper part is computed, then mirrored
void host_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb, const double* dk,
                  double* C, int ldc, bool sym);
// complex LU solve A X = B (A n x n col-major, B n x k col-major), in place on B
bool host_lu_solve_complex(int n, std::vector<cd> A, cd* B, int k);

}  // namespace care
