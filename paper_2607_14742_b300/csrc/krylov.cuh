// Sparse operator, fused SpMM and the block BiCGStab shifted solver.
#pragma once

#include "common.cuh"

namespace care {

// A^T in CSR with values of type T (the prepared operator of care_op).
template <class T>
struct OpT {
  int n = 0, nnz = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const T* val = nullptr;
  const T* diag = nullptr;
  const T* rowsum = nullptr;  // set: apply in the difference form (FP32 operator)
  bool diag_const = true;
  bool full_diag = false;
};
OpT<double> op64(const care_op& op);
OpT<float> op32(const care_op& op);

// Per-column state of the block BiCGStab recurrences (one entry per real
// column, or per complex column in complex mode).  Scalars are kept in FP64.
struct KState {
  double rho_re, rho_im, alpha_re, alpha_im, omega_re, omega_im, beta_re, beta_im;
  double bnorm2, rnorm2;
  int flag;  // 0 active, 1 converged, 2 breakdown
  int iters;
};
struct KHeader {
  int n_active;
  unsigned counter;
  int pad[2];
};

// Workspace of one block Krylov solve of at most kMaxRealCols real columns.
template <class T>
struct KrylovWork {
  T *X = nullptr, *R = nullptr, *Rh = nullptr, *P = nullptr, *V = nullptr, *S = nullptr, *Tt = nullptr;
  T *Ph = nullptr, *Sh = nullptr, *Dinv = nullptr;
  // ILU(0) factors (ping-pong for the fixed-point sweeps), diagonal positions,
  // and the temporaries of the triangular Jacobi sweeps
  bool ilu = false;
  T *F0 = nullptr, *F1 = nullptr, *Y1 = nullptr, *Y2 = nullptr, *Y3 = nullptr;
  int* dpos = nullptr;
  int ilu_sweeps = 3, tri_sweeps = 2;
  KState* st = nullptr;
  KHeader* hdr = nullptr;
  double* partial = nullptr;
  double* out = nullptr;
  int n = 0;
  // restarted GMRES (allocated when gm_restart > 0): restart + 1 basis blocks,
  // the preconditioned block, per-column Hessenberg / Givens state, dot scratch
  int gm_restart = 0;
  T *GV = nullptr, *GZ = nullptr;
  double *GS = nullptr, *GH = nullptr, *GP = nullptr;
  // exact ILU(0): ready flags per row, the row ticket, the error word
  int *iflags = nullptr, *iticket = nullptr, *ierr = nullptr;
};
// nnz_ilu >= 0 also allocates the ILU(0) preconditioner for an operator with
// that many entries (jacobi must then be true: the factor uses Ph / Sh / Dinv).
template <class T>
KrylovWork<T> krylov_alloc(Arena& ar, int n, bool jacobi, long nnz_ilu = -1, int gmres_restart = 0);

struct KrylovResult {
  int iters = 0;
  int unconverged = 0;  // columns not converged (limit or breakdown)
  long long spmm = 0;
  double bytes = 0.0;   // algorithmic HBM bytes of the solve (see krylov_bicgstab)
};

// Preconditioner of a solve: 0 none, 1 Jacobi, 2 ILU(0).
// Solves (A^T + sigma I) X = RHS for `cols` real columns (complex interleaved
// columns when cplx: cols = 2 * complex columns), cols <= kMaxRealCols.
// rhs/sol are row-major with leading dimensions ld_rhs / ld_sol (reals).
template <class T>
KrylovResult krylov_bicgstab(const OpT<T>& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol,
                             int ld_sol, int cols, double tol, int maxit, int precond,
                             KrylovWork<T>& w, cudaStream_t s);

// Restarted GMRES(restart) on the same systems, one Krylov space per column
// (complex columns in complex arithmetic), right-preconditioned (precond as above)
// so that the stopping test is on the true residual: per-column relative residual
// <= tol; maxit caps the Arnoldi steps (matrix products) of each column.  Classical
// Gram-Schmidt with reorthogonalisation, Givens rotations on the Hessenberg matrix.
template <class T>
KrylovResult krylov_gmres(const OpT<T>& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol, int ld_sol,
                          int cols, double tol, int maxit, int precond, KrylovWork<T>& w, cudaStream_t s);

// Dense-direct shifted solve (Section 4's dense direct solvers): M_p formed densely
// from the operator, LU with partial pivoting, all `cols` real columns at once
// (complex interleaved when cplx).  iters = 1; unconverged = cols if a pivot was
// exactly zero.  Synchronises s.
template <class T>
struct DluWork {
  T* M = nullptr;     // n x n (complex: 2 n^2) column-major factors
  int* ipiv = nullptr;
  T* cbuf = nullptr;  // two copies of the next pivot column
  int* info = nullptr;
  int n = 0;
};
template <class T>
DluWork<T> dlu_alloc(Arena& ar, int n);
template <class T>
KrylovResult dense_lu_solve(const care_op& op, cd sigma, bool cplx, const T* rhs, int ld_rhs, T* sol, int ld_sol,
                            int cols, const DluWork<T>& w, cudaStream_t s);

// The ILU(0) factor of M_p (fixed-point sweeps, or exact) copied into F (values on
// the pattern of A^T; complex interleaved when cplx).  Synchronises s.
template <class T>
void ilu0_factor(const OpT<T>& op, cd sigma, bool cplx, bool exact, KrylovWork<T>& w, T* F, cudaStream_t s);

// Y = (A^T + sigma I) X on `cols` real columns (any width; complex when cplx).
template <class T>
void spmm(const OpT<T>& op, cd sigma, bool cplx, const T* X, int ldx, T* Y, int ldy, int cols,
          cudaStream_t s);

}  // namespace care
