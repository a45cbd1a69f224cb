/*
 * care_b300.h -- C ABI of the B300 (sm_103a) mixed-precision low-rank CARE solver.
 *
 * Problem (paper Section 1, Eq. (1.1)):  A^T X + X A - X B B^T X + C^T C = 0,
 * A (n x n) sparse and stable, B (n x m), C (p x n), m, p << n; the stabilising
 * solution is returned as a low-rank factor X ~ Z Z^T.
 *
 * Method: Framework 1 of the paper (Section 2) realised with NLR-ADI for the
 * initial approximation and LR-ADI for the correction Lyapunov equations
 * (Section 4).  Shifted solves use a block BiCGStab on M_p = (A + p I)^T with the
 * closed-loop feedback handled by the Sherman-Morrison-Woodbury formula
 * (Section 4).  The residual factor decomposition (Algorithm 1) and the solution
 * factor decomposition (Algorithm 2) always run in FP64.
 *
 * Conventions (all entry points):
 *  - Pointers to matrices are DEVICE pointers unless a parameter says "host".
 *  - Boundary matrices (B, C, K, W, Z, C+, C-) are FP64 COLUMN-MAJOR with the
 *    given leading dimension, as in LAPACK.  The kernel-level entry points
 *    (care_spmm, care_gram, care_shifted_solve) take ROW-MAJOR blocks, the
 *    library's internal layout, with a leading dimension counted in reals.
 *  - The caller owns every buffer.  The library allocates no device memory:
 *    each solver entry point takes a device workspace whose size the matching
 *    *_workspace_size query returns.  Host-side bookkeeping uses ordinary heap
 *    memory.
 *  - Work is issued on the given CUDA stream (0 = legacy default stream).  The
 *    solver entry points synchronise that stream internally (the iteration
 *    control runs on the host), so outputs are complete when they return.
 *    care_spmm and care_gram are asynchronous.
 *  - Errors are reported only through the returned care_status; nothing
 *    throws across the ABI.  After CARE_ERR_CUDA the stream's state is
 *    undefined.
 *  - Not thread-safe per stream: concurrent calls must use distinct streams
 *    and distinct workspaces.
 */
#ifndef CARE_B300_H
#define CARE_B300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* care_stream_t; /* identical to cudaStream_t */

typedef enum {
  CARE_OK = 0,
  CARE_ERR_INVALID_ARG = 1,   /* bad size, null pointer, leading dimension too small   */
  CARE_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed            */
  CARE_ERR_WORKSPACE = 3,     /* work_bytes smaller than the workspace query's result   */
  CARE_ERR_RANK_CAPACITY = 4, /* a factor would exceed its column capacity              */
  CARE_NOT_CONVERGED = 5,     /* k_max refinement steps without reaching tol (Z valid)  */
  CARE_STAGNATED = 6,         /* residual ratio above stag_ratio (Section 5; Z valid)   */
  CARE_INNER_FAILED = 7,      /* LR-ADI / Krylov made no progress                       */
  CARE_UNSTABLE = 8,          /* A_k not stable: no projected Ritz value with Re < 0,   */
                              /* or the LR-ADI residual grows by more than 1e12        */
  CARE_NONFINITE = 9,         /* NaN/Inf met in inputs or iterates                      */
  CARE_ERR_SMALL_DENSE = 10,  /* a small dense host factorisation failed                */
  CARE_TIMEOUT = 11           /* a bounded device wait (tensor-core pipeline) expired;  */
                              /* the kernel drained its copies and returned            */
} care_status;

typedef enum {
  CARE_PREC_FP64 = 0,       /* u_s = u = u_r = u_c = FP64: the all-FP64 path            */
  CARE_PREC_MIXED_FP32 = 1, /* u_s = FP32 (NLR-ADI and inner LR-ADI); u, u_r, u_c = FP64 */
  CARE_PREC_MIXED_TF32 = 2, /* as MIXED_FP32, and the Grams of the shift generation (the */
                            /* shift-basis orthonormalisation and the projected matrix)  */
                            /* on the tensor cores with TF32 inputs, FP32 accumulation   */
  CARE_PREC_MIXED_BF16 = 3  /* the same with BF16 inputs.  The paper names tensor cores  */
                            /* as future work (Section 6); only products whose use       */
                            /* tolerates their rounding (Ritz values for the shifts)     */
                            /* take them, the Krylov, ADI-norm and refinement arithmetic */
                            /* stays FP32 / FP64                                         */
} care_prec;

/* Method of the shifted solves.  Block Krylov (one Krylov space per right-hand-
 * side column): BiCGStab (default), or restarted GMRES with right
 * preconditioning, the method of the paper's GPU experiments (Section 5.2),
 * restart gmres_restart_lo / _hi for FP32 / FP64 solves.  Or dense direct:
 * M_p = (A + p I)^T formed densely and factored by LU with partial pivoting in
 * the solve's precision for every shift (the solvers of the stability study,
 * Section 5.1, and Section 4's dense-direct cost class); for n <=
 * CARE_DENSE_LU_MAX_N, with 2 n^2 values of the inner precision added to the
 * workspace. */
typedef enum { CARE_KRYLOV_BICGSTAB = 0, CARE_KRYLOV_GMRES = 1, CARE_KRYLOV_DENSE_LU = 2 } care_krylov;
#define CARE_DENSE_LU_MAX_N 8192
/* Preconditioner of the shifted solves (right preconditioning): Jacobi, ILU(0) by
 * three fixed-point sweeps with Jacobi-swept triangular solves (Chow & Patel; the
 * default, row-parallel), or ILU(0) computed exactly with exact triangular solves
 * (the paper's preconditioner, Section 5.2; sync-free row ordering with bounded
 * waits, sequential along the elimination's dependency chains). */
typedef enum {
  CARE_PRECOND_NONE = 0,
  CARE_PRECOND_JACOBI = 1,
  CARE_PRECOND_ILU0 = 2,
  CARE_PRECOND_ILU0_EXACT = 3
} care_precond;

/* A itself (not A^T) in CSR: int32 row pointers (n+1) and column indices (nnz),
 * FP64 values (nnz); device pointers; column indices need not be sorted. */
typedef struct {
  int n;
  int nnz;
  const int* rowptr;
  const int* colind;
  const double* val;
} care_csr;

/* Parameters.  care_opts_default() fills in the paper's values (Section 5:
 * eta_r = 1e-4 max|lambda(H)|, eta_s = 10 u max|lambda(P)|, tau_L = 1e-12 / 1e-5,
 * k_max = 20, j_max = 50; GMRES tolerances 1e-10 / 1e-5 and iteration limits
 * 200 / 100 of Section 5.2 reused for the block Krylov solver). */
typedef struct {
  int kmax;              /* refinement steps of Framework 1                          */
  int jmax;              /* LR-ADI shifts per Lyapunov solve                         */
  int newton_max;        /* NLR-ADI Newton steps                                     */
  int adi_cap;           /* column capacity of one LR-ADI factor (workspace sizing)  */
  double eta_r_rel;      /* Algorithm 1 truncation, relative to max|lambda(H)|       */
  double eta_s_mult;     /* Algorithm 2 truncation: eta_s = eta_s_mult*u*max|sigma|  */
  double tau_L_lo;       /* LR-ADI tolerance with FP32 inner solves                  */
  double tau_L_hi;       /* LR-ADI tolerance with FP64 inner solves                  */
  double tau_N_lo;       /* NLR-ADI Newton tolerance (relative change of K), FP32    */
  double tau_N_hi;       /* same, FP64                                               */
  double krylov_tol_lo;  /* per-column relative residual, FP32 shifted solves        */
  double krylov_tol_hi;  /* same, FP64                                               */
  int krylov_maxit_lo;   /* FP32 iteration limit                                     */
  int krylov_maxit_hi;   /* FP64 iteration limit                                     */
  int krylov;            /* care_krylov                                              */
  int precond;           /* care_precond                                             */
  int krylov_chunk;      /* max right-hand-side columns per Krylov call (<= 64)      */
  double stag_ratio;     /* refinement stops if ||R_{k+1}|| / ||R_k|| > stag_ratio   */
  int shift_hmin;        /* min. projection basis width for shift generation         */
  int ilu_sweeps;        /* ILU(0) fixed-point sweeps per shift (CARE_PRECOND_ILU0)  */
  int tri_sweeps;        /* Jacobi sweeps per triangular factor in the ILU(0) apply  */
  int verbose;           /* 0 silent, 1 per outer step, 2 per ADI step (stderr)      */
  int inner_compress;    /* FP32 inner solves only (default 2).  0: the +/- factors   */
                         /* go to Algorithm 2 as computed (jointly compressed only   */
                         /* when their capacity is reached); 1: also compress each   */
                         /* sign group at the end when wider than max(2b, 512) (a    */
                         /* u_s truncation relative to ||X_+-||, which can slow the  */
                         /* refinement); 2: compress X_+ - X_- jointly in FP64 at    */
                         /* the end, truncated at 1e-8 relative to the correction    */
                         /* itself.  FP64 inner factors are always compressed (at    */
                         /* FP64 accuracy).                                          */
  int gmres_restart_lo;  /* GMRES restart length, FP32 solves (Section 5.2: 30)      */
  int gmres_restart_hi;  /* GMRES restart length, FP64 solves (Section 5.2: 50)      */
} care_opts;

#define CARE_HIST_MAX 32

typedef struct {
  int status;             /* care_status of the call                                  */
  int rank;               /* columns of Z written                                     */
  int iter0_outer;        /* NLR-ADI Newton steps                                     */
  int iter0_inner;        /* total LR-ADI shifts in NLR-ADI                           */
  int iter_outer;         /* refinement steps (Algorithm 1 evaluations)               */
  int iter_inner;         /* total LR-ADI shifts in the correction solves             */
  long long krylov_iters; /* block Krylov iterations (all shifted solves)             */
  long long spmm_calls;   /* SpMM launches                                            */
  int krylov_unconverged; /* shifted solves that hit the iteration limit              */
  int nhist;              /* entries of res_hist                                      */
  double res_hist[CARE_HIST_MAX]; /* ||R(Z_k)||_F / ||C^T C||_F per refinement step  */
  double res_rel_CtC;     /* final ||R(Z Z^T)||_F / ||C^T C||_F (FP64, Algorithm 1)   */
  double res_paper;       /* final Res of Section 5                                   */
  double ms_phase[4];     /* wall ms: NLR-ADI, Algorithm 1, inner LR-ADI, Algorithm 2 */
  double ms_total;        /* wall ms of the call                                      */
  double gram_ms[2];      /* device ms (CUDA events on the call's stream) of the Gram */
                          /* products X^T Y, [0] FP64 and [1] FP32 inputs            */
  double gram_gflop[2];   /* their algorithmic GFLOP: 2 n a b, or n a (a+1) for X^T X */
  long long gram_calls[2];/* their number                                             */
  double gemm_ms[2];      /* the same for the tall-skinny products Y = alpha X S + beta */
  double gemm_gflop[2];   /* Y (n x a times a x b; 2 n a b GFLOP), [0] FP64, [1] FP32   */
  long long gemm_calls[2];/* inputs                                                     */
  double tc_ms[2];        /* device ms of the products run on the tensor cores with    */
  double tc_gflop[2];     /* BF16 slices ([0] FP64 operands, care_gram_tc mode 0; [1]  */
  long long tc_calls[2];  /* FP32 operands, mode 3), their algorithmic GFLOP (2 n a b, */
                          /* n a (a+1) for X^T X) and number; Grams and X S together   */
  double krylov_ms;       /* device ms of the block Krylov shifted solves (events)     */
  double krylov_gbyte;    /* their algorithmic HBM GB (per-iteration pass count)       */
  long long host_syncs;   /* stream synchronisations made by the host control          */
  long long lowp_gram_calls; /* TF32 / BF16 tensor-core Grams (MIXED_TF32 / _BF16)     */
} care_info;

/* Prepared operator: A^T in CSR (FP64 and FP32 values) plus its diagonal, laid
 * out inside caller memory by care_op_prepare.  Treat as read-only. */
typedef struct {
  int n, nnz;
  int* rowptr_t;    /* A^T row pointers (n+1)                                       */
  int* colind_t;    /* A^T column indices (nnz), sorted within rows                  */
  double* val64_t;  /* A^T values FP64                                               */
  float* val32_t;   /* A^T values rounded to FP32                                    */
  double* diag64;   /* diag(A)                                                       */
  float* diag32;
  float* rowsum32_t;  /* row sums of A^T (FP64 sums rounded to FP32): the FP32 operator is
                         applied in the difference form sum_j a_ij (x_j - x_i) + s_i x_i */
  int max_row_nnz;  /* longest row of A^T                                            */
  int diag_const;   /* 1 if all diagonal entries are equal (Jacobi is then a no-op)  */
  int full_diag;    /* 1 if every row stores its diagonal entry (required by ILU(0)) */
  double a_fro;     /* ||A||_F                                                       */
} care_op;

/* ---- parameters, status ------------------------------------------------- */

/* Fills *opts with the paper's parameter values (see care_opts). */
void care_opts_default(care_opts* opts);

/* Static string for a care_status value (never NULL). */
const char* care_status_string(int status);

/* Library build string (compiler, target architecture). */
const char* care_version(void);

/* ---- operator --------------------------------------------------------- */

/* Bytes of device memory care_op_prepare needs for an n x n matrix with nnz
 * entries. */
care_status care_op_size(int n, int nnz, size_t* bytes);

/* Builds the prepared operator of A inside mem (device, >= care_op_size bytes,
 * 256-byte aligned): transposes A on the device, sorts each row of A^T by column,
 * rounds the values to FP32, extracts the diagonal and ||A||_F.  Synchronises s.
 * The matrix M_p = (A + p I)^T of the shifted solves (Section 4, SMW formula)
 * is applied from this transpose with the shift p fused in the kernel, the
 * identity kept in the working precision (Section 5). */
care_status care_op_prepare(const care_csr* A, void* mem, size_t bytes, care_stream_t s, care_op* op);

/* ---- kernel-level entry points (row-major blocks) ----------------------- */

/* Y = (A^T + p I) X for an n x b block (Section 4: the operator M_p of the shifted
 * solves).  dtype 0 = FP64, 1 = FP32 (values of op->val64_t / val32_t).  cplx = 0:
 * X, Y real, row i at X + i*ldx, ldx >= b; cplx = 1: X, Y complex interleaved
 * (re, im) pairs, ldx >= 2b reals, p = p_re + i p_im.  Asynchronous on s. */
care_status care_spmm(const care_op* op, int dtype, int cplx, double p_re, double p_im,
                      const void* X, int ldx, int b, void* Y, int ldy, care_stream_t s);

/* G = X^T Y for row-major X (n x a, ldx) and Y (n x b, ldy), dtype as above,
 * accumulated per thread in the input precision and across threads in FP64;
 * G is FP64 row-major a x b (ldg >= b).  work: device scratch of
 * care_gram_work_size(n, a, b) bytes.  Asynchronous on s.  Used for the
 * tall-skinny products of Algorithms 1 and 2 and of LR-ADI (Section 4). */
size_t care_gram_work_size(int n, int a, int b);
care_status care_gram(int dtype, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy,
                      double* G, int ldg, void* work, size_t work_bytes, care_stream_t s);

/* Allocation-free variant of care_gram, for callers that cannot allocate device
 * memory at call time: for example a control loop with hard deadlines that
 * reserved all of its memory at start-up, or a plug-in whose host framework's
 * allocator owns the device memory.  The paper has no counterpart to this
 * entry point.  It computes the same G = X^T Y (same layouts, same precision
 * rules) without a workspace argument: its split-K scratch is a fixed
 * file-scope device array of CARE_GRAM_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB),
 * which every GPU that loads the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *  - a * b must not exceed CARE_GRAM_NOALLOC_SCRATCH_DOUBLES, else
 *    CARE_ERR_INVALID_ARG; long row ranges are handled with fewer, longer
 *    row slices, so results may differ from care_gram in the last bits.
 *  - The 8 MiB are reserved by the CUDA driver when it loads the library's
 *    device code on a device.  Under lazy module loading (the CUDA default)
 *    that happens on the first call into the library on that device, which
 *    also looks up the scratch's device address (cudaGetSymbolAddress).  So
 *    make one warm-up call (any shape) at start-up, with the device current,
 *    before the allocation-free phase and before any stream capture.
 *  - All calls share the one scratch array and it keeps the last call's
 *    contents; every entry a call reads is written by that call first.  Calls
 *    that overlap on the GPU (different streams, or different host threads
 *    without ordering) race on the scratch and give wrong results.
 *  - Asynchronous on s. */
#define CARE_GRAM_NOALLOC_SCRATCH_DOUBLES 1048576
care_status care_gram_noalloc(int dtype, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy,
                              double* G, int ldg, care_stream_t s);

/* Shifted block solve with feedback (Section 4, SMW formula):
 *   V = ((A - B K^T)^T + p I)^{-1} W,  i.e.  (A_k + p I)^{-T} W,  A_k = A - B K^T,
 * for an n x b block W; B, K FP64 column-major n x m (K may be NULL: no
 * feedback).  W: real FP64 column-major n x b.  V: FP64 column-major n x b,
 * real when p_im == 0 (entry (i, j) at V[i + j*ldv]) and complex otherwise,
 * stored as interleaved (re, im) pairs like complex128 (entry (i, j) at
 * V[2*(i + j*ldv)] and V[2*(i + j*ldv) + 1]); ldv >= n in entries.
 * prec selects the arithmetic of the Krylov solve.  iters (host, may be NULL)
 * receives the Krylov iteration count. */
care_status care_shifted_solve_workspace_size(const care_op* op, int m, int b, care_prec prec,
                                              const care_opts* opts, size_t* bytes);
care_status care_shifted_solve(const care_op* op, const double* B, int ldb, const double* K, int ldk,
                               int m, double p_re, double p_im, const double* W, int ldw, int b,
                               care_prec prec, const care_opts* opts, double* V, int ldv,
                               void* work, size_t work_bytes, care_stream_t s, int* iters);

/* Autotuner for the shifted solves (no paper counterpart), in two stages on the
 * operator at a mid-spectrum shift p = -0.05 max|a_ii|:
 *  1. SpMM launch shape: 16-byte vectors per thread in {1, 2, 4} (fewer threads
 *     per row, more gathers in flight per thread) x {4, 8} CTAs per SM for the
 *     row-block kernels, with grid-stride rows (contiguous row blocks per CTA,
 *     settable with care_set_launch_shape, lost on every operator measured),
 *     timed on a b-column block in the working precision (median of 5
 *     launches); then the vectors per thread for each other width class of the
 *     Krylov blocks (vectors per row <= 2, <= 4, <= 8, <= 16, more); the
 *     fastest are applied process-wide.
 *  2. Shifted solves (SMW + block Krylov) of a b-column and a 128-column
 *     right-hand side (deterministic pseudo-random entries; the wide one is where
 *     the chunking matters) with that shape over krylov in {BiCGStab, GMRES},
 *     precond in {ILU0 with tri_sweeps 2, 3, ILU0_EXACT, NONE} and krylov_chunk
 *     in {32, 64}; keeps the configuration with the smallest total time whose
 *     solves converged.
 * On return opts->krylov, precond, tri_sweeps and krylov_chunk hold the choice
 * and *best_ms (host, may be NULL) its total time.  The choice is kept for the life of
 * the process per (device, n, nnz, m, b, prec): a later call with the same key
 * applies it without timing (a serving process tunes each operator shape once).
 * work: device scratch of care_autotune_workspace_size bytes.  Synchronises s. */
care_status care_autotune_workspace_size(const care_op* op, int m, int b, care_prec prec, size_t* bytes);
care_status care_autotune(const care_op* op, int m, int b, care_prec prec, care_opts* opts, void* work,
                          size_t work_bytes, care_stream_t s, double* best_ms);
/* The process-wide launch shape (autotuner stage 1): SpMM vectors per thread
 * (1, 2 or 4), CTAs per SM (1..8) of the row-block kernels, SpMM row order
 * (0 grid-stride, 1 contiguous blocks per CTA).  get writes the vectors per
 * thread of the 5 width classes (spmm_vpt: host array of 5) and always
 * succeeds (returns 0); set applies one value to every width class and returns
 * CARE_ERR_INVALID_ARG for other values. */
int care_get_launch_shape(int* spmm_vpt, int* ctas_per_sm, int* spmm_blocked);
care_status care_set_launch_shape(int spmm_vpt, int ctas_per_sm, int spmm_blocked);

/* ---- solver entry points ------------------------------------------------ */

/* Workspace for care_solve / lyap_lradi / care_residual_factor on an n x n
 * operator with nnz entries, m inputs, p outputs (or RHS width b for
 * lyap_lradi), factor capacity r_cap, precision policy prec. */
care_status care_workspace_size(int n, int nnz, int m, int p, int r_cap, care_prec prec,
                                const care_opts* opts, size_t* bytes);

/* Framework 1 (Section 2) with the ADI realisation of Section 4:
 *   Z_1 <- NLR-ADI in u_s (FP32 for CARE_PREC_MIXED_FP32, FP64 otherwise);
 *   loop k = 1..k_max: Algorithm 1 in FP64 -> C+, C-, ||R(Z_k)||_F;
 *     stop if ||R||_F <= tol ||C^T C||_F (or stagnation, Section 5);
 *     LR-ADI in u_s on A_k^T X + X A_k + [C+,C-][C+,C-]^T-split = 0;
 *     Algorithm 2 in FP64 -> Z_{k+1}.
 * A: CSR of A (device).  B (n x m, ldb) and C (p x n, ldc): FP64 column-major,
 * device.  Z: output, FP64 column-major n x r_cap (ldz >= n), device; the
 * first info->rank columns hold the factor, X ~ Z Z^T.  Returns CARE_OK on
 * convergence; CARE_NOT_CONVERGED / CARE_STAGNATED still return a factor: the
 * last one, or the one before it if the last refinement step increased the
 * residual (info->res_rel_CtC is the residual of the returned factor).
 * Synchronises s.  info (host) may be NULL. */
care_status care_solve(const care_csr* A, const double* B, int ldb, int m, const double* C, int ldc,
                       int p, double tol, care_prec prec, const care_opts* opts, double* Z, int ldz,
                       int r_cap, void* work, size_t work_bytes, care_stream_t s, care_info* info);

/* Batched Framework 1 for `count` independent CAREs of uneven sizes (no paper
 * counterpart; the paper solves one CARE at a time).  Instance i has A[i], B[i]
 * (n_i x m[i], ldb[i]), C[i] (p[i] x n_i, ldc[i]) and output Z[i] (n_i x r_cap[i],
 * ldz[i]), all as for care_solve; tol, prec, opts are shared.  Instances are
 * ordered by estimated cost n_i (m_i + p_i) (largest first) and taken from a
 * shared queue by `workers` host threads, each with its own CUDA stream and its
 * own slice of `work`, so that instances overlap on the GPU.  Each instance is
 * solved exactly as care_solve would (same kernels, same order of operations):
 * results are bitwise identical to individual calls.  The caller's stream s
 * waits for all workers before the call returns.  info (host, may be NULL) is
 * an array of count entries.  Returns CARE_OK if every instance converged,
 * otherwise the first non-OK status in instance order (all entries of info are
 * filled either way). */
care_status care_workspace_size_batched(int count, const care_csr* const* A, const int* m, const int* p,
                                        const int* r_cap, care_prec prec, const care_opts* opts, int workers,
                                        size_t* bytes);
care_status care_solve_batched(int count, const care_csr* const* A, const double* const* B, const int* ldb,
                               const int* m, const double* const* C, const int* ldc, const int* p, double tol,
                               care_prec prec, const care_opts* opts, double* const* Z, const int* ldz,
                               const int* r_cap, int workers, void* work, size_t work_bytes, care_stream_t s,
                               care_info* info);

/* Batched Framework 1, serving mode (no paper counterpart): `count` <= 256
 * independent CAREs, each on its own host thread and CUDA stream with its own
 * workspace slice, as care_solve_batched, except that the shifted solves of all
 * instances (Section 4's dominant work) are gathered: when every instance still
 * solving has a shifted solve pending (or after 2 ms), ONE persistent
 * cooperative launch runs block BiCGStab (right Jacobi preconditioning) on all
 * of them over a work list of row tiles of every instance, with per-column
 * convergence and early exit.  opts->krylov and opts->precond are replaced by
 * BiCGStab + Jacobi, and the Krylov iteration limits are raised to at least
 * 400 (FP32) / 800 (FP64), four times the paper's, since Jacobi is the weaker
 * preconditioner.  Results agree with
 * care_solve to the solver tolerances, not bitwise (a different preconditioner
 * and summation order).  batch_launches (host, may be NULL) receives the
 * number of batched launches.  Other arguments as for care_solve_batched. */
care_status care_workspace_size_batched_persistent(int count, const care_csr* const* A, const int* m, const int* p,
                                                   const int* r_cap, care_prec prec, const care_opts* opts,
                                                   size_t* bytes);
care_status care_solve_batched_persistent(int count, const care_csr* const* A, const double* const* B,
                                          const int* ldb, const int* m, const double* const* C, const int* ldc,
                                          const int* p, double tol, care_prec prec, const care_opts* opts,
                                          double* const* Z, const int* ldz, const int* r_cap, void* work,
                                          size_t work_bytes, care_stream_t s, care_info* info,
                                          long long* batch_launches);

/* LR-ADI (Section 4) for  (A - B K^T)^T X + X (A - B K^T) + W W^T = 0,  X ~ Z Z^T.
 * B, K: FP64 column-major n x m (both NULL or m = 0: no feedback).  W: FP64
 * column-major n x b.  Runs in the inner precision of prec with tolerance tol on
 * ||W_j^T W_j||_2 / ||W_0^T W_0||_2.  Z: FP64 column-major output, capacity
 * r_cap columns; info->rank = columns written, info->iter_inner = shifts used.
 * Requires A - B K^T stable. */
care_status lyap_lradi(const care_csr* A, const double* B, int ldb, const double* K, int ldk, int m,
                       const double* W, int ldw, int b, double tol, care_prec prec,
                       const care_opts* opts, double* Z, int ldz, int r_cap, void* work,
                       size_t work_bytes, care_stream_t s, care_info* info);

/* Algorithm 1 (Section 2) in FP64: factors R(Z Z^T) = C+ C+^T - C- C-^T with
 * eigenvalues of H kept when lambda >= eta_r or lambda <= -eta_r,
 * eta_r = eta_r_rel * max|lambda(H)|.  Z: FP64 column-major n x r.  Cp, Cm: FP64
 * column-major outputs with capacity c_cap columns each; *rp, *rm (host) receive
 * their widths; *res_fro (host) receives ||R(Z Z^T)||_F = ||H||_F before
 * truncation.  Cp/Cm may be NULL to get the norm only. */
care_status care_residual_factor(const care_csr* A, const double* B, int ldb, int m, const double* C,
                                 int ldc, int p, const double* Z, int ldz, int r, double eta_r_rel,
                                 double* Cp, int ldcp, int* rp, double* Cm, int ldcm, int* rm,
                                 int c_cap, double* res_fro, void* work, size_t work_bytes,
                                 care_stream_t s);

/* Number of kernels this library has launched in the process so far (all
 * entry points, all streams); for launch accounting in benchmarks. */
unsigned long long care_kernel_launches(void);

/* The ILU(0) factor of M_p = (A + p I)^T on the pattern of A^T (the shifted
 * solves' preconditioner, Section 5.2): exact = 1 computes it exactly (IKJ
 * elimination on the pattern), exact = 0 by the three fixed-point sweeps the
 * default preconditioner uses.  F (device): nnz values of dtype (0 FP64, 1 FP32)
 * in the order of op's A^T rows, complex interleaved (2 nnz) when p_im != 0;
 * the strictly lower entries hold L (unit diagonal implied), the others U.
 * Requires every diagonal entry stored (op->full_diag).  work:
 * care_ilu0_work_size bytes.  Synchronises s. */
size_t care_ilu0_work_size(const care_op* op, int dtype);
care_status care_ilu0(const care_op* op, int dtype, int exact, double p_re, double p_im, void* F, void* work,
                      size_t work_bytes, care_stream_t s);

/* Symmetric eigendecomposition on the device, the one Algorithms 1-2 use for
 * H = T M T^T and P = Gamma N Gamma^T (FP64): Householder tridiagonalisation,
 * bisection for every eigenvalue, inverse iteration for the eigenvectors of the
 * eigenvalues w <= lo or w >= hi (the ones the truncation at eta_r / eta_s keeps),
 * back-transformation.  A: device, n x n row-major (lda), symmetric (only
 * (A + A^T)/2 is used; A is not modified).  w (host, n): all eigenvalues,
 * ascending.  V (device, may be NULL: eigenvalues only): the selected
 * eigenvectors as rows of length n, in ascending eigenvalue order; *nsel (host)
 * their number (V needs nsel x n doubles, at most n x n).  work:
 * care_symeig_work_size(n) bytes.  Synchronises s. */
size_t care_symeig_work_size(int n);
care_status care_symeig(int n, const double* A, int lda, double* w, double* V, double lo, double hi, int* nsel,
                        void* work, size_t work_bytes, care_stream_t s);

/* Measured FP64 FMA throughput of the CUDA cores in TFLOP/s (8 independent
 * dependent-FMA chains per thread over 8 CTAs per SM; best of 3 timed runs with
 * CUDA events on s): the denominator of the FP64 product rooflines. */
care_status care_fp64_peak(double* tflops, care_stream_t s);

/* ---- tensor-core products (tcgen05 + TMA, sm_103a) ---------------------- */
/* The dense n x r by r x r contractions of Algorithms 1-2 and of LR-ADI
 * (Section 4 complexity, O(n q^2)) on the tensor cores.  mode 0 is
 * FP64-accurate: every row of X^T and Y^T (column of X, Y) is scaled by a power
 * of two, rounded to a 56-bit fixed-point integer relative to its largest entry
 * and split exactly into eight 7-bit BF16 slices; the 43 slice products with
 * a + b <= 8 run on the BF16 tensor pipe with exact integer chunk sums (the
 * splitting idea of Ozaki et al. 2012).  mode 3 is the FP32-accurate
 * counterpart for FP32 operands (28-bit fixed point, four slices, the 10 pairs
 * with a + b <= 3, all summed exactly): the FP32 products of the inner solves.
 * mode 1 = TF32 inputs, mode 2 = BF16 inputs, both with FP32 accumulation (the
 * low-precision Grams of the CARE_PREC_MIXED_TF32 / _BF16 shift generation). */
int care_tc_available(void);        /* 1 on an sm_103 device with the driver's TMA encoder */
/* Solver use of the mode-0 products: 0 off (FP64 FMA on the CUDA cores), 1 where
 * profitable (default: contraction >= 1024, both output sizes >= 48, >= 2 GFLOP),
 * 2 every FP64 product of the solver (for tests).  Process-wide. */
void care_set_tensor_cores(int on);

/* Test hook for the failure path: while on, the tensor-core kernels issue no
 * operand copies, so their first bounded wait (2 s) expires; they record the
 * error, release their tensor memory and return, and the entry point reports
 * CARE_TIMEOUT with the context intact.  Process-wide; off by default. */
void care_tc_test_starve(int on);

/* Device scratch for care_gram_tc / care_gemm_ts (tc = 1) with a + b <= maxdim. */
size_t care_tc_work_size(int maxdim);

/* G = X^T Y on the tensor cores; X (n x a, ldx), Y (n x b, ldy) row-major, FP64
 * for mode 0 and FP32 for modes 1-3; G FP64 row-major a x b (ldg).  X == Y with
 * the same ld computes the upper tiles only and mirrors them (exactly
 * symmetric).  work: care_tc_work_size(a + b) bytes.  Synchronises s (reads
 * the kernels' error word): CARE_TIMEOUT if a bounded wait expired. */
care_status care_gram_tc(int mode, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy, double* G,
                         int ldg, void* work, size_t work_bytes, care_stream_t s);

/* Y = alpha X S + beta Y, X (n x a, ldx) and Y (n x b, ldy) row-major, S (a x b,
 * lds) row-major FP64 on the device; dtype 0 FP64 X, Y; 1 FP32 X, Y.  tc = 1:
 * tensor-core slices, FP64-accurate (dtype 0) or FP32-accurate (dtype 1) (work:
 * care_tc_work_size(a + b) bytes; synchronises s); tc = 0: FP64/FP32 FMA on the
 * CUDA cores (work unused, asynchronous).  The tall-skinny product of
 * Algorithms 1-2 (C+- and Z_{k+1} formation) and of the CGS2 projections. */
care_status care_gemm_ts(int dtype, int tc, int n, int a, int b, double alpha, const void* X, int ldx, const double* S,
                         int lds, double beta, void* Y, int ldy, void* work, size_t work_bytes, care_stream_t s);

/* ---- small dense host routines (exported for host-only tests) ----------- */

/* Symmetric eigendecomposition of the column-major n x n matrix A (host):
 * eigenvalues ascending in w, orthonormal eigenvectors in V (column-major,
 * may be NULL).  Householder tridiagonalisation + implicit QR with Wilkinson
 * shifts.  Returns CARE_OK or CARE_ERR_SMALL_DENSE. */
care_status care_host_symeig(int n, const double* A, double* w, double* V);

/* The same, with eigenvectors only for the eigenvalues w <= lo or w >= hi (the
 * other columns of V are set to zero); all eigenvalues are returned.  This is
 * the form Algorithms 1-2 use, which keep the eigenpairs beyond their
 * truncation thresholds (eta_r, eta_s).  V must not be NULL. */
care_status care_host_symeig_outside(int n, const double* A, double* w, double* V, double lo, double hi);

/* Upper Cholesky factor of the SPD column-major n x n matrix G = R^T R (R
 * column-major, lower part zero).  CARE_ERR_SMALL_DENSE if G is not SPD. */
care_status care_host_cholesky_upper(int n, const double* G, double* R);

/* Rank-revealing Cholesky with complete (diagonal) pivoting of the positive
 * semidefinite row-major c x c matrix G: stops when the largest remaining
 * pivot is <= tol or after max_rank (> 0) pivots.  Writes the rank to *rank,
 * the pivot order to piv[0 .. rank) and R (rank x c, row-major, original
 * column order, rows beyond the rank zero; R must hold c x c) with
 * G ~= R^T R.  The orthonormalisations of Algorithms 1-2 are built on it. */
care_status care_host_pivoted_cholesky(int c, const double* G, double tol, int max_rank, int* piv, double* R,
                                       int* rank);

/* Largest eigenvalue of the symmetric n x n matrix G (host), as LR-ADI's
 * stopping test ||W^T W||_2 needs it: Lanczos with full reorthogonalisation to a
 * relative residual bound of 1e-13, or the full eigenvalue computation for
 * n <= 96 or without convergence in 120 steps. */
care_status care_host_sym_lmax(int n, const double* G, double* lmax);

/* Inverse of the upper triangular row-major r x r matrix U (Ui row-major). */
care_status care_host_upper_inverse(int r, const double* U, double* Ui);

/* C = A diag(d) B^T for row-major A (m x k, lda), B (n x k, ldb), C (m x n,
 * ldc); d may be NULL (identity).  sym != 0: B is A, m == n, and C is formed
 * from its upper part and mirrored (exactly symmetric). */
care_status care_host_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                              const double* d, double* C, int ldc, int sym);

/* Eigenvalues of a real column-major n x n matrix (host): Hessenberg reduction
 * and Francis double-shift QR; real parts in wr, imaginary parts in wi. */
care_status care_host_eigvals(int n, const double* A, double* wr, double* wi);

#ifdef __cplusplus
}
#endif
#endif /* CARE_B300_H */
