// Host orchestration of the CARE solver: context, buffers, and the algorithm
// steps (SMW shifted solve, projection shifts, LR-ADI, NLR-ADI, Algorithms 1-2).
#pragma once

#include <chrono>
#include <vector>

#include "batch.cuh"
#include "dense.cuh"
#include "krylov.cuh"
#include "tc.cuh"

namespace care {

struct Ctx {
  cudaStream_t s = nullptr;
  care_opts o{};
  Arena ar;
  care_op op{};
  long op_nnz = 0;  // entries of A (sizes the ILU(0) factors before the operator exists)
  double* dS = nullptr;  // staging for small matrices (device)
  size_t dS_cap = 0;
  double* dG = nullptr;  // Gram results (device)
  size_t dG_cap = 0;
  double* gw = nullptr;  // Gram split-K scratch
  size_t gw_cap = 0;
  double* dsm = nullptr;  // device scratch of the small dense algebra (Algorithms 1-2)
  size_t dsm_cap = 0;
  long long krylov_iters = 0, spmm_calls = 0;
  double ms_gram = 0.0, ms_host = 0.0;  // Gram kernels (synchronised) and host small-dense time
  // device time (CUDA events on s) and algorithmic GFLOP of the Gram products,
  // [0] FP64 inputs, [1] FP32 inputs
  double gram_ms[2] = {0.0, 0.0}, gram_gflop[2] = {0.0, 0.0};
  long long gram_calls[2] = {0, 0};
  cudaEvent_t ge0 = nullptr, ge1 = nullptr;
  // the same for the tall-skinny products X S (gemm_c): their event pairs are queued
  // and read at the next point where the stream has been synchronised (harvest_timings)
  double gemm_ms[2] = {0.0, 0.0}, gemm_gflop[2] = {0.0, 0.0};
  long long gemm_calls[2] = {0, 0};
  struct PendingTiming {
    cudaEvent_t e0, e1;
    double gflop;
    int k;
  };
  std::vector<PendingTiming> tpend;
  std::vector<cudaEvent_t> tpool;
  int krylov_unconverged = 0;
  // tensor-core products: scratch, the operand-width limit it was sized for, and
  // whether a product ran since the last check of its error word
  TcScratch tc;
  int tc_maxdim = 0;
  bool tc_used = false;
  int lowp = 0;  // low-precision tensor-core Grams of the shift generation: 0 off, 1 TF32, 2 BF16
  long long lowp_calls = 0;
  // device time and algorithmic GFLOP of the sliced tensor-core products, [0] FP64
  // operands (8 slices), [1] FP32 operands (4 slices)
  double tc_ms[2] = {0.0, 0.0}, tc_gflop[2] = {0.0, 0.0};
  long long tc_calls[2] = {0, 0};
  // device time (CUDA events around each block Krylov solve) and its algorithmic bytes
  double kry_ms = 0.0, kry_gbyte = 0.0;
  cudaEvent_t ke0 = nullptr, ke1 = nullptr;
  long long host_syncs = 0;  // stream synchronisations of the host control
  // batched serving mode: the shifted solves go to this broker (one persistent
  // launch over the pending solves of all instances) instead of the block Krylov
  BatchBroker* broker = nullptr;
  bool counting() const { return ar.counting(); }
  Ctx() = default;
  Ctx(const Ctx&) = delete;
  Ctx& operator=(const Ctx&) = delete;
  ~Ctx() {
    if (ge0) cudaEventDestroy(ge0);
    if (ge1) cudaEventDestroy(ge1);
    if (ke0) cudaEventDestroy(ke0);
    if (ke1) cudaEventDestroy(ke1);
    for (const PendingTiming& t : tpend) {
      cudaEventDestroy(t.e0);
      cudaEventDestroy(t.e1);
    }
    for (cudaEvent_t e : tpool) cudaEventDestroy(e);
  }
};

// Reads the queued product timings; every queued event has been recorded on c.s
// before the synchronisation that precedes this call, so nothing waits here in
// practice (cudaEventSynchronize returns at once).
inline void harvest_timings(Ctx& c) {
  for (const Ctx::PendingTiming& t : c.tpend) {
    CARE_CUDA(cudaEventSynchronize(t.e1));
    float ms = 0.f;
    CARE_CUDA(cudaEventElapsedTime(&ms, t.e0, t.e1));
    if (t.k >= 2) {
      c.tc_ms[t.k - 2] += ms;
      c.tc_gflop[t.k - 2] += t.gflop;
      c.tc_calls[t.k - 2] += 1;
    } else {
      c.gemm_ms[t.k] += ms;
      c.gemm_gflop[t.k] += t.gflop;
      c.gemm_calls[t.k] += 1;
    }
    c.tpool.push_back(t.e0);
    c.tpool.push_back(t.e1);
  }
  c.tpend.clear();
  if (c.tc_used) {
    c.tc_used = false;
    const int e = tc_check(c.tc, c.s);
    CARE_REQUIRE(e == 0, CARE_TIMEOUT, "tensor-core product: a bounded wait expired");
  }
}

inline cudaEvent_t timing_event(Ctx& c) {
  if (!c.tpool.empty()) {
    cudaEvent_t e = c.tpool.back();
    c.tpool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  CARE_CUDA(cudaEventCreate(&e));
  return e;
}

// Whether an FP64 product of this shape (contraction k, output a x b, operand widths
// adding up to dims) runs on the tensor cores (FP64-accurate slices).
inline bool tc_use(const Ctx& c, long k, int a, int b, int dims) {
  return c.tc.ok() && dims <= c.tc_maxdim && tc_f64_profitable(k, a, b) && tc_available();
}

// gemm_ts on c.s (Y = alpha X S + beta Y), timed with CUDA events on the same stream;
// [0] FP64 / [1] FP32 inputs on the CUDA cores, [2] FP64 / [3] FP32 inputs on the
// tensor cores (sliced); algorithmic GFLOP 2 n a b
template <class Ti, class To>
inline void gemm_c(Ctx& c, long n, int a, int b, double alpha, const Ti* X, int ldx, const double* S, int lds,
                   double beta, To* Y, int ldy) {
  if (n <= 0 || a <= 0 || b <= 0) {
    gemm_ts<Ti, To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, c.s);
    return;
  }
  if (c.tpend.size() >= 512) harvest_timings(c);  // bounds the queue (waits for the oldest)
  cudaEvent_t e0 = timing_event(c), e1 = timing_event(c);
  CARE_CUDA(cudaEventRecord(e0, c.s));
  int k = sizeof(Ti) == 8 ? 0 : 1;
  if (tc_use(c, n, a, b, a + b)) {
    if constexpr (sizeof(Ti) == 8)
      tc_gemm_ts_f64<To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, c.tc, c.tc_maxdim, c.s);
    else
      tc_gemm_ts_f32acc<To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, c.tc, c.tc_maxdim, c.s);
    c.tc_used = true;
    k = sizeof(Ti) == 8 ? 2 : 3;
  } else {
    gemm_ts<Ti, To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, c.s);
  }
  CARE_CUDA(cudaEventRecord(e1, c.s));
  c.tpend.push_back({e0, e1, 2.0 * (double)n * a * b * 1e-9, k});
}

// host <-> device helpers for small matrices
const double* upload(Ctx& c, const std::vector<double>& h);
// lowp: the Gram may run on the tensor cores in TF32 / BF16 (Ctx::lowp) -- only for
// products whose use tolerates ~1e-3 relative error (shift generation)
template <class T>
std::vector<double> gram_h(Ctx& c, long n, int a, int b, const T* X, int ldx, const T* Y, int ldy,
                           bool lowp = false);

// Rank-revealing orthonormalisation X (n x cols) -> Q (in place, n x rank) with
// X = Q T (T rank x cols, row-major).  Column-scaled eigendecomposition of the
// Gram matrix (SVQB, Stathopoulos & Wu 2002) keeps directions with scaled
// eigenvalue > drop_rel * max; an optional second pass (Cholesky QR of the
// result) restores orthogonality to working accuracy.  colfloor2 (optional,
// host) gives per-column squared norms below which a column counts as zero.
struct OrthOut {
  int rank = 0;
  std::vector<double> T;     // rank x cols
  std::vector<double> Rinv;  // non-empty: the basis is buf * Rinv (rank x rank, row-major), see defer_rinv
};
// With `out` (one pass only) the basis is written there and X is left intact.
// defer_rinv (second pass only): the last product of the Cholesky QR, basis =
// Y1 R^{-1}, is not formed; Y1 is left in buf and R^{-1} returned in Rinv, for
// callers that only multiply the basis by a small matrix S (they form
// Y1 (R^{-1} S) instead, saving an n x rank x rank product).  If the second
// Cholesky fails, the basis is formed in X as without the flag and Rinv is empty.
template <class T>
OrthOut orth_rr(Ctx& c, long n, int cols, T* X, int ldx, T* buf, int ldb, double drop_rel,
                const std::vector<double>* colfloor2, bool second_pass, int max_rank, T* out, int ldo,
                bool defer_rinv = false, bool lowp_gram = false);

// X (n x cols) -= Q (Q^T X) twice (classical Gram-Schmidt with
// reorthogonalisation); returns the r x cols coefficients.
template <class T>
std::vector<double> cgs2(Ctx& c, long n, const T* Q, int ldq, int r, T* X, int ldx, int cols);

// Inner (u_s precision) solver state: block Krylov work, SMW, LR-ADI, NLR-ADI.
template <class T>
struct Inner {
  int n = 0, m = 0, bcap = 0, adicap = 0, hcap = 0;
  KrylovWork<T> kw;
  DluWork<T> dw;  // dense-direct shifted solves (CARE_KRYLOV_DENSE_LU)
  T *B = nullptr, *K = nullptr, *Knew = nullptr, *Kd = nullptr;  // n x m (ldm)
  T *W = nullptr, *W0 = nullptr;                                 // n x bcap (ldw)
  T *RHS = nullptr, *SOL = nullptr;                              // n x 2(bcap+m) (ldr)
  T *Z = nullptr;   // n x adicap (ldz): X_+ factor from the left, X_- factor from the right
  T *Zs = nullptr;  // n x adicap scratch (compression)
  T *Q = nullptr, *FQ = nullptr, *Qt = nullptr;                  // n x hcap (ldq)
  int ldm = 0, ldw = 0, ldr = 0, ldz = 0, ldq = 0;
  bool jacobi = false;
  // optional FP64 blocks (n x f64cap, ld f64ld) for the joint compression of the
  // +/- factors when their capacity is reached (set by sessions that have them)
  double *f64a = nullptr, *f64b = nullptr;
  int f64ld = 0, f64cap = 0;
  void alloc(Ctx& c, int n_, int m_, int bcap_, int adicap_, int hcap_);
};

struct AdiResult {
  int np = 0, nm = 0;  // factor columns: X_+ in Z[:, 0:np], X_- in Z[:, adicap-nm : adicap]
  int steps = 0;       // shifts used (a complex pair counts 2)
  int compressions = 0;
  bool converged = false;
  double res = 0.0;    // final ||W^T W||_2 / ||W_0^T W_0||_2
};

// LR-ADI for F X + X F^T + W0 W0^T = 0, F = A^T - K B^T (hasK), on the first
// b columns of in.W0; the first rp columns belong to X_+, the rest to X_-
// (the two correction equations of Framework 1 solved as one block).  If
// knew, accumulates K_new += Z_blk (Z_blk^T B) into in.Knew (requires rp = b).
// When the factor reaches its capacity it is column-compressed; if that does
// not free enough room the solve stops early (inexact inner solve).
// compress_end: 0 none; 1 column-compress each factor group at the end (inner-
// precision truncation) before Algorithm 2; 2 compress X_+ - X_- jointly in FP64.
template <class T>
AdiResult lradi(Ctx& c, Inner<T>& in, int b, int rp, bool hasK, double tol, int jmax, bool knew,
                int compress_end = 0);

struct NlrResult {
  int newton = 0, adi = 0, cols = 0;
  bool converged = false;
};
// NLR-ADI: Newton-Kleinman with LR-ADI inner solves; C^T (n x p, row-major T,
// ldw) must be in in.W0's first p columns on entry (it is re-read each step).
template <class T>
NlrResult nlradi(Ctx& c, Inner<T>& in, const T* Ct, int ldct, int p, double tol_lyap, double tol_newton,
                 int newton_max, int jmax);

template <class T>
OpT<T> op_of(const Ctx& c);

// One SMW shifted block solve (V in the leading columns of in.SOL) for the
// first b columns of in.W, with or without the feedback term.
template <class T>
void smw_solve_public(Ctx& c, Inner<T>& in, double p_re, double p_im, int b, bool hasK);

double now_ms();

// ---- device small dense algebra (Algorithms 1-2, factor compression) -------------
// A bump allocator over the context's device scratch for the small matrices (the
// products H = T M T^T and P = Gamma N Gamma^T, their eigendecompositions and the
// coefficient blocks); a fresh one per algorithm step.
struct DevSmall {
  double* base = nullptr;
  size_t cap = 0, off = 0;
  double* get(size_t n) {
    n = (n + 31) / 32 * 32;
    CARE_REQUIRE(off + n <= cap, CARE_ERR_WORKSPACE, "small dense device scratch too small");
    double* p = base + off;
    off += n;
    return p;
  }
};
double* to_dev(Ctx& c, DevSmall& ds, const std::vector<double>& h);
// symmetric M = L R^T (rt x rt) of the row-major factors L (rt x k) and Rt = R^T
// (k x rt), on the device (tensor cores where profitable)
double* dev_small_product(Ctx& c, DevSmall& ds, int rt, int k, const std::vector<double>& L,
                          const std::vector<double>& Rt);
// S[i][col] = V[q[col]][i] * sc[col] (i < rows): eigenvectors (rows of V, ldv)
// gathered and scaled into the columns of the row-major block S (ld = cols)
void eig_coeffs(Ctx& c, DevSmall& ds, int rows, int cols, const double* V, int ldv, const std::vector<int>& q,
                const std::vector<double>& sc, double* S);

}  // namespace care
