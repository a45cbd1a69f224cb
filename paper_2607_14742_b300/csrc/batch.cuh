// Batched shifted solves over many CARE instances (k_batch.cu): one persistent
// cooperative launch of block BiCGStab over a work list of row tiles of every
// pending request, and the broker that gathers the requests of the instance
// threads of care_solve_batched_persistent.
#pragma once

#include "krylov.cuh"

namespace care {

constexpr int kBatchMaxReq = 256;  // requests per launch

// Per-column (complex: per column pair) recurrence scalars of the batched solve.
struct BatchSlot {
  double rho_re, rho_im, alpha_re, alpha_im, omega_re, omega_im, beta_re, beta_im;
  double bnorm2, rnorm2;
  int flag;  // 0 active, 1 converged, 2 breakdown, 3 iteration limit
  int iters;
};

// One shifted solve M_p X = RHS, M_p = (A + p I)^T (the prepared A^T), on `cols`
// real columns (complex interleaved pairs when cplx).  The caller fills the
// operator, the shift, rhs / sol (row-major, leading dimensions in reals), the
// Krylov blocks (n x kMaxRealCols each, from the instance's KrylovWork), Dinv
// (2 n values, or null: no preconditioning), tol2 = tol^2 and maxit; the launch
// fills the layout fields.
template <class T>
struct BatchReq {
  long n = 0;
  int cols = 0, cplx = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const T* av = nullptr;
  const T* rs = nullptr;    // row sums (difference form of the FP32 operator) or null
  const T* diag = nullptr;  // a_ii
  double sre = 0.0, sim = 0.0;
  const T* rhs = nullptr;
  int ld_rhs = 0;
  T* sol = nullptr;
  int ld_sol = 0;
  T *X = nullptr, *R = nullptr, *Rh = nullptr, *P = nullptr, *V = nullptr, *S = nullptr, *Tt = nullptr;
  T *Ph = nullptr, *Sh = nullptr, *Dinv = nullptr;
  double tol2 = 0.0;
  int maxit = 0;
  // layout (set by batch_launch)
  int ld = 0, nvec = 0, nv2 = 0, rpt = 0, tile0 = 0, ntiles = 0, slot0 = 0;
  size_t pbase = 0;
};

template <class T>
struct BatchArgs {
  const BatchReq<T>* req;
  int nreq, ntiles;
  BatchSlot* slots;
  int nslot;
  double* partial;
  int* active;
  int* iters;
  int* ractive;       // active columns per request (last reduction)
  int* ractive_next;  // the same, being counted
  int maxit;
};

// Device scratch of one launch with at most max_req requests.
size_t batch_scratch_bytes(int max_req);
// One persistent launch over `reqs` on s (synchronises s); returns the iterations
// run and, if slots_out, the final per-column scalars (index reqs[k].slot0 + j).
template <class T>
int batch_launch(std::vector<BatchReq<T>>& reqs, char* scratch, size_t scratch_bytes, cudaStream_t s,
                 std::vector<BatchSlot>* slots_out);

// Gathers the shifted solves of `instances` host threads into batched launches: a
// request waits until every instance still solving has one pending (or a short
// time has passed), then one thread launches them all and the others wait.
class BatchBroker {
 public:
  BatchBroker(int instances, int elem_bytes, char* scratch, size_t scratch_bytes);
  ~BatchBroker();
  BatchBroker(const BatchBroker&) = delete;
  BatchBroker& operator=(const BatchBroker&) = delete;
  // Solve q (its inputs produced on `caller`); blocks until the batch containing
  // it has run.  iters = the request's largest column iteration count.
  template <class T>
  KrylovResult solve(BatchReq<T> q, cudaStream_t caller);
  // An instance has finished (it posts no more requests).
  void instance_done();
  long long launches() const;
  long long requests() const;

 private:
  struct Impl;
  Impl* p;
};

}  // namespace care
