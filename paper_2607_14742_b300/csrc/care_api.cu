// Algorithms 1 and 2, Framework 1, operator preparation, and the C ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <atomic>
#include <functional>
#include <string>
#include <mutex>
#include <thread>

#include <omp.h>

#include "solver.cuh"

#define CARE_STR2(x) #x
#define CARE_STR(x) CARE_STR2(x)

namespace care {

constexpr double kU64 = 1.1102230246251565e-16;  // FP64 unit roundoff (Section 1 table)
unsigned long long launches();

// ---------------------------------------------------------- operator ------
static size_t op_bytes(int n, int nnz) {
  Arena a;
  a.get<int>((size_t)n + 1);   // rowptr_t
  a.get<int>((size_t)nnz);     // colind_t
  a.get<double>((size_t)nnz);  // val64_t
  a.get<float>((size_t)nnz);   // val32_t
  a.get<double>((size_t)n);    // diag64
  a.get<float>((size_t)n);     // diag32
  a.get<float>((size_t)n);     // rowsum32_t
  a.get<int>((size_t)n + 1);   // cursor / counts
  a.get<double>(4);            // reductions
  return a.off;
}

__global__ void k_count_cols(int n, const int* rp, const int* ci, int* cnt) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k) atomicAdd(&cnt[ci[k]], 1);
}

// exclusive scan of cnt[0..n) into rp[0..n] (single CTA, 1024 threads)
__global__ void k_scan(int n, const int* cnt, int* rp) {
  __shared__ long part[1024];
  const int t = threadIdx.x;
  const long chunk = ((long)n + 1023) / 1024;
  const long b = t * chunk, e = std::min<long>((long)n, b + chunk);
  long s = 0;
  for (long i = b; i < e; ++i) s += cnt[i];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    long acc = 0;
    for (int i = 0; i < 1024; ++i) {
      const long v = part[i];
      part[i] = acc;
      acc += v;
    }
  }
  __syncthreads();
  long acc = part[t];
  for (long i = b; i < e; ++i) {
    rp[i] = (int)acc;
    acc += cnt[i];
  }
  if (e == n && b < e) rp[n] = (int)acc;
  if (n == 0 && t == 0) rp[0] = 0;
}

__global__ void k_scatter(int n, const int* rp, const int* ci, const double* v, const int* rpt, int* cursor,
                          int* cit, double* vt) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      const int j = ci[k];
      const int pos = rpt[j] + atomicAdd(&cursor[j], 1);
      cit[pos] = (int)i;
      vt[pos] = v[k];
    }
}

// sort each row of A^T by column (insertion sort; rows are short), merge
// duplicate-free; cast values; extract the diagonal
__global__ void k_finish_rows(int n, const int* rpt, int* cit, double* vt, float* vt32, double* d64,
                              float* d32, float* rs32, double* missing, int* maxrow) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int b = rpt[i], e = rpt[i + 1];
    for (int k = b + 1; k < e; ++k) {
      const int c = cit[k];
      const double v = vt[k];
      int q = k - 1;
      while (q >= b && cit[q] > c) {
        cit[q + 1] = cit[q];
        vt[q + 1] = vt[q];
        --q;
      }
      cit[q + 1] = c;
      vt[q + 1] = v;
    }
    double dg = 0.0, rs = 0.0;
    bool has = false;
    for (int k = b; k < e; ++k) {
      vt32[k] = (float)vt[k];
      rs += vt[k];
      if (cit[k] == i) {
        dg += vt[k];
        has = true;
      }
    }
    if (!has) atomicAdd(missing, 1.0);
    atomicMax(maxrow, e - b);
    rs32[i] = (float)rs;
    d64[i] = dg;
    d32[i] = (float)dg;
  }
}

// red[0] = sum v^2, red[1] = min diag, red[2] = max diag (one CTA, fixed order)
__global__ void k_op_stats(int n, int nnz, const double* v, const double* d, double* red) {
  __shared__ double s0[1024], s1[1024], s2[1024];
  const int t = threadIdx.x;
  double a = 0.0, mn = INFINITY, mx = -INFINITY;
  for (long k = t; k < nnz; k += 1024) a += v[k] * v[k];
  for (long k = t; k < n; k += 1024) {
    mn = fmin(mn, d[k]);
    mx = fmax(mx, d[k]);
  }
  s0[t] = a; s1[t] = mn; s2[t] = mx;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (t < w) {
      s0[t] += s0[t + w];
      s1[t] = fmin(s1[t], s1[t + w]);
      s2[t] = fmax(s2[t], s2[t + w]);
    }
    __syncthreads();
  }
  if (t == 0) {
    red[0] = s0[0];
    red[1] = s1[0];
    red[2] = s2[0];
  }
}

static void prepare_op(const care_csr* A, void* mem, size_t bytes, cudaStream_t s, care_op* op) {
  const int n = A->n, nnz = A->nnz;
  CARE_REQUIRE(bytes >= op_bytes(n, nnz), CARE_ERR_WORKSPACE, "operator memory too small");
  Arena a;
  a.base = static_cast<char*>(mem);
  a.cap = bytes;
  op->n = n;
  op->nnz = nnz;
  op->rowptr_t = a.get<int>((size_t)n + 1);
  op->colind_t = a.get<int>((size_t)nnz);
  op->val64_t = a.get<double>((size_t)nnz);
  op->val32_t = a.get<float>((size_t)nnz);
  op->diag64 = a.get<double>((size_t)n);
  op->diag32 = a.get<float>((size_t)n);
  op->rowsum32_t = a.get<float>((size_t)n);
  int* cnt = a.get<int>((size_t)n + 1);
  double* red = a.get<double>(4);
  const int g = device_sms() * 4;
  CARE_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)n + 1), s));
  k_count_cols<<<g, 256, 0, s>>>(n, A->rowptr, A->colind, cnt);
  CARE_LAUNCH();
  k_scan<<<1, 1024, 0, s>>>(n, cnt, op->rowptr_t);
  CARE_LAUNCH();
  CARE_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)n + 1), s));
  k_scatter<<<g, 256, 0, s>>>(n, A->rowptr, A->colind, A->val, op->rowptr_t, cnt, op->colind_t, op->val64_t);
  CARE_LAUNCH();
  CARE_CUDA(cudaMemsetAsync(red, 0, sizeof(double) * 4, s));
  CARE_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  k_finish_rows<<<g, 256, 0, s>>>(n, op->rowptr_t, op->colind_t, op->val64_t, op->val32_t, op->diag64,
                                    op->diag32, op->rowsum32_t, red + 3, cnt);
  CARE_LAUNCH();
  k_op_stats<<<1, 1024, 0, s>>>(n, nnz, op->val64_t, op->diag64, red);
  CARE_LAUNCH();
  double h[4];
  int mr = 0;
  CARE_CUDA(cudaMemcpyAsync(&mr, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaMemcpyAsync(h, red, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  op->full_diag = h[3] == 0.0 ? 1 : 0;
  op->max_row_nnz = mr;
  op->a_fro = std::sqrt(h[0]);
  op->diag_const = (n == 0 || h[1] == h[2]) ? 1 : 0;
}

// ---------------------------------------------------------- problem -------
struct Prob {
  long n = 0;
  int m = 0, p = 0;
  double* B64 = nullptr;  // n x m row-major
  double* Ct64 = nullptr; // n x p row-major (C^T)
  int ldb = 0, ldc = 0;
  double ctc_fro = 0.0, btb_fro = 0.0;
};

struct Ref {
  double *QZ = nullptr, *QZn = nullptr, *Zm = nullptr, *Wb = nullptr, *Wb2 = nullptr;
  int ldq = 0, ldbig = 0, rcap = 0, bigcap = 0;
  int r = 0;
  std::vector<double> s;  // Z = QZ diag(s)
};

static void alloc_prob(Ctx& c, Prob& P, long n, int m, int p) {
  P.n = n; P.m = m; P.p = p;
  P.ldb = pad_ld<double>(std::max(m, 1));
  P.ldc = pad_ld<double>(std::max(p, 1));
  P.B64 = c.ar.get<double>((size_t)n * P.ldb);
  P.Ct64 = c.ar.get<double>((size_t)n * P.ldc);
}

static void alloc_ref(Ctx& c, Ref& R, long n, int rcap, int bigcap) {
  R.rcap = rcap;
  R.bigcap = bigcap;
  R.ldq = pad_ld<double>(std::max(rcap, 1));
  R.ldbig = pad_ld<double>(std::max(bigcap, 1));
  R.QZ = c.ar.get<double>((size_t)n * R.ldq);
  R.QZn = c.ar.get<double>((size_t)n * R.ldq);
  R.Zm = c.ar.get<double>((size_t)n * R.ldq);
  R.Wb = c.ar.get<double>((size_t)n * R.ldbig);
  R.Wb2 = c.ar.get<double>((size_t)n * R.ldbig);
}

// device scratch of the small dense algebra of Algorithms 1-2 for matrices up to
// rt x rt formed from factors with k columns: the product, its eigendecomposition
// work and eigenvectors, and the coefficient blocks
static size_t dense_scratch_elems(int rt, int k) {
  const size_t r2 = (size_t)rt * rt;
  return r2 + std::max(2 * (size_t)rt * k + 64, dev_symeig_work_elems(rt) + 4 * r2 + 8 * (size_t)rt + 4096) + 4096;
}

// tc_maxdim > 0 also reserves the scratch of the tensor-core FP64 products whose
// operand widths add up to at most tc_maxdim (Algorithms 1-2); dense_rt > 0 the
// device scratch of the small dense algebra (dense_scratch_elems).
static void alloc_small(Ctx& c, long n, int maxc, int smallcap, int tc_maxdim = 0, int dense_rt = 0,
                        int dense_k = 0) {
  if (dense_rt > 0) {
    c.dsm_cap = dense_scratch_elems(dense_rt, dense_k);
    c.dsm = c.ar.get<double>(c.dsm_cap);
  }
  if (tc_maxdim > 0) {
    // reserved whether or not the tensor cores are switched on, so that the
    // workspace query does not depend on the switch
    c.tc = tc_alloc(c.ar, tc_maxdim);
    c.tc_maxdim = tc_maxdim;
    if (!c.counting()) CARE_CUDA(cudaMemsetAsync(c.tc.err, 0, sizeof(int), c.s));
  }
  c.dS_cap = (size_t)smallcap;
  c.dS = c.ar.get<double>(c.dS_cap);
  c.dG_cap = (size_t)smallcap;
  c.dG = c.ar.get<double>(c.dG_cap);
  const long tiles = (long)((maxc + 63) / 64) * ((maxc + 63) / 64);
  // room for the split-K partials of any product up to maxc x maxc (at least
  // one slice of the widest one, up to 128 MB for the narrower ones)
  c.gw_cap = std::max((size_t)(2L * device_sms() + tiles + 2) * 64 * 64, (size_t)1 << 24);
  c.gw = c.ar.get<double>(c.gw_cap);
}

// boundary (column-major FP64) -> internal row-major problem data
static void load_prob(Ctx& c, Prob& P, const double* B, int ldb, const double* C, int ldc) {
  if (P.m) copy2d<double, double>(P.n, P.m, B, 1, ldb, P.B64, P.ldb, 1, 1.0, c.s);
  if (P.p) copy2d<double, double>(P.n, P.p, C, ldc, 1, P.Ct64, P.ldc, 1, 1.0, c.s);
  std::vector<double> G = gram_h<double>(c, P.n, P.p, P.p, P.Ct64, P.ldc, P.Ct64, P.ldc);
  double s = 0.0;
  for (double v : G) s += v * v;
  P.ctc_fro = std::sqrt(s);
  std::vector<double> Gb = gram_h<double>(c, P.n, P.m, P.m, P.B64, P.ldb, P.B64, P.ldb);
  s = 0.0;
  for (double v : Gb) s += v * v;
  P.btb_fro = std::sqrt(s);
  CARE_REQUIRE(std::isfinite(P.ctc_fro) && std::isfinite(P.btb_fro), CARE_NONFINITE, "B or C not finite");
}

// ------------------------------------------------------- Algorithm 1 ------
struct Alg1Out {
  double res = 0.0;  // ||R||_F = ||H||_F (before truncation)
  int rp = 0, rm = 0;
  std::vector<double> QB;  // rq x m = Q_Z^T B
};

// Residual factor decomposition (Algorithm 1) in FP64 for Z = Q_Z T_Z:
// F = [Z, A^T Z, Z Z^T B, C^T] is expressed in the orthonormal basis
// [Q_Z, Q_perp], where Q_perp spans the part of [A^T Z, C^T] outside range(Q_Z)
// (Z Z^T B lies in range(Q_Z)), giving F = U T; H = T M T^T; its
// eigenvalues give ||R||_F and, after truncation at +-eta_r, the factors
// C+- = U Q+- |Lambda+-|^{1/2}, written as To (row-major) into Cout = [C+ | C-].
template <class To>
static Alg1Out alg1(Ctx& c, const Prob& P, Ref& R, int rq, const std::vector<double>& TZ, int r, double eta_rel,
                    To* Cout, int ldco, int ccap) {
  Alg1Out o;
  const long n = P.n;
  const int m = P.m, p = P.p;
  const int q1 = r + p;
  CARE_REQUIRE(q1 <= R.bigcap, CARE_ERR_RANK_CAPACITY, "Algorithm 1: [A^T Z, C^T] exceeds capacity");
  // W = [A^T Z | C^T]
  if (r) {
    spmm<double>(op64(c.op), cd{0.0, 0.0}, false, R.Zm, R.ldq, R.Wb, R.ldbig, r, c.s);
    c.spmm_calls++;
  }
  if (p) copy2d<double, double>(n, p, P.Ct64, P.ldc, 1, R.Wb + r, R.ldbig, 1, 1.0, c.s);
  std::vector<double> Cw = cgs2<double>(c, n, R.QZ, R.ldq, rq, R.Wb, R.ldbig, q1);  // rq x q1
  o.QB = gram_h<double>(c, n, rq, m, R.QZ, R.ldq, P.B64, P.ldb);
  std::vector<double> fl(q1, 0.0);
  for (int j = 0; j < q1; ++j) {
    double s = 0.0;
    for (int i = 0; i < rq; ++i) s += Cw[(size_t)i * q1 + j] * Cw[(size_t)i * q1 + j];
    fl[j] = 1e-28 * s;
  }
  OrthOut O = orth_rr<double>(c, n, q1, R.Wb, R.ldbig, R.Wb2, R.ldbig, 1e-12, &fl, true, 0, nullptr, 0,
                              Cout != nullptr);
  const int qp = O.rank;
  const int rt = rq + qp;
  // T blocks, each rt x (r | r | m | p), row-major
  std::vector<double> tZ((size_t)rt * r, 0.0), tA((size_t)rt * r, 0.0), tK((size_t)rt * m, 0.0),
      tC((size_t)rt * p, 0.0);
  for (int i = 0; i < rq; ++i)
    for (int j = 0; j < r; ++j) tZ[(size_t)i * r + j] = TZ[(size_t)i * r + j];
  for (int i = 0; i < rt; ++i) {
    for (int j = 0; j < r; ++j) tA[(size_t)i * r + j] = i < rq ? Cw[(size_t)i * q1 + j] : O.T[(size_t)(i - rq) * q1 + j];
    for (int j = 0; j < p; ++j)
      tC[(size_t)i * p + j] = i < rq ? Cw[(size_t)i * q1 + r + j] : O.T[(size_t)(i - rq) * q1 + r + j];
  }
  // K = Z Z^T B -> coefficients T_Z T_Z^T (Q_Z^T B) in the Q_Z rows
  {
    std::vector<double> TT((size_t)rq * rq, 0.0);
    host_gemm_nt(rq, rq, r, TZ.data(), r, TZ.data(), r, nullptr, TT.data(), rq, true);
    for (int i = 0; i < rq; ++i)
      for (int j = 0; j < m; ++j) {
        double s = 0.0;
        for (int k = 0; k < rq; ++k) s += TT[(size_t)i * rq + k] * o.QB[(size_t)k * m + j];
        tK[(size_t)i * m + j] = s;
      }
  }
  // H = tZ tA^T + tA tZ^T - tK tK^T + tC tC^T  (= T M T^T) = L R^T with
  // L = [tZ, tA, tK, tC] and R = [tA, tZ, -tK, tC], formed on the device
  DevSmall ds{c.dsm, c.dsm_cap, 0};
  const int kq = 2 * r + m + p;
  std::vector<double> L((size_t)rt * kq), Rt((size_t)kq * rt);
  for (int i = 0; i < rt; ++i) {
    double* li = &L[(size_t)i * kq];
    for (int j = 0; j < r; ++j) {
      li[j] = tZ[(size_t)i * r + j];
      li[r + j] = tA[(size_t)i * r + j];
      Rt[(size_t)j * rt + i] = tA[(size_t)i * r + j];
      Rt[(size_t)(r + j) * rt + i] = tZ[(size_t)i * r + j];
    }
    for (int j = 0; j < m; ++j) {
      li[2 * r + j] = tK[(size_t)i * m + j];
      Rt[(size_t)(2 * r + j) * rt + i] = -tK[(size_t)i * m + j];
    }
    for (int j = 0; j < p; ++j) {
      li[2 * r + m + j] = tC[(size_t)i * p + j];
      Rt[(size_t)(2 * r + m + j) * rt + i] = tC[(size_t)i * p + j];
    }
  }
  double* H = dev_small_product(c, ds, rt, kq, L, Rt);
  // eigenvalues on the device; eigenvectors only for those kept by the truncation at
  // +-eta_r (none when only ||R||_F is wanted)
  std::vector<double> lam;
  const size_t ew = dev_symeig_work_elems(rt);
  double* ework = ds.get(ew);
  double* Vd = ds.get((size_t)rt * rt);
  const double th = now_ms();
  auto kept_r = [eta_rel, want = Cout != nullptr](double l, double lmx) {
    if (!want) return false;
    const double e = eta_rel * lmx;
    return e > 0 ? (l >= e || l <= -e) : l != 0.0;
  };
  std::vector<int> sel = dev_symeig_select(rt, H, rt, lam, Vd, kept_r, ework, ew, c.s);
  c.ms_host += now_ms() - th;
  c.host_syncs += 3;
  double ss = 0.0, lmax = 0.0;
  for (double l : lam) {
    ss += l * l;
    lmax = std::max(lmax, std::fabs(l));
  }
  o.res = std::sqrt(ss);
  CARE_REQUIRE(std::isfinite(o.res), CARE_NONFINITE, "residual not finite");
  if (!Cout) return o;
  const double eta = eta_rel * lmax;
  // the kept eigenpairs: positive ones in descending order, then negative ones ascending
  std::vector<int> pos(rt, -1);
  for (int q = 0; q < (int)sel.size(); ++q) pos[sel[q]] = q;
  std::vector<int> jp, jm;
  for (int t = rt - 1; t >= 0; --t)
    if (pos[t] >= 0 && (eta > 0 ? lam[t] >= eta : lam[t] > 0)) jp.push_back(t);
  for (int t = 0; t < rt; ++t)
    if (pos[t] >= 0 && (eta > 0 ? lam[t] <= -eta : lam[t] < 0)) jm.push_back(t);
  o.rp = (int)jp.size();
  o.rm = (int)jm.size();
  const int cw = o.rp + o.rm;
  CARE_REQUIRE(cw <= ccap, CARE_ERR_RANK_CAPACITY, "Algorithm 1: residual factor exceeds capacity");
  if (cw == 0) return o;
  // coefficient block S (rt x cw) = V(:, kept) |Lambda|^{1/2}: rows 0..rq-1 go with Q_Z,
  // rows rq.. with the new directions
  std::vector<double> scl(cw);
  std::vector<int> qi(cw);
  for (int col = 0; col < cw; ++col) {
    const int t = col < o.rp ? jp[col] : jm[col - o.rp];
    qi[col] = pos[t];
    scl[col] = std::sqrt(std::fabs(lam[t]));
  }
  double* S = ds.get((size_t)rt * cw);
  eig_coeffs(c, ds, rt, cw, Vd, rt, qi, scl, S);
  gemm_c<double, To>(c, n, rq, cw, 1.0, R.QZ, R.ldq, S, cw, 0.0, Cout, ldco);
  if (qp) {
    const double* S2 = S + (size_t)rq * cw;
    const double* Vb = R.Wb;
    if (!O.Rinv.empty()) {
      // deferred R^{-1} of the Cholesky QR second pass: basis Wb2, coefficients R^{-1} S2
      double* RS = ds.get((size_t)qp * cw);
      const double* dRi = to_dev(c, ds, O.Rinv);
      gemm_c<double, double>(c, qp, qp, cw, 1.0, dRi, qp, S2, cw, 0.0, RS, cw);
      S2 = RS;
      Vb = R.Wb2;
    }
    gemm_c<double, To>(c, n, qp, cw, 1.0, Vb, R.ldbig, S2, cw, 1.0, Cout, ldco);
  }
  return o;
}

// ------------------------------------------------------- Algorithm 2 ------
// Solution factor decomposition (Algorithm 2) in FP64: G = [Z, Y] with
// Z = Q_Z diag(s) and the new factor Y (n x ny, precision Ti) carrying signs
// N = diag(I, sign); G = V Gamma with V = [Q_Z, Q_perp]; P = Gamma N Gamma^T;
// keep sigma >= eta_s = eta_s_mult * u * max|sigma|; Z_new = V Theta+ Sigma+^{1/2}
// (kept as Q_Z <- V Theta+, s <- Sigma+^{1/2}).
template <class Ti>
static void alg2(Ctx& c, Ref& R, long n, const Ti* Yp, int np, const Ti* Ym, int nm, int ldy, double eta_mult) {
  const int ny = np + nm;
  CARE_REQUIRE(ny <= R.bigcap, CARE_ERR_RANK_CAPACITY, "Algorithm 2: update exceeds capacity");
  const int r = R.r;
  std::vector<double> sign(ny, 1.0);
  for (int j = np; j < ny; ++j) sign[j] = -1.0;
  if (np) copy2d<Ti, double>(n, np, Yp, ldy, 1, R.Wb, R.ldbig, 1, 1.0, c.s);
  if (nm) copy2d<Ti, double>(n, nm, Ym, ldy, 1, R.Wb + np, R.ldbig, 1, 1.0, c.s);
  std::vector<double> Cy = cgs2<double>(c, n, R.QZ, R.ldq, r, R.Wb, R.ldbig, ny);  // r x ny
  std::vector<double> fl(ny, 0.0);
  for (int j = 0; j < ny; ++j) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += Cy[(size_t)i * ny + j] * Cy[(size_t)i * ny + j];
    fl[j] = 1e-28 * s;
  }
  OrthOut O = orth_rr<double>(c, n, ny, R.Wb, R.ldbig, R.Wb2, R.ldbig, 1e-12, &fl, true, 0, nullptr, 0, true);
  const int qp = O.rank, rt = r + qp, sc = r + ny;
  // Gamma (rt x sc) and P = Gamma N Gamma^T
  std::vector<double> Gam((size_t)rt * sc, 0.0), Nd(sc);
  for (int i = 0; i < r; ++i) {
    Gam[(size_t)i * sc + i] = R.s[i];
    for (int j = 0; j < ny; ++j) Gam[(size_t)i * sc + r + j] = Cy[(size_t)i * ny + j];
  }
  for (int i = 0; i < qp; ++i)
    for (int j = 0; j < ny; ++j) Gam[(size_t)(r + i) * sc + r + j] = O.T[(size_t)i * ny + j];
  for (int j = 0; j < sc; ++j) Nd[j] = j < r ? 1.0 : sign[j - r];
  // P = Gamma N Gamma^T on the device
  DevSmall ds{c.dsm, c.dsm_cap, 0};
  std::vector<double> GNt((size_t)sc * rt);
  for (int i = 0; i < rt; ++i)
    for (int j = 0; j < sc; ++j) GNt[(size_t)j * rt + i] = Gam[(size_t)i * sc + j] * Nd[j];
  double* Pd = dev_small_product(c, ds, rt, sc, Gam, GNt);
  // eigenvectors only for the eigenvalues kept by the truncation at eta_s
  std::vector<double> sig;
  const size_t ew = dev_symeig_work_elems(rt);
  double* ework = ds.get(ew);
  double* Vd = ds.get((size_t)rt * rt);
  const double th = now_ms();
  auto kept_s = [eta_mult](double sg, double smx) { return sg >= eta_mult * kU64 * smx && sg > 0.0; };
  std::vector<int> sel = dev_symeig_select(rt, Pd, rt, sig, Vd, kept_s, ework, ew, c.s);
  c.ms_host += now_ms() - th;
  c.host_syncs += 3;
  double smax = 0.0;
  for (double v : sig) smax = std::max(smax, std::fabs(v));
  const double eta = eta_mult * kU64 * smax;
  std::vector<int> pos(rt, -1);
  for (int q = 0; q < (int)sel.size(); ++q) pos[sel[q]] = q;
  std::vector<int> keep;
  for (int t = rt - 1; t >= 0; --t)
    if (pos[t] >= 0 && sig[t] >= eta && sig[t] > 0.0) keep.push_back(t);
  const int rn = (int)keep.size();
  CARE_REQUIRE(rn <= R.rcap, CARE_ERR_RANK_CAPACITY, "solution rank exceeds r_cap");
  std::vector<double> snew(rn), ones(rn, 1.0);
  std::vector<int> qi(rn);
  for (int col = 0; col < rn; ++col) {
    snew[col] = std::sqrt(sig[keep[col]]);
    qi[col] = pos[keep[col]];
  }
  if (rn) {
    double* S = ds.get((size_t)rt * rn);
    eig_coeffs(c, ds, rt, rn, Vd, rt, qi, ones, S);
    if (r) gemm_c<double, double>(c, n, r, rn, 1.0, R.QZ, R.ldq, S, rn, 0.0, R.QZn, R.ldq);
    if (qp) {
      const double* S2 = S + (size_t)r * rn;
      const double* Vb = R.Wb;
      if (!O.Rinv.empty()) {
        double* RS = ds.get((size_t)qp * rn);
        const double* dRi = to_dev(c, ds, O.Rinv);
        gemm_c<double, double>(c, qp, qp, rn, 1.0, dRi, qp, S2, rn, 0.0, RS, rn);
        S2 = RS;
        Vb = R.Wb2;
      }
      gemm_c<double, double>(c, n, qp, rn, 1.0, Vb, R.ldbig, S2, rn, r ? 1.0 : 0.0, R.QZn, R.ldq);
    }
  }
  std::swap(R.QZ, R.QZn);
  R.r = rn;
  R.s = snew;
}

// Z = Q_Z diag(s) into R.Zm
static void materialize_Z(Ctx& c, Ref& R, long n) {
  if (!R.r) return;
  copy2d<double, double>(n, R.r, R.QZ, R.ldq, 1, R.Zm, R.ldq, 1, 1.0, c.s);
  scale_cols<double>(n, R.r, R.Zm, R.ldq, upload(c, R.s), c.s);
}

static double res_paper(const Ctx& c, const Prob& P, const Ref& R, double res) {
  double s4 = 0.0;
  for (double v : R.s) s4 += v * v * v * v;
  const double ztz = std::sqrt(s4);
  const double den = 2.0 * c.op.a_fro * ztz + P.btb_fro * ztz * ztz + P.ctc_fro;
  return den > 0 ? res / den : 0.0;
}

// ----------------------------------------------------------- sessions -----
struct Caps {
  int rcap, bcap, adicap, hcap, bigcap, maxc, small;
};
static Caps caps_for(int n, int m, int p, int rcap, const care_opts& o) {
  Caps k;
  k.rcap = std::max(rcap, 1);
  k.bcap = std::max(2 * k.rcap + p + m, p + m);
  k.adicap = std::max(o.adi_cap, 2 * (p + m));
  k.hcap = 64;
  k.bigcap = std::max(k.rcap + p, k.adicap);
  k.maxc = std::max({k.bigcap, 2 * (k.bcap + m), k.rcap + k.bigcap});
  const size_t rt = (size_t)k.rcap + k.bigcap;
  k.small = (int)std::min<size_t>(rt * rt + 2 * (size_t)k.bcap * k.bcap + 2 * (size_t)(2 * (k.bcap + m)) * (2 * (k.bcap + m)) + 65536,
                                  (size_t)1 << 30);
  (void)n;
  return k;
}

template <class T>
struct Session {
  Prob P;
  Ref R;
  Inner<T> in;
  T* CtT = nullptr;  // n x p, inner precision
  int ldct = 0;
};

template <class T>
static void alloc_session(Ctx& c, Session<T>& S, int n, int nnz, int m, int p, const Caps& k, bool ref) {
  // tensor-core scratch: the FP64 products of Algorithms 1-2 (reference sessions) or the
  // low-precision Grams of the shift generation (width <= 2 x 64)
  alloc_small(c, n, k.maxc, k.small, ref ? std::max(k.rcap + k.bigcap, 2 * k.bigcap) : 256,
              ref ? std::max(2 * k.rcap + p, k.rcap + k.bigcap) : 0,
              ref ? std::max(2 * k.rcap + m + p, k.rcap + k.bigcap) : 0);
  alloc_prob(c, S.P, n, m, p);
  S.in.alloc(c, n, m, k.bcap, k.adicap, k.hcap);
  S.ldct = pad_ld<T>(std::max(p, 1));
  S.CtT = c.ar.get<T>((size_t)n * S.ldct);
  if (ref) alloc_ref(c, S.R, n, k.rcap, k.bigcap);
  (void)nnz;
}

static void begin(Ctx& c, const care_opts* opts, cudaStream_t s, void* work, size_t bytes) {
  if (opts) c.o = *opts;
  else care_opts_default(&c.o);
  set_verbose(c.o.verbose);
  c.s = s;
  c.ar.base = static_cast<char*>(work);
  c.ar.cap = bytes;
  c.ar.off = 0;
}

// Framework 1 (Section 2) with NLR-ADI / LR-ADI inner solves in precision T.
template <class T>
static care_status solve_impl(Ctx& c, const care_csr* A, const double* B, int ldb, int m, const double* C,
                              int ldc, int p, double tol, double* Zout, int ldz, int r_cap, care_info* info) {
  const double t0 = now_ms();
  const int n = A->n;
  c.op_nnz = A->nnz;
  const Caps k = caps_for(n, m, p, r_cap, c.o);
  // operator first (its memory leads the workspace)
  void* opmem = c.ar.get<char>(op_bytes(n, A->nnz));
  Session<T> S;
  alloc_session<T>(c, S, n, A->nnz, m, p, k, true);
  if (c.counting()) return CARE_OK;
  prepare_op(A, opmem, op_bytes(n, A->nnz), c.s, &c.op);
  load_prob(c, S.P, B, ldb, C, ldc);
  // Algorithm 1/2's FP64 blocks are free during the correction solves: the joint
  // compression of the +/- factors works in them
  S.in.f64a = S.R.Wb;
  S.in.f64b = S.R.Wb2;
  S.in.f64ld = S.R.ldbig;
  S.in.f64cap = S.R.bigcap;
  copy2d<double, T>(n, m, S.P.B64, S.P.ldb, 1, S.in.B, S.in.ldm, 1, 1.0, c.s);
  copy2d<double, T>(n, p, S.P.Ct64, S.P.ldc, 1, S.CtT, S.ldct, 1, 1.0, c.s);
  const bool lo = sizeof(T) == 4;
  const double tauL = lo ? c.o.tau_L_lo : c.o.tau_L_hi;
  const double tauN = lo ? c.o.tau_N_lo : c.o.tau_N_hi;
  care_info inf{};
  // 1. initial approximation by NLR-ADI in u_s
  double t1 = now_ms();
  NlrResult nr = nlradi<T>(c, S.in, S.CtT, S.ldct, p, tauL, tauN, c.o.newton_max, c.o.jmax);
  inf.iter0_outer = nr.newton;
  inf.iter0_inner = nr.adi;
  // store Z_1 in u (FP64): compress [Z_1] with N = I (Algorithm 2 on G = Z_1)
  S.R.r = 0;
  S.R.s.clear();
  alg2<T>(c, S.R, n, S.in.Z, nr.cols, nullptr, 0, S.in.ldz, c.o.eta_s_mult);
  CARE_CUDA(cudaStreamSynchronize(c.s));
  inf.ms_phase[0] += now_ms() - t1;
  care_status st = CARE_NOT_CONVERGED;
  double prev = -1.0, res = 0.0;
  // the factor before the last Algorithm 2 (its basis stays in QZn until the next
  // update): returned instead of the last one if the last step made the residual worse
  int prev_r = 0;
  std::vector<double> prev_s;
  auto revert_if_worse = [&]() {
    if (prev > 0 && res > prev && !prev_s.empty()) {
      std::swap(S.R.QZ, S.R.QZn);
      S.R.r = prev_r;
      S.R.s = prev_s;
      res = prev;
      if (inf.nhist < CARE_HIST_MAX) inf.res_hist[inf.nhist++] = S.P.ctc_fro > 0 ? res / S.P.ctc_fro : res;
    }
  };
  for (int it = 1; it <= c.o.kmax + 1; ++it) {
    t1 = now_ms();
    materialize_Z(c, S.R, n);
    std::vector<double> TZ((size_t)S.R.r * S.R.r, 0.0);
    for (int i = 0; i < S.R.r; ++i) TZ[(size_t)i * S.R.r + i] = S.R.s[i];
    Alg1Out a1 = alg1<T>(c, S.P, S.R, S.R.r, TZ, S.R.r, c.o.eta_r_rel, S.in.W0, S.in.ldw, S.in.bcap);
    CARE_CUDA(cudaStreamSynchronize(c.s));
    inf.ms_phase[1] += now_ms() - t1;
    res = a1.res;
    const double rel = S.P.ctc_fro > 0 ? res / S.P.ctc_fro : res;
    if (inf.nhist < CARE_HIST_MAX) inf.res_hist[inf.nhist++] = rel;
    inf.iter_outer = it;
    if (verbose_level() >= 1)
      fprintf(stderr,
              "[care] refine k=%d rank=%d res=%.3e rp=%d rm=%d  t=%.1f s (nlradi %.0f, alg1 %.0f, lradi %.0f, alg2 %.0f ms; "
              "gram %.0f ms, host eig %.0f ms so far)\n",
              it, S.R.r, rel, a1.rp, a1.rm, (now_ms() - t0) * 1e-3, inf.ms_phase[0], inf.ms_phase[1], inf.ms_phase[2],
              inf.ms_phase[3], c.ms_gram, c.ms_host);
    if (rel <= tol) {
      st = CARE_OK;
      break;
    }
    if (prev > 0 && res / prev > c.o.stag_ratio) {
      st = CARE_STAGNATED;
      revert_if_worse();
      break;
    }
    if (it == c.o.kmax + 1) {
      revert_if_worse();
      break;
    }
    prev = res;
    // K_k = Z Z^T B = Q_Z (s^2 .* Q_Z^T B) in u_s
    const int r = S.R.r;
    std::vector<double> KB((size_t)r * m);
    for (int i = 0; i < r; ++i)
      for (int j = 0; j < m; ++j) KB[(size_t)i * m + j] = S.R.s[i] * S.R.s[i] * a1.QB[(size_t)i * m + j];
    gemm_c<double, T>(c, n, r, m, 1.0, S.R.QZ, S.R.ldq, upload(c, KB), m, 0.0, S.in.K, S.in.ldm);
    t1 = now_ms();
    const int bw = a1.rp + a1.rm;
    // FP64 inner factors are compressed at FP64 accuracy (harmless before Algorithm 2's own
    // truncation at 10u); FP32 ones as asked (inner_compress): a per-sign u_s truncation
    // relative to ||X_+-|| can exceed the correction X_+ - X_- itself, the joint one is
    // relative to the correction
    const int cmp = sizeof(T) == 8 ? 1 : c.o.inner_compress;
    AdiResult ad = lradi<T>(c, S.in, bw, a1.rp, true, tauL, c.o.jmax, false, cmp);
    inf.iter_inner += ad.steps;
    CARE_CUDA(cudaStreamSynchronize(c.s));
    inf.ms_phase[2] += now_ms() - t1;
    t1 = now_ms();
    prev_r = S.R.r;
    prev_s = S.R.s;
    alg2<T>(c, S.R, n, S.in.Z, ad.np, S.in.Z + (S.in.adicap - ad.nm), ad.nm, S.in.ldz, c.o.eta_s_mult);
    CARE_CUDA(cudaStreamSynchronize(c.s));
    inf.ms_phase[3] += now_ms() - t1;
  }
  // output Z = Q_Z diag(s), column-major FP64
  CARE_REQUIRE(S.R.r <= r_cap, CARE_ERR_RANK_CAPACITY, "rank exceeds r_cap");
  materialize_Z(c, S.R, n);
  if (S.R.r) copy2d<double, double>(n, S.R.r, S.R.Zm, S.R.ldq, 1, Zout, 1, ldz, 1.0, c.s);
  CARE_CUDA(cudaStreamSynchronize(c.s));
  inf.status = st;
  inf.rank = S.R.r;
  inf.res_rel_CtC = S.P.ctc_fro > 0 ? res / S.P.ctc_fro : res;
  inf.res_paper = res_paper(c, S.P, S.R, res);
  inf.krylov_iters = c.krylov_iters;
  inf.spmm_calls = c.spmm_calls;
  inf.krylov_unconverged = c.krylov_unconverged;
  inf.ms_total = now_ms() - t0;
  harvest_timings(c);
  for (int q = 0; q < 2; ++q) {
    inf.tc_ms[q] = c.tc_ms[q];
    inf.tc_gflop[q] = c.tc_gflop[q];
    inf.tc_calls[q] = c.tc_calls[q];
  }
  inf.krylov_ms = c.kry_ms;
  inf.krylov_gbyte = c.kry_gbyte;
  inf.host_syncs = c.host_syncs;
  inf.lowp_gram_calls = c.lowp_calls;
  for (int q = 0; q < 2; ++q) {
    inf.gram_ms[q] = c.gram_ms[q];
    inf.gram_gflop[q] = c.gram_gflop[q];
    inf.gram_calls[q] = c.gram_calls[q];
    inf.gemm_ms[q] = c.gemm_ms[q];
    inf.gemm_gflop[q] = c.gemm_gflop[q];
    inf.gemm_calls[q] = c.gemm_calls[q];
  }
  if (info) *info = inf;
  return st;
}

template <class T>
static care_status lradi_impl(Ctx& c, const care_csr* A, const double* B, int ldb, const double* K, int ldk,
                              int m, const double* W, int ldw, int b, double tol, double* Zout, int ldz,
                              int r_cap, care_info* info) {
  const double t0 = now_ms();
  const int n = A->n;
  c.op_nnz = A->nnz;
  care_opts o2 = c.o;
  o2.adi_cap = std::max(c.o.adi_cap, r_cap);
  const Caps k = caps_for(n, std::max(m, 1), b, 1, o2);
  void* opmem = c.ar.get<char>(op_bytes(n, A->nnz));
  Session<T> S;
  alloc_session<T>(c, S, n, A->nnz, std::max(m, 1), b, k, false);
  if (c.counting()) return CARE_OK;
  prepare_op(A, opmem, op_bytes(n, A->nnz), c.s, &c.op);
  const bool hasK = m > 0 && B && K;
  if (hasK) {
    copy2d<double, T>(n, m, B, 1, ldb, S.in.B, S.in.ldm, 1, 1.0, c.s);
    copy2d<double, T>(n, m, K, 1, ldk, S.in.K, S.in.ldm, 1, 1.0, c.s);
  } else {
    S.in.m = 0;
  }
  copy2d<double, T>(n, b, W, 1, ldw, S.in.W0, S.in.ldw, 1, 1.0, c.s);
  AdiResult a = lradi<T>(c, S.in, b, b, hasK, tol, c.o.jmax, false);
  CARE_REQUIRE(a.np <= r_cap, CARE_ERR_RANK_CAPACITY, "LR-ADI factor exceeds r_cap");
  if (a.np) copy2d<T, double>(n, a.np, S.in.Z, S.in.ldz, 1, Zout, 1, ldz, 1.0, c.s);
  CARE_CUDA(cudaStreamSynchronize(c.s));
  care_info inf{};
  inf.rank = a.np;
  inf.iter_inner = a.steps;
  inf.krylov_iters = c.krylov_iters;
  inf.spmm_calls = c.spmm_calls;
  inf.krylov_unconverged = c.krylov_unconverged;
  inf.res_rel_CtC = a.res;
  inf.status = a.converged ? CARE_OK : CARE_NOT_CONVERGED;
  inf.ms_total = now_ms() - t0;
  harvest_timings(c);
  for (int q = 0; q < 2; ++q) {
    inf.tc_ms[q] = c.tc_ms[q];
    inf.tc_gflop[q] = c.tc_gflop[q];
    inf.tc_calls[q] = c.tc_calls[q];
  }
  inf.krylov_ms = c.kry_ms;
  inf.krylov_gbyte = c.kry_gbyte;
  inf.host_syncs = c.host_syncs;
  inf.lowp_gram_calls = c.lowp_calls;
  for (int q = 0; q < 2; ++q) {
    inf.gram_ms[q] = c.gram_ms[q];
    inf.gram_gflop[q] = c.gram_gflop[q];
    inf.gram_calls[q] = c.gram_calls[q];
    inf.gemm_ms[q] = c.gemm_ms[q];
    inf.gemm_gflop[q] = c.gemm_gflop[q];
    inf.gemm_calls[q] = c.gemm_calls[q];
  }
  if (info) *info = inf;
  return (care_status)inf.status;
}

static care_status resfac_impl(Ctx& c, const care_csr* A, const double* B, int ldb, int m, const double* C,
                               int ldc, int p, const double* Z, int ldz, int r, double eta_r_rel, double* Cp,
                               int ldcp, int* rp, double* Cm, int ldcm, int* rm, int c_cap, double* res_fro) {
  const int n = A->n;
  care_opts o2 = c.o;
  o2.adi_cap = 1;
  const Caps k = caps_for(n, m, p, std::max(r, 1), o2);
  void* opmem = c.ar.get<char>(op_bytes(n, A->nnz));
  Prob P;
  Ref R;
  alloc_small(c, n, k.maxc, k.small, 3 * k.rcap + p + m, 2 * k.rcap + p, 2 * k.rcap + m + p);
  alloc_prob(c, P, n, m, p);
  alloc_ref(c, R, n, k.rcap, std::max(k.rcap + p, k.rcap));
  const int ccap = std::max(c_cap, 0);
  const int ldo = pad_ld<double>(std::max(2 * k.rcap + m + p, 1));
  double* Cout = c.ar.get<double>((size_t)n * ldo);
  if (c.counting()) return CARE_OK;
  prepare_op(A, opmem, op_bytes(n, A->nnz), c.s, &c.op);
  load_prob(c, P, B, ldb, C, ldc);
  // Z (column-major) -> row-major; orthonormal basis Q_Z with Z = Q_Z T_Z
  std::vector<double> TZ;
  int rq = 0;
  if (r) {
    copy2d<double, double>(n, r, Z, 1, ldz, R.Zm, R.ldq, 1, 1.0, c.s);
    copy2d<double, double>(n, r, R.Zm, R.ldq, 1, R.QZ, R.ldq, 1, 1.0, c.s);
    OrthOut O = orth_rr<double>(c, n, r, R.QZ, R.ldq, R.QZn, R.ldq, 1e-12, nullptr, true, 0, nullptr, 0);
    rq = O.rank;
    TZ = O.T;
  }
  const bool want = Cp != nullptr || Cm != nullptr;
  Alg1Out a = alg1<double>(c, P, R, rq, TZ, r, eta_r_rel, want ? Cout : nullptr, ldo, 2 * k.rcap + m + p);
  if (res_fro) *res_fro = a.res;
  if (rp) *rp = a.rp;
  if (rm) *rm = a.rm;
  if (want) {
    CARE_REQUIRE(a.rp <= ccap && a.rm <= ccap, CARE_ERR_RANK_CAPACITY, "residual factor exceeds c_cap");
    if (Cp && a.rp) copy2d<double, double>(n, a.rp, Cout, ldo, 1, Cp, 1, ldcp, 1.0, c.s);
    if (Cm && a.rm) copy2d<double, double>(n, a.rm, Cout + a.rp, ldo, 1, Cm, 1, ldcm, 1.0, c.s);
  }
  CARE_CUDA(cudaStreamSynchronize(c.s));
  return CARE_OK;
}

template <class T>
static care_status shifted_impl(Ctx& c, const care_op* op, const double* B, int ldb, const double* K, int ldk,
                                int m, double pre, double pim, const double* W, int ldw, int b, double* V,
                                int ldv, int* iters) {
  const long n = op->n;
  c.op_nnz = op->nnz;
  Inner<T> in;
  alloc_small(c, n, 2 * (b + m) + 64, 4 * (b + m + 8) * (b + m + 8) + 65536);
  in.alloc(c, (int)n, std::max(m, 1), b, 1, 1);
  if (c.counting()) return CARE_OK;
  c.op = *op;
  const bool hasK = m > 0 && K != nullptr && B != nullptr;
  if (hasK) {
    copy2d<double, T>(n, m, B, 1, ldb, in.B, in.ldm, 1, 1.0, c.s);
    copy2d<double, T>(n, m, K, 1, ldk, in.K, in.ldm, 1, 1.0, c.s);
  }
  copy2d<double, T>(n, b, W, 1, ldw, in.W, in.ldw, 1, 1.0, c.s);
  // the SMW solve of the LR-ADI step, without the ADI update
  const long long it0 = c.krylov_iters;
  smw_solve_public<T>(c, in, pre, pim, b, hasK);
  const bool cplx = pim != 0.0;
  if (cplx) {
    // complex interleaved column-major output: re/im of entry (i, j) at 2(i + j ldv) (+1)
    copy2d<T, double>(n, b, in.SOL, in.ldr, 2, V, 2, 2L * ldv, 1.0, c.s);
    copy2d<T, double>(n, b, in.SOL + 1, in.ldr, 2, V + 1, 2, 2L * ldv, 1.0, c.s);
  } else {
    copy2d<T, double>(n, b, in.SOL, in.ldr, 1, V, 1, ldv, 1.0, c.s);
  }
  CARE_CUDA(cudaStreamSynchronize(c.s));
  if (iters) *iters = (int)(c.krylov_iters - it0);
  return c.krylov_unconverged ? CARE_INNER_FAILED : CARE_OK;
}

}  // namespace care

// ================================================================ C ABI ====
using namespace care;

static care_status run_guarded(const std::function<care_status()>& f) {
  try {
    return f();
  } catch (const CudaError& e) {
    if (verbose_level() > 0) fprintf(stderr, "[care] CUDA error %s at %s (line %d)\n", cudaGetErrorString(e.err), e.what, e.line);
    return CARE_ERR_CUDA;
  } catch (const StatusError& e) {
    if (verbose_level() > 0) fprintf(stderr, "[care] %s: %s\n", care_status_string(e.status), e.what);
    return e.status;
  } catch (...) {
    return CARE_ERR_CUDA;
  }
}

extern "C" {

void care_opts_default(care_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->kmax = 20;
  o->jmax = 50;
  o->newton_max = 50;
  o->adi_cap = 2048;
  o->eta_r_rel = 1e-4;
  o->eta_s_mult = 10.0;
  o->tau_L_lo = 1e-5;
  o->tau_L_hi = 1e-12;
  o->tau_N_lo = 1e-5;
  o->tau_N_hi = 1e-10;
  o->krylov_tol_lo = 1e-5;
  o->krylov_tol_hi = 1e-10;
  o->krylov_maxit_lo = 100;
  o->krylov_maxit_hi = 200;
  o->krylov = CARE_KRYLOV_BICGSTAB;
  o->precond = CARE_PRECOND_ILU0;
  o->krylov_chunk = 64;
  o->stag_ratio = 0.999;
  o->shift_hmin = 4;
  o->ilu_sweeps = 3;
  o->tri_sweeps = 2;
  o->verbose = 0;
  o->inner_compress = 2;
  o->gmres_restart_lo = 30;
  o->gmres_restart_hi = 50;
}

const char* care_status_string(int s) {
  switch (s) {
    case CARE_OK: return "CARE_OK";
    case CARE_ERR_INVALID_ARG: return "CARE_ERR_INVALID_ARG";
    case CARE_ERR_CUDA: return "CARE_ERR_CUDA";
    case CARE_ERR_WORKSPACE: return "CARE_ERR_WORKSPACE";
    case CARE_ERR_RANK_CAPACITY: return "CARE_ERR_RANK_CAPACITY";
    case CARE_NOT_CONVERGED: return "CARE_NOT_CONVERGED";
    case CARE_STAGNATED: return "CARE_STAGNATED";
    case CARE_INNER_FAILED: return "CARE_INNER_FAILED";
    case CARE_UNSTABLE: return "CARE_UNSTABLE";
    case CARE_NONFINITE: return "CARE_NONFINITE";
    case CARE_ERR_SMALL_DENSE: return "CARE_ERR_SMALL_DENSE";
    case CARE_TIMEOUT: return "CARE_TIMEOUT";
    default: return "CARE_UNKNOWN_STATUS";
  }
}

const char* care_version(void) {
  return "b300-care 0.1 (sm_103a, CUDA " CARE_STR(__CUDACC_VER_MAJOR__) "." CARE_STR(__CUDACC_VER_MINOR__) ")";
}

care_status care_op_size(int n, int nnz, size_t* bytes) {
  if (n < 0 || nnz < 0 || !bytes) return CARE_ERR_INVALID_ARG;
  *bytes = op_bytes(n, nnz);
  return CARE_OK;
}

care_status care_op_prepare(const care_csr* A, void* mem, size_t bytes, care_stream_t s, care_op* op) {
  if (!A || !op || A->n < 0 || A->nnz < 0 || (A->n > 0 && (!A->rowptr || !mem))) return CARE_ERR_INVALID_ARG;
  if (A->nnz > 0 && (!A->colind || !A->val)) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    prepare_op(A, mem, bytes, (cudaStream_t)s, op);
    return CARE_OK;
  });
}

care_status care_spmm(const care_op* op, int dtype, int cplx, double pre, double pim, const void* X, int ldx,
                      int b, void* Y, int ldy, care_stream_t s) {
  if (!op || b < 0 || (dtype != 0 && dtype != 1) || (!cplx && pim != 0.0)) return CARE_ERR_INVALID_ARG;
  const int w = cplx ? 2 * b : b;
  if (ldx < w || ldy < w || (op->n > 0 && b > 0 && (!X || !Y))) return CARE_ERR_INVALID_ARG;
  const int vec = dtype == 0 ? 2 : 4;
  if (ldx % vec || ldy % vec || ((uintptr_t)X % 16) || ((uintptr_t)Y % 16)) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    if (dtype == 0)
      spmm<double>(op64(*op), cd{pre, pim}, cplx != 0, (const double*)X, ldx, (double*)Y, ldy, w, (cudaStream_t)s);
    else
      spmm<float>(op32(*op), cd{pre, pim}, cplx != 0, (const float*)X, ldx, (float*)Y, ldy, w, (cudaStream_t)s);
    return CARE_OK;
  });
}

size_t care_gram_work_size(int n, int a, int b) { return gram_work_elems(n, a, b) * sizeof(double); }

care_status care_gram(int dtype, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy, double* G,
                      int ldg, void* work, size_t work_bytes, care_stream_t s) {
  if (n < 0 || a < 0 || b < 0 || (dtype != 0 && dtype != 1) || ldx < a || ldy < b || ldg < b) return CARE_ERR_INVALID_ARG;
  if (a > 0 && b > 0 && (!G || !work || (n > 0 && (!X || !Y)))) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    const size_t el = work_bytes / sizeof(double);
    if (dtype == 0) gram<double>(n, a, b, (const double*)X, ldx, (const double*)Y, ldy, G, ldg, (double*)work, el, (cudaStream_t)s);
    else gram<float>(n, a, b, (const float*)X, ldx, (const float*)Y, ldy, G, ldg, (double*)work, el, (cudaStream_t)s);
    return CARE_OK;
  });
}

care_status care_gram_noalloc(int dtype, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy,
                              double* G, int ldg, care_stream_t s) {
  if (n < 0 || a < 0 || b < 0 || (dtype != 0 && dtype != 1) || ldx < a || ldy < b || ldg < b) return CARE_ERR_INVALID_ARG;
  if ((long)a * b > CARE_GRAM_NOALLOC_SCRATCH_DOUBLES) return CARE_ERR_INVALID_ARG;
  if (a > 0 && b > 0 && (!G || (n > 0 && (!X || !Y)))) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    if (dtype == 0) gram_noalloc<double>(n, a, b, (const double*)X, ldx, (const double*)Y, ldy, G, ldg, (cudaStream_t)s);
    else gram_noalloc<float>(n, a, b, (const float*)X, ldx, (const float*)Y, ldy, G, ldg, (cudaStream_t)s);
    return CARE_OK;
  });
}

care_status care_shifted_solve_workspace_size(const care_op* op, int m, int b, care_prec prec, const care_opts* opts,
                                              size_t* bytes) {
  if (!op || !bytes || m < 0 || b <= 0) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    Ctx c;
    begin(c, opts, nullptr, nullptr, 0);
    c.op = *op;
    if (prec == CARE_PREC_FP64)
      shifted_impl<double>(c, op, nullptr, 0, nullptr, 0, m, 0, 0, nullptr, 0, b, nullptr, 0, nullptr);
    else
      shifted_impl<float>(c, op, nullptr, 0, nullptr, 0, m, 0, 0, nullptr, 0, b, nullptr, 0, nullptr);
    *bytes = c.ar.peak + 256;
    return CARE_OK;
  });
}

care_status care_shifted_solve(const care_op* op, const double* B, int ldb, const double* K, int ldk, int m,
                               double pre, double pim, const double* W, int ldw, int b, care_prec prec,
                               const care_opts* opts, double* V, int ldv, void* work, size_t work_bytes,
                               care_stream_t s, int* iters) {
  if (!op || !W || !V || b <= 0 || m < 0 || ldw < op->n || ldv < op->n || !work) return CARE_ERR_INVALID_ARG;
  if (m > 0 && K && (!B || ldb < op->n || ldk < op->n)) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    Ctx c;
    begin(c, opts, (cudaStream_t)s, work, work_bytes);
    if (prec == CARE_PREC_FP64)
      return shifted_impl<double>(c, op, B, ldb, K, ldk, K ? m : 0, pre, pim, W, ldw, b, V, ldv, iters);
    return shifted_impl<float>(c, op, B, ldb, K, ldk, K ? m : 0, pre, pim, W, ldw, b, V, ldv, iters);
  });
}

// deterministic pseudo-random right-hand side for the autotuner (SplitMix64 hash of the index)
__global__ void k_fill_hash(long count, double* x) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x1220ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
  }
}

// Stage 2 times every configuration on two right-hand sides: the request's width b
// and a wide block of kTuneWide columns, where the Krylov chunking matters (the
// correction solves of the refinement have hundreds of columns).
constexpr int kTuneWide = 128;
static int tune_wb(int b) { return std::max(b, kTuneWide); }

// autotuner scratch: right-hand side W (n x max(b, kTuneWide) FP64), solution V
// (the same, complex FP64), the SpMM stage's blocks X, Y (n x kMaxRealCols FP64
// each: room for every width class), then the solver workspace
static size_t autotune_head_bytes(long n, int b) {
  return (((size_t)n * tune_wb(b) * 8 * 3 + (size_t)n * kMaxRealCols * 8 * 2) + 4095) & ~size_t(4095);
}

care_status care_autotune_workspace_size(const care_op* op, int m, int b, care_prec prec, size_t* bytes) {
  if (!op || !bytes || b <= 0 || m < 0) return CARE_ERR_INVALID_ARG;
  size_t s1 = 0;
  for (int kr = 0; kr < 2; ++kr) {
    care_opts o;
    care_opts_default(&o);
    o.precond = CARE_PRECOND_ILU0_EXACT;  // the ILU workspace of both ILU(0) variants
    o.krylov = kr == 0 ? CARE_KRYLOV_BICGSTAB : CARE_KRYLOV_GMRES;
    size_t sk = 0;
    care_status st = care_shifted_solve_workspace_size(op, std::max(m, 1), tune_wb(b), prec, &o, &sk);
    if (st != CARE_OK) return st;
    s1 = std::max(s1, sk);
  }
  *bytes = s1 + autotune_head_bytes(op->n, b) + 4096;
  return CARE_OK;
}

// Tuned choices per (device, n, nnz, m, b, prec), kept for the life of the process.
struct TuneKey {
  int dev, n, nnz, m, b, prec;
  bool operator==(const TuneKey& o) const {
    return dev == o.dev && n == o.n && nnz == o.nnz && m == o.m && b == o.b && prec == o.prec;
  }
};
struct TuneVal {
  int krylov, precond, tri_sweeps, chunk, vpt[kSpmmBuckets], ctas, blocked;
  double best_ms;
};
static std::mutex g_tune_mu;
static std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

care_status care_autotune(const care_op* op, int m, int b, care_prec prec, care_opts* opts, void* work,
                          size_t work_bytes, care_stream_t s, double* best_ms) {
  if (!op || !opts || !work || b <= 0) return CARE_ERR_INVALID_ARG;
  int cur_dev = 0;
  if (cudaGetDevice(&cur_dev) != cudaSuccess) return CARE_ERR_CUDA;
  const TuneKey key{cur_dev, op->n, op->nnz, m, b, (int)prec};
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : g_tune_cache)
      if (kv.first == key) {
        const TuneVal& v = kv.second;
        opts->krylov = v.krylov;
        opts->precond = v.precond;
        opts->tri_sweeps = v.tri_sweeps;
        opts->krylov_chunk = v.chunk;
        for (int k = 0; k < kSpmmBuckets; ++k) set_tuned_spmm_vpt_bucket(k, v.vpt[k]);
        set_tuned_ctas_per_sm(v.ctas);
        set_tuned_spmm_blocked(v.blocked);
        if (best_ms) *best_ms = v.best_ms;
        return CARE_OK;
      }
  }
  size_t need = 0;
  care_status st = care_autotune_workspace_size(op, m, b, prec, &need);
  if (st != CARE_OK) return st;
  if (work_bytes < need) return CARE_ERR_WORKSPACE;
  const long n = op->n;
  char* base = static_cast<char*>(work);
  const int wb = tune_wb(b);
  double* W = reinterpret_cast<double*>(base);
  double* V = W + (size_t)n * wb;
  double* SX = V + (size_t)n * wb * 2;
  double* SY = SX + (size_t)n * kMaxRealCols;
  const size_t head = autotune_head_bytes(n, b);
  void* sw = base + head;
  const size_t sw_bytes = work_bytes - head;
  cudaStream_t cs = (cudaStream_t)s;
  k_fill_hash<<<device_sms() * 4, 256, 0, cs>>>((long)n * wb, W);
  k_fill_hash<<<device_sms() * 4, 256, 0, cs>>>((long)n * kMaxRealCols, SX);
  if (cudaGetLastError() != cudaSuccess) return CARE_ERR_CUDA;
  // mid-spectrum shift from the largest diagonal magnitude
  std::vector<double> d(n);
  if (cudaMemcpyAsync(d.data(), op->diag64, sizeof(double) * n, cudaMemcpyDeviceToHost, cs) != cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return CARE_ERR_CUDA;
  double dmax = 0.0;
  for (double v : d) dmax = std::max(dmax, std::fabs(v));
  const double p = -0.05 * (dmax > 0 ? dmax : 1.0);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int prev_ctas = tuned_ctas_per_sm(), prev_blk = tuned_spmm_blocked();
  int prev_vpt[kSpmmBuckets];
  for (int k = 0; k < kSpmmBuckets; ++k) prev_vpt[k] = tuned_spmm_vpt(2 << k);  // a width of class k
  // stage 1: SpMM launch shape on the operator in the working precision (median of
  // 5 timed launches after 2 warm-up ones).  1a: CTAs per SM, row order and vectors
  // per thread at the request's width b; 1b: vectors per thread for the other width
  // classes (the Krylov solves run chunks of up to kMaxRealCols columns)
  const bool f64 = prec == CARE_PREC_FP64;
  const int vec = f64 ? 2 : 4;
  auto time_spmm = [&](int width) -> double {
    const int ld = f64 ? (int)pad_ld<double>(width) : (int)pad_ld<float>(width);
    std::vector<float> ms;
    for (int r = 0; r < 7; ++r) {
      cudaEventRecord(e0, cs);
      const care_status q = run_guarded([&] {
        if (f64) spmm<double>(op64(*op), cd{p, 0.0}, false, SX, ld, SY, ld, width, cs);
        else spmm<float>(op32(*op), cd{p, 0.0}, false, reinterpret_cast<const float*>(SX), ld,
                         reinterpret_cast<float*>(SY), ld, width, cs);
        return CARE_OK;
      });
      cudaEventRecord(e1, cs);
      cudaEventSynchronize(e1);
      if (q != CARE_OK) return 1e300;
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      if (r >= 2) ms.push_back(t);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
  };
  const int vpts[3] = {1, 2, 4}, ctas[2] = {4, 8};
  int best_ctas = prev_ctas, best_blk = prev_blk;
  int best_vpt[kSpmmBuckets];
  for (int k = 0; k < kSpmmBuckets; ++k) best_vpt[k] = prev_vpt[k];
  const int b_width = std::min(b, kMaxRealCols);
  const int b_bucket = spmm_bucket((b_width + vec - 1) / vec);
  {
    double bst = 1e300;
    // contiguous row blocks (bl = 1) lost to grid-stride rows on every stencil operator
    // measured, and inside the fused Krylov kernels; the tuner keeps grid-stride rows
    for (int bl = 0; bl < 1; ++bl)
      for (int ci = 0; ci < 2; ++ci)
        for (int vi = 0; vi < 3; ++vi) {
          set_tuned_ctas_per_sm(ctas[ci]);
          set_tuned_spmm_blocked(bl);
          set_tuned_spmm_vpt(vpts[vi]);
          const double t = time_spmm(b_width);
          if (t < bst) {
            bst = t;
            best_vpt[b_bucket] = vpts[vi];
            best_ctas = ctas[ci];
            best_blk = bl;
          }
        }
    set_tuned_ctas_per_sm(best_ctas);
    set_tuned_spmm_blocked(best_blk);
  }
  // 1b: one representative width per other class (vectors per row 2, 4, 8, 16, 32)
  for (int k = 0; k < kSpmmBuckets; ++k) {
    if (k == b_bucket) continue;
    const int width = std::min(kMaxRealCols, vec * (2 << k));
    double bst = 1e300;
    for (int vi = 0; vi < 3; ++vi) {
      set_tuned_spmm_vpt(vpts[vi]);
      const double t = time_spmm(width);
      if (t < bst) {
        bst = t;
        best_vpt[k] = vpts[vi];
      }
    }
  }
  for (int k = 0; k < kSpmmBuckets; ++k) set_tuned_spmm_vpt_bucket(k, best_vpt[k]);
  // stage 2: shifted-solve configurations with that shape
  double best = 1e300;
  care_opts bestopt = *opts;
  const int chunks[2] = {32, 64};
  struct Pc {
    int precond, sweeps;
  };
  const Pc pcs[4] = {{CARE_PRECOND_ILU0, 2}, {CARE_PRECOND_ILU0, 3}, {CARE_PRECOND_ILU0_EXACT, 1},
                     {CARE_PRECOND_NONE, 1}};
  for (int kr = 0; kr < 2; ++kr)
    for (int pc = 0; pc < 4; ++pc)
      for (int ki = 0; ki < 2; ++ki) {
        care_opts o = *opts;
        o.krylov = kr == 0 ? CARE_KRYLOV_BICGSTAB : CARE_KRYLOV_GMRES;
        o.precond = pcs[pc].precond;
        o.tri_sweeps = pcs[pc].sweeps;
        o.krylov_chunk = chunks[ki];
        double tot = 0.0;
        bool ok = true;
        for (const int width : {b, kTuneWide}) {
          int iters = 0;
          // one untimed run (graph capture, caches), one timed run
          care_shifted_solve(op, nullptr, n, nullptr, n, 0, p, 0.0, W, n, width, prec, &o, V, n, sw, sw_bytes, s,
                             &iters);
          cudaEventRecord(e0, cs);
          care_status r = care_shifted_solve(op, nullptr, n, nullptr, n, 0, p, 0.0, W, n, width, prec, &o, V, n,
                                             sw, sw_bytes, s, &iters);
          cudaEventRecord(e1, cs);
          cudaEventSynchronize(e1);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          ok = ok && r == CARE_OK;
          tot += ms;
        }
        if (ok && tot < best) {
          best = tot;
          bestopt = o;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e300) {
    set_tuned_ctas_per_sm(prev_ctas);
    for (int k = 0; k < kSpmmBuckets; ++k) set_tuned_spmm_vpt_bucket(k, prev_vpt[k]);
    set_tuned_spmm_blocked(prev_blk);
    return CARE_INNER_FAILED;
  }
  opts->krylov = bestopt.krylov;
  opts->precond = bestopt.precond;
  opts->krylov_chunk = bestopt.krylov_chunk;
  opts->tri_sweeps = bestopt.tri_sweeps;
  if (best_ms) *best_ms = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneVal tv{bestopt.krylov, bestopt.precond, bestopt.tri_sweeps, bestopt.krylov_chunk, {}, best_ctas, best_blk,
               best};
    for (int k = 0; k < kSpmmBuckets; ++k) tv.vpt[k] = best_vpt[k];
    g_tune_cache.push_back({key, tv});
  }
  return CARE_OK;
}

int care_get_launch_shape(int* spmm_vpt, int* ctas_per_sm, int* spmm_blocked) {
  if (spmm_vpt)
    for (int k = 0; k < kSpmmBuckets; ++k) spmm_vpt[k] = tuned_spmm_vpt(2 << k);  // a width of class k
  if (ctas_per_sm) *ctas_per_sm = tuned_ctas_per_sm();
  if (spmm_blocked) *spmm_blocked = tuned_spmm_blocked();
  return 0;
}

care_status care_set_launch_shape(int spmm_vpt, int ctas_per_sm, int spmm_blocked) {
  if ((spmm_vpt != 1 && spmm_vpt != 2 && spmm_vpt != 4) || ctas_per_sm < 1 || ctas_per_sm > 8 ||
      (spmm_blocked != 0 && spmm_blocked != 1))
    return CARE_ERR_INVALID_ARG;
  set_tuned_spmm_vpt(spmm_vpt);
  set_tuned_ctas_per_sm(ctas_per_sm);
  set_tuned_spmm_blocked(spmm_blocked);
  return CARE_OK;
}

care_status care_workspace_size(int n, int nnz, int m, int p, int r_cap, care_prec prec, const care_opts* opts,
                                size_t* bytes) {
  if (n < 0 || nnz < 0 || m < 0 || p < 0 || r_cap <= 0 || !bytes) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    size_t best = 0;
    for (int mode = 0; mode < 3; ++mode) {
      Ctx c;
      begin(c, opts, nullptr, nullptr, 0);
      care_csr A{n, nnz, nullptr, nullptr, nullptr};
      if (mode == 0) {
        if (prec == CARE_PREC_FP64) solve_impl<double>(c, &A, nullptr, n, m, nullptr, p, p, 0, nullptr, n, r_cap, nullptr);
        else solve_impl<float>(c, &A, nullptr, n, m, nullptr, p, p, 0, nullptr, n, r_cap, nullptr);
      } else if (mode == 1) {
        // lyap_lradi with right-hand side width p and feedback width m
        if (prec == CARE_PREC_FP64) lradi_impl<double>(c, &A, nullptr, n, nullptr, n, m, nullptr, n, p, 0, nullptr, n, r_cap, nullptr);
        else lradi_impl<float>(c, &A, nullptr, n, nullptr, n, m, nullptr, n, p, 0, nullptr, n, r_cap, nullptr);
      } else {
        resfac_impl(c, &A, nullptr, n, m, nullptr, p, p, nullptr, n, r_cap, 0, nullptr, n, nullptr, nullptr, n, nullptr, 0, nullptr);
      }
      best = std::max(best, c.ar.peak);
    }
    *bytes = best + 256;
    return CARE_OK;
  });
}

care_status care_solve(const care_csr* A, const double* B, int ldb, int m, const double* C, int ldc, int p,
                       double tol, care_prec prec, const care_opts* opts, double* Z, int ldz, int r_cap, void* work,
                       size_t work_bytes, care_stream_t s, care_info* info) {
  if (!A || A->n <= 0 || m <= 0 || p <= 0 || !B || !C || !Z || !work || ldb < A->n || ldc < p || ldz < A->n ||
      r_cap <= 0 || !(tol > 0))
    return CARE_ERR_INVALID_ARG;
  if (!A->rowptr || !A->colind || !A->val) return CARE_ERR_INVALID_ARG;
  if (prec < CARE_PREC_FP64 || prec > CARE_PREC_MIXED_BF16) return CARE_ERR_INVALID_ARG;
  care_status st = run_guarded([&] {
    Ctx c;
    begin(c, opts, (cudaStream_t)s, work, work_bytes);
    c.lowp = prec == CARE_PREC_MIXED_TF32 ? 1 : (prec == CARE_PREC_MIXED_BF16 ? 2 : 0);
    if (prec == CARE_PREC_FP64) return solve_impl<double>(c, A, B, ldb, m, C, ldc, p, tol, Z, ldz, r_cap, info);
    return solve_impl<float>(c, A, B, ldb, m, C, ldc, p, tol, Z, ldz, r_cap, info);
  });
  if (info) info->status = st;
  return st;
}

// ---- batched solve -------------------------------------------------------
static size_t solve_ws_bytes(const care_csr* A, int m, int p, int r_cap, care_prec prec, const care_opts* opts) {
  size_t b = 0;
  if (care_workspace_size(A->n, A->nnz, m, p, r_cap, prec, opts, &b) != CARE_OK) return 0;
  return (b + 4095) & ~size_t(4095);
}

care_status care_workspace_size_batched(int count, const care_csr* const* A, const int* m, const int* p,
                                        const int* r_cap, care_prec prec, const care_opts* opts, int workers,
                                        size_t* bytes) {
  if (count < 0 || workers <= 0 || !bytes || (count > 0 && (!A || !m || !p || !r_cap))) return CARE_ERR_INVALID_ARG;
  size_t mx = 0;
  for (int i = 0; i < count; ++i) {
    if (!A[i]) return CARE_ERR_INVALID_ARG;
    const size_t b = solve_ws_bytes(A[i], m[i], p[i], r_cap[i], prec, opts);
    if (b == 0) return CARE_ERR_INVALID_ARG;
    mx = std::max(mx, b);
  }
  const int w = std::max(1, std::min(workers, count));
  *bytes = mx * (size_t)w;
  return CARE_OK;
}

care_status care_solve_batched(int count, const care_csr* const* A, const double* const* B, const int* ldb,
                               const int* m, const double* const* C, const int* ldc, const int* p, double tol,
                               care_prec prec, const care_opts* opts, double* const* Z, const int* ldz,
                               const int* r_cap, int workers, void* work, size_t work_bytes, care_stream_t s,
                               care_info* info) {
  if (count < 0 || workers <= 0) return CARE_ERR_INVALID_ARG;
  if (count == 0) return CARE_OK;
  if (!A || !B || !ldb || !m || !C || !ldc || !p || !Z || !ldz || !r_cap || !work) return CARE_ERR_INVALID_ARG;
  size_t need = 0;
  care_status st = care_workspace_size_batched(count, A, m, p, r_cap, prec, opts, workers, &need);
  if (st != CARE_OK) return st;
  if (work_bytes < need) return CARE_ERR_WORKSPACE;
  const int W = std::max(1, std::min(workers, count));
  const size_t slice = need / W;
  // longest-processing-time order by estimated cost n (m + p)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return (double)A[x]->n * (m[x] + p[x]) > (double)A[y]->n * (m[y] + p[y]);
  });
  std::vector<care_status> status(count, CARE_OK);
  std::vector<care_info> infos(count);
  std::atomic<int> next{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CARE_ERR_CUDA;
  // workers start after the caller's stream has reached this point
  cudaEvent_t start_ev = nullptr;
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess) return CARE_ERR_CUDA;
  if (cudaEventRecord(start_ev, (cudaStream_t)s) != cudaSuccess) {
    cudaEventDestroy(start_ev);
    return CARE_ERR_CUDA;
  }
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  std::vector<cudaStream_t> streams(W, nullptr);
  std::vector<cudaEvent_t> done(W, nullptr);
  bool setup_ok = true;
  for (int w = 0; w < W; ++w) {
    setup_ok &= cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking) == cudaSuccess;
    setup_ok &= cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming) == cudaSuccess;
    if (setup_ok) setup_ok &= cudaStreamWaitEvent(streams[w], start_ev, 0) == cudaSuccess;
  }
  if (setup_ok) {
    std::vector<std::thread> pool;
    for (int w = 0; w < W; ++w) {
      pool.emplace_back([&, w] {
        cudaSetDevice(dev);
        omp_set_num_threads(std::max(1, hw / W));  // share the host cores between workers
        char* base = static_cast<char*>(work) + slice * w;
        for (int k = next.fetch_add(1); k < count; k = next.fetch_add(1)) {
          const int i = order[k];
          status[i] = care_solve(A[i], B[i], ldb[i], m[i], C[i], ldc[i], p[i], tol, prec, opts, Z[i], ldz[i],
                                 r_cap[i], base, slice, (care_stream_t)streams[w], &infos[i]);
        }
        cudaEventRecord(done[w], streams[w]);
      });
    }
    for (auto& t : pool) t.join();
    for (int w = 0; w < W; ++w) cudaStreamWaitEvent((cudaStream_t)s, done[w], 0);
  }
  for (int w = 0; w < W; ++w) {
    if (streams[w]) cudaStreamDestroy(streams[w]);
    if (done[w]) cudaEventDestroy(done[w]);
  }
  cudaEventDestroy(start_ev);
  if (!setup_ok) return CARE_ERR_CUDA;
  if (info)
    for (int i = 0; i < count; ++i) info[i] = infos[i];
  for (int i = 0; i < count; ++i)
    if (status[i] != CARE_OK) return status[i];
  return CARE_OK;
}

// ---- batched serving mode: shifted solves of all instances in shared launches --
static care_opts persistent_opts(const care_opts* opts) {
  care_opts o;
  if (opts) o = *opts;
  else care_opts_default(&o);
  o.krylov = CARE_KRYLOV_BICGSTAB;
  o.precond = CARE_PRECOND_JACOBI;
  // Jacobi needs more iterations than ILU(0) on the stencil operators: four times
  // the limits (a request whose columns have all converged drops out of the
  // launch's phases, so it pays nothing for the others' iterations)
  o.krylov_maxit_lo = std::max(o.krylov_maxit_lo, 4 * 100);
  o.krylov_maxit_hi = std::max(o.krylov_maxit_hi, 4 * 200);
  return o;
}

care_status care_workspace_size_batched_persistent(int count, const care_csr* const* A, const int* m, const int* p,
                                                   const int* r_cap, care_prec prec, const care_opts* opts,
                                                   size_t* bytes) {
  if (count < 0 || !bytes || (count > 0 && (!A || !m || !p || !r_cap))) return CARE_ERR_INVALID_ARG;
  if (count > kBatchMaxReq) return CARE_ERR_INVALID_ARG;
  const care_opts o = persistent_opts(opts);
  size_t tot = 0;
  for (int i = 0; i < count; ++i) {
    if (!A[i]) return CARE_ERR_INVALID_ARG;
    const size_t b = solve_ws_bytes(A[i], m[i], p[i], r_cap[i], prec, &o);
    if (b == 0) return CARE_ERR_INVALID_ARG;
    tot += b;
  }
  size_t sb = 0;
  const care_status st = run_guarded([&] {
    sb = batch_scratch_bytes(std::max(count, 1));
    return CARE_OK;
  });
  if (st != CARE_OK) return st;
  *bytes = tot + ((sb + 4095) & ~size_t(4095));
  return CARE_OK;
}

care_status care_solve_batched_persistent(int count, const care_csr* const* A, const double* const* B,
                                          const int* ldb, const int* m, const double* const* C, const int* ldc,
                                          const int* p, double tol, care_prec prec, const care_opts* opts,
                                          double* const* Z, const int* ldz, const int* r_cap, void* work,
                                          size_t work_bytes, care_stream_t s, care_info* info,
                                          long long* batch_launches) {
  if (count < 0 || count > kBatchMaxReq) return CARE_ERR_INVALID_ARG;
  if (count == 0) return CARE_OK;
  if (!A || !B || !ldb || !m || !C || !ldc || !p || !Z || !ldz || !r_cap || !work) return CARE_ERR_INVALID_ARG;
  if (prec < CARE_PREC_FP64 || prec > CARE_PREC_MIXED_BF16) return CARE_ERR_INVALID_ARG;
  size_t need = 0;
  care_status st = care_workspace_size_batched_persistent(count, A, m, p, r_cap, prec, opts, &need);
  if (st != CARE_OK) return st;
  if (work_bytes < need) return CARE_ERR_WORKSPACE;
  const care_opts o = persistent_opts(opts);
  // per-instance slices of the workspace, then the launch scratch
  std::vector<size_t> off(count + 1, 0);
  for (int i = 0; i < count; ++i) off[i + 1] = off[i] + solve_ws_bytes(A[i], m[i], p[i], r_cap[i], prec, &o);
  char* base = static_cast<char*>(work);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CARE_ERR_CUDA;
  std::vector<care_status> status(count, CARE_OK);
  std::vector<care_info> infos(count);
  cudaEvent_t start_ev = nullptr;
  if (cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming) != cudaSuccess) return CARE_ERR_CUDA;
  if (cudaEventRecord(start_ev, (cudaStream_t)s) != cudaSuccess) {
    cudaEventDestroy(start_ev);
    return CARE_ERR_CUDA;
  }
  std::vector<cudaStream_t> streams(count, nullptr);
  std::vector<cudaEvent_t> done(count, nullptr);
  bool setup_ok = true;
  for (int i = 0; i < count; ++i) {
    setup_ok &= cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) == cudaSuccess;
    setup_ok &= cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming) == cudaSuccess;
    if (setup_ok) setup_ok &= cudaStreamWaitEvent(streams[i], start_ev, 0) == cudaSuccess;
  }
  long long launches = 0;
  if (setup_ok) {
    st = run_guarded([&] {
      BatchBroker broker(count, prec == CARE_PREC_FP64 ? 8 : 4, base + off[count], work_bytes - off[count]);
      const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
      std::vector<std::thread> pool;
      for (int i = 0; i < count; ++i) {
        pool.emplace_back([&, i] {
          cudaSetDevice(dev);
          omp_set_num_threads(std::max(1, hw / count));
          status[i] = run_guarded([&] {
            struct Done {
              BatchBroker& b;
              ~Done() { b.instance_done(); }
            } guard{broker};
            Ctx c;
            begin(c, &o, streams[i], base + off[i], off[i + 1] - off[i]);
            c.broker = &broker;
            c.lowp = prec == CARE_PREC_MIXED_TF32 ? 1 : (prec == CARE_PREC_MIXED_BF16 ? 2 : 0);
            if (prec == CARE_PREC_FP64)
              return solve_impl<double>(c, A[i], B[i], ldb[i], m[i], C[i], ldc[i], p[i], tol, Z[i], ldz[i],
                                        r_cap[i], &infos[i]);
            return solve_impl<float>(c, A[i], B[i], ldb[i], m[i], C[i], ldc[i], p[i], tol, Z[i], ldz[i], r_cap[i],
                                     &infos[i]);
          });
          infos[i].status = status[i];
          cudaEventRecord(done[i], streams[i]);
        });
      }
      for (auto& t : pool) t.join();
      for (int i = 0; i < count; ++i) cudaStreamWaitEvent((cudaStream_t)s, done[i], 0);
      launches = broker.launches();
      return CARE_OK;
    });
  }
  for (int i = 0; i < count; ++i) {
    if (streams[i]) cudaStreamDestroy(streams[i]);
    if (done[i]) cudaEventDestroy(done[i]);
  }
  cudaEventDestroy(start_ev);
  if (!setup_ok) return CARE_ERR_CUDA;
  if (st != CARE_OK) return st;
  if (batch_launches) *batch_launches = launches;
  if (info)
    for (int i = 0; i < count; ++i) info[i] = infos[i];
  for (int i = 0; i < count; ++i)
    if (status[i] != CARE_OK) return status[i];
  return CARE_OK;
}

care_status lyap_lradi(const care_csr* A, const double* B, int ldb, const double* K, int ldk, int m, const double* W,
                       int ldw, int b, double tol, care_prec prec, const care_opts* opts, double* Z, int ldz,
                       int r_cap, void* work, size_t work_bytes, care_stream_t s, care_info* info) {
  if (!A || A->n <= 0 || b <= 0 || !W || !Z || !work || ldw < A->n || ldz < A->n || r_cap <= 0 || !(tol > 0))
    return CARE_ERR_INVALID_ARG;
  if (m > 0 && B && K && (ldb < A->n || ldk < A->n)) return CARE_ERR_INVALID_ARG;
  if (prec < CARE_PREC_FP64 || prec > CARE_PREC_MIXED_BF16) return CARE_ERR_INVALID_ARG;
  care_status st = run_guarded([&] {
    Ctx c;
    begin(c, opts, (cudaStream_t)s, work, work_bytes);
    const int mm = (B && K) ? m : 0;
    c.lowp = prec == CARE_PREC_MIXED_TF32 ? 1 : (prec == CARE_PREC_MIXED_BF16 ? 2 : 0);
    if (prec == CARE_PREC_FP64) return lradi_impl<double>(c, A, B, ldb, K, ldk, mm, W, ldw, b, tol, Z, ldz, r_cap, info);
    return lradi_impl<float>(c, A, B, ldb, K, ldk, mm, W, ldw, b, tol, Z, ldz, r_cap, info);
  });
  if (info) info->status = st;
  return st;
}

care_status care_residual_factor(const care_csr* A, const double* B, int ldb, int m, const double* C, int ldc, int p,
                                 const double* Z, int ldz, int r, double eta_r_rel, double* Cp, int ldcp, int* rp,
                                 double* Cm, int ldcm, int* rm, int c_cap, double* res_fro, void* work,
                                 size_t work_bytes, care_stream_t s) {
  if (!A || A->n <= 0 || m <= 0 || p <= 0 || r < 0 || !B || !C || (r > 0 && !Z) || !work || ldb < A->n ||
      ldc < p || (r > 0 && ldz < A->n) || eta_r_rel < 0)
    return CARE_ERR_INVALID_ARG;
  if ((Cp && ldcp < A->n) || (Cm && ldcm < A->n)) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    Ctx c;
    begin(c, nullptr, (cudaStream_t)s, work, work_bytes);
    return resfac_impl(c, A, B, ldb, m, C, ldc, p, Z, ldz, r, eta_r_rel, Cp, ldcp, rp, Cm, ldcm, rm, c_cap, res_fro);
  });
}

unsigned long long care_kernel_launches(void) { return care::launches(); }

size_t care_ilu0_work_size(const care_op* op, int dtype) {
  if (!op) return 0;
  Arena a;
  if (dtype == 0) krylov_alloc<double>(a, op->n, true, op->nnz);
  else krylov_alloc<float>(a, op->n, true, op->nnz);
  return a.off + 256;
}

care_status care_ilu0(const care_op* op, int dtype, int exact, double p_re, double p_im, void* F, void* work,
                      size_t work_bytes, care_stream_t s) {
  if (!op || !F || !work || (dtype != 0 && dtype != 1)) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    Arena a;
    a.base = static_cast<char*>(work);
    a.cap = work_bytes;
    const bool cplx = p_im != 0.0;
    if (dtype == 0) {
      KrylovWork<double> w = krylov_alloc<double>(a, op->n, true, op->nnz);
      ilu0_factor<double>(op64(*op), cd{p_re, p_im}, cplx, exact != 0, w, (double*)F, (cudaStream_t)s);
    } else {
      KrylovWork<float> w = krylov_alloc<float>(a, op->n, true, op->nnz);
      ilu0_factor<float>(op32(*op), cd{p_re, p_im}, cplx, exact != 0, w, (float*)F, (cudaStream_t)s);
    }
    return CARE_OK;
  });
}

size_t care_symeig_work_size(int n) { return n > 0 ? dev_symeig_work_elems(n) * sizeof(double) + 256 : 256; }

care_status care_symeig(int n, const double* A, int lda, double* w, double* V, double lo, double hi, int* nsel,
                        void* work, size_t work_bytes, care_stream_t s) {
  if (n < 0 || (n > 0 && (!A || !w || !work || lda < n)) || !nsel) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    std::vector<double> wh;
    std::vector<int> sel = dev_symeig_select(
        n, A, lda, wh, V, [lo, hi, V](double l, double) { return V != nullptr && (l <= lo || l >= hi); },
        static_cast<double*>(work), work_bytes / sizeof(double), (cudaStream_t)s);
    std::copy(wh.begin(), wh.end(), w);
    *nsel = (int)sel.size();
    CARE_CUDA(cudaStreamSynchronize((cudaStream_t)s));
    return CARE_OK;
  });
}

care_status care_fp64_peak(double* tflops, care_stream_t s) {
  if (!tflops) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    *tflops = fp64_fma_peak_tflops((cudaStream_t)s);
    return CARE_OK;
  });
}

int care_tc_available(void) {
  const bool ok = tc_available();
  cudaGetLastError();
  return ok ? 1 : 0;
}

void care_set_tensor_cores(int on) { tc_set_enabled(on); }

void care_tc_test_starve(int on) { tc_set_test_starve(on); }

size_t care_tc_work_size(int maxdim) {
  Arena a;
  tc_alloc(a, std::max(maxdim, 1));
  return a.off + 256;
}

care_status care_gram_tc(int mode, int n, int a, int b, const void* X, int ldx, const void* Y, int ldy, double* G,
                         int ldg, void* work, size_t work_bytes, care_stream_t s) {
  if (mode < 0 || mode > 3 || n < 0 || a < 0 || b < 0 || ldx < a || ldy < b || ldg < b) return CARE_ERR_INVALID_ARG;
  if (a > 0 && b > 0 && (!G || !work || (n > 0 && (!X || !Y)))) return CARE_ERR_INVALID_ARG;
  if (a == 0 || b == 0) return CARE_OK;
  return run_guarded([&] {
    CARE_REQUIRE(tc_available(), CARE_ERR_CUDA, "tensor cores (sm_103a) not available");
    Arena ar;
    ar.base = static_cast<char*>(work);
    ar.cap = work_bytes;
    const int md = a + b;
    TcScratch sc = tc_alloc(ar, md);
    cudaStream_t cs = (cudaStream_t)s;
    CARE_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int), cs));
    if (mode == 0)
      tc_gram_f64(n, a, b, (const double*)X, ldx, (const double*)Y, ldy, G, ldg, sc, md, cs);
    else if (mode == 3)
      tc_gram_f32acc(n, a, b, (const float*)X, ldx, (const float*)Y, ldy, G, ldg, sc, md, cs);
    else
      tc_gram_lowp(mode, n, a, b, (const float*)X, ldx, (const float*)Y, ldy, G, ldg, sc, md, cs);
    return tc_check(sc, cs) ? CARE_TIMEOUT : CARE_OK;
  });
}

care_status care_gemm_ts(int dtype, int tc, int n, int a, int b, double alpha, const void* X, int ldx, const double* S,
                         int lds, double beta, void* Y, int ldy, void* work, size_t work_bytes, care_stream_t s) {
  if ((dtype != 0 && dtype != 1) || n < 0 || a < 0 || b < 0 || ldx < a || lds < b || ldy < b) return CARE_ERR_INVALID_ARG;
  if (n > 0 && b > 0 && (!Y || (a > 0 && (!X || !S)))) return CARE_ERR_INVALID_ARG;
  if (tc && !work) return CARE_ERR_INVALID_ARG;
  return run_guarded([&] {
    cudaStream_t cs = (cudaStream_t)s;
    if (tc && a > 0) {
      CARE_REQUIRE(tc_available(), CARE_ERR_CUDA, "tensor cores (sm_103a) not available");
      Arena ar;
      ar.base = static_cast<char*>(work);
      ar.cap = work_bytes;
      TcScratch sc = tc_alloc(ar, a + b);
      CARE_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int), cs));
      if (dtype == 0)
        tc_gemm_ts_f64<double>(n, a, b, alpha, (const double*)X, ldx, S, lds, beta, (double*)Y, ldy, sc, a + b, cs);
      else
        tc_gemm_ts_f32acc<float>(n, a, b, alpha, (const float*)X, ldx, S, lds, beta, (float*)Y, ldy, sc, a + b, cs);
      return tc_check(sc, cs) ? CARE_TIMEOUT : CARE_OK;
    }
    if (dtype == 0)
      gemm_ts<double, double>(n, a, b, alpha, (const double*)X, ldx, S, lds, beta, (double*)Y, ldy, cs);
    else
      gemm_ts<float, float>(n, a, b, alpha, (const float*)X, ldx, S, lds, beta, (float*)Y, ldy, cs);
    return CARE_OK;
  });
}

care_status care_host_symeig(int n, const double* A, double* w, double* V) {
  if (n < 0 || (n > 0 && (!A || !w))) return CARE_ERR_INVALID_ARG;
  return host_symeig(n, A, w, V) ? CARE_OK : CARE_ERR_SMALL_DENSE;
}

care_status care_host_cholesky_upper(int n, const double* G, double* R) {
  if (n < 0 || (n > 0 && (!G || !R))) return CARE_ERR_INVALID_ARG;
  return host_cholesky_upper(n, G, R) ? CARE_OK : CARE_ERR_SMALL_DENSE;
}

care_status care_host_pivoted_cholesky(int c, const double* G, double tol, int max_rank, int* piv, double* R,
                                       int* rank) {
  if (c < 0 || !rank || (c > 0 && (!G || !piv || !R))) return CARE_ERR_INVALID_ARG;
  std::vector<int> pv;
  std::vector<double> Rv;
  const int r = c ? host_pivoted_cholesky(c, G, tol, max_rank, pv, Rv) : 0;
  std::fill(R, R + (size_t)c * c, 0.0);
  std::copy(Rv.begin(), Rv.end(), R);
  std::copy(pv.begin(), pv.end(), piv);
  *rank = r;
  return CARE_OK;
}

care_status care_host_sym_lmax(int n, const double* G, double* lmax) {
  if (n < 0 || !lmax || (n > 0 && !G)) return CARE_ERR_INVALID_ARG;
  const double l = host_sym_lmax(n, G);
  if (!std::isfinite(l)) return CARE_ERR_SMALL_DENSE;
  *lmax = l;
  return CARE_OK;
}

care_status care_host_upper_inverse(int r, const double* U, double* Ui) {
  if (r < 0 || (r > 0 && (!U || !Ui))) return CARE_ERR_INVALID_ARG;
  host_upper_inverse(r, U, Ui);
  return CARE_OK;
}

care_status care_host_gemm_nt(int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                              const double* d, double* C, int ldc, int sym) {
  if (m < 0 || n < 0 || k < 0 || (sym && (m != n || A != B || lda != ldb)) || ldc < n ||
      (m > 0 && k > 0 && (!A || lda < k)) || (n > 0 && k > 0 && (!B || ldb < k)) || (m > 0 && n > 0 && !C))
    return CARE_ERR_INVALID_ARG;
  if (k == 0) {
    for (int i = 0; i < m; ++i) std::fill(C + (size_t)i * ldc, C + (size_t)i * ldc + n, 0.0);
    return CARE_OK;
  }
  host_gemm_nt(m, n, k, A, lda, B, ldb, d, C, ldc, sym != 0);
  return CARE_OK;
}

care_status care_host_symeig_outside(int n, const double* A, double* w, double* V, double lo, double hi) {
  if (n < 0 || (n > 0 && (!A || !w || !V))) return CARE_ERR_INVALID_ARG;
  return host_symeig_select(n, A, w, V, [lo, hi](double l, double) { return l <= lo || l >= hi; })
             ? CARE_OK
             : CARE_ERR_SMALL_DENSE;
}

care_status care_host_eigvals(int n, const double* A, double* wr, double* wi) {
  if (n < 0 || (n > 0 && (!A || !wr || !wi))) return CARE_ERR_INVALID_ARG;
  return host_eigvals(n, A, wr, wi) ? CARE_OK : CARE_ERR_SMALL_DENSE;
}

}  // extern "C"
