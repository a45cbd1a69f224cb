// Inner (u_s precision) solver: SMW shifted block solves, projection shifts,
// LR-ADI and NLR-ADI (Section 4), plus the orthogonalisation helpers shared
// with Algorithms 1 and 2.
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>

#include "solver.cuh"

namespace care {

static thread_local int g_verbose = 0;  // per calling thread (batched workers solve concurrently)
int verbose_level() { return g_verbose; }
void set_verbose(int v) { g_verbose = v; }

static std::atomic<int> g_ctas_per_sm{8};
int tuned_ctas_per_sm() { return g_ctas_per_sm.load(std::memory_order_relaxed); }
void set_tuned_ctas_per_sm(int v) { g_ctas_per_sm.store(v < 1 ? 1 : (v > 8 ? 8 : v)); }
static std::atomic<int> g_spmm_vpt[kSpmmBuckets] = {1, 1, 1, 1, 1};
static int clamp_vpt(int v) { return v >= 4 ? 4 : (v >= 2 ? 2 : 1); }
int tuned_spmm_vpt(int nvec) { return g_spmm_vpt[spmm_bucket(nvec)].load(std::memory_order_relaxed); }
void set_tuned_spmm_vpt(int v) {
  for (int b = 0; b < kSpmmBuckets; ++b) g_spmm_vpt[b].store(clamp_vpt(v));
}
void set_tuned_spmm_vpt_bucket(int bucket, int v) {
  if (bucket >= 0 && bucket < kSpmmBuckets) g_spmm_vpt[bucket].store(clamp_vpt(v));
}
static std::atomic<int> g_spmm_blocked{0};
int tuned_spmm_blocked() { return g_spmm_blocked.load(std::memory_order_relaxed); }
void set_tuned_spmm_blocked(int v) { g_spmm_blocked.store(v ? 1 : 0); }

static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launch_n(long delta) { g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(); }

int device_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 148;
  }
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
      cudaGetLastError();
      v = 148;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

template <>
OpT<double> op_of<double>(const Ctx& c) { return op64(c.op); }
template <>
OpT<float> op_of<float>(const Ctx& c) { return op32(c.op); }

const double* upload(Ctx& c, const std::vector<double>& h) {
  CARE_REQUIRE(h.size() <= c.dS_cap, CARE_ERR_WORKSPACE, "small-matrix staging too small");
  if (!h.empty())
    CARE_CUDA(cudaMemcpyAsync(c.dS, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  return c.dS;
}

template <class T>
std::vector<double> gram_h(Ctx& c, long n, int a, int b, const T* X, int ldx, const T* Y, int ldy, bool lowp) {
  std::vector<double> h((size_t)a * b, 0.0);
  if (a == 0 || b == 0) return h;
  CARE_REQUIRE((size_t)a * b <= c.dG_cap, CARE_ERR_WORKSPACE, "gram output staging too small");
  const double t0 = verbose_level() >= 1 ? (cudaStreamSynchronize(c.s), now_ms()) : 0.0;
  if (!c.ge0) {
    CARE_CUDA(cudaEventCreate(&c.ge0));
    CARE_CUDA(cudaEventCreate(&c.ge1));
  }
  CARE_CUDA(cudaEventRecord(c.ge0, c.s));
  const bool sym0 = a == b && (const void*)X == (const void*)Y && ldx == ldy;
  bool on_tc = false;
  if (sizeof(T) == 4 && lowp && c.lowp && c.tc.ok() && a + b <= c.tc_maxdim && tc_available()) {
    // TF32 / BF16 tensor-core Gram of the shift generation (CARE_PREC_MIXED_TF32 / _BF16)
    tc_gram_lowp(c.lowp, n, a, b, reinterpret_cast<const float*>(X), ldx, reinterpret_cast<const float*>(Y), ldy,
                 c.dG, b, c.tc, c.tc_maxdim, c.s);
    c.tc_used = true;
    c.lowp_calls++;
  } else if (tc_use(c, n, a, b, sym0 ? a : a + b)) {
    if constexpr (sizeof(T) == 8)
      tc_gram_f64(n, a, b, X, ldx, Y, ldy, c.dG, b, c.tc, c.tc_maxdim, c.s);
    else
      tc_gram_f32acc(n, a, b, X, ldx, Y, ldy, c.dG, b, c.tc, c.tc_maxdim, c.s);
    c.tc_used = on_tc = true;
  } else {
    gram<T>(n, a, b, X, ldx, Y, ldy, c.dG, b, c.gw, c.gw_cap, c.s);
  }
  CARE_CUDA(cudaEventRecord(c.ge1, c.s));
  CARE_CUDA(cudaMemcpyAsync(h.data(), c.dG, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  CARE_CUDA(cudaStreamSynchronize(c.s));
  c.host_syncs++;
  harvest_timings(c);
  float ms = 0.f;
  CARE_CUDA(cudaEventElapsedTime(&ms, c.ge0, c.ge1));
  const int k = sizeof(T) == 8 ? 0 : 1;
  const double gf = (sym0 ? (double)n * a * (a + 1) : 2.0 * n * a * b) * 1e-9;
  if (on_tc) {
    c.tc_ms[k] += ms;
    c.tc_gflop[k] += gf;
    c.tc_calls[k] += 1;
  } else {
    c.gram_ms[k] += ms;
    c.gram_gflop[k] += gf;
    c.gram_calls[k] += 1;
  }
  if (verbose_level() >= 1) c.ms_gram += now_ms() - t0;
  return h;
}
template std::vector<double> gram_h<float>(Ctx&, long, int, int, const float*, int, const float*, int, bool);
template std::vector<double> gram_h<double>(Ctx&, long, int, int, const double*, int, const double*, int, bool);

// --------------------------------------------------- small dense on device --
double* to_dev(Ctx& c, DevSmall& ds, const std::vector<double>& h) {
  double* d = ds.get(std::max<size_t>(h.size(), 1));
  if (!h.empty()) CARE_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  return d;
}

double* dev_small_product(Ctx& c, DevSmall& ds, int rt, int k, const std::vector<double>& L,
                          const std::vector<double>& Rt) {
  double* M = ds.get((size_t)rt * rt);
  const size_t mark = ds.off;
  const double* dL = to_dev(c, ds, L);
  const double* dRt = to_dev(c, ds, Rt);
  gemm_c<double, double>(c, rt, k, rt, 1.0, dL, k, dRt, rt, 0.0, M, rt);
  ds.off = mark;  // the factors are dead once the (stream-ordered) product has run
  return M;
}

__global__ void k_eig_coeffs(int rows, int cols, const double* __restrict__ V, int ldv, const int* __restrict__ q,
                             const double* __restrict__ sc, double* __restrict__ S) {
  const long total = (long)rows * cols;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t / cols), col = (int)(t % cols);
    S[t] = V[(long)q[col] * ldv + i] * sc[col];
  }
}

void eig_coeffs(Ctx& c, DevSmall& ds, int rows, int cols, const double* V, int ldv, const std::vector<int>& q,
                const std::vector<double>& sc, double* S) {
  if (rows == 0 || cols == 0) return;
  int* dq = reinterpret_cast<int*>(ds.get((size_t)cols));
  CARE_CUDA(cudaMemcpyAsync(dq, q.data(), sizeof(int) * cols, cudaMemcpyHostToDevice, c.s));
  const double* dsc = to_dev(c, ds, sc);
  k_eig_coeffs<<<device_sms() * 4, 256, 0, c.s>>>(rows, cols, V, ldv, dq, dsc, S);
  CARE_LAUNCH();
}

// ------------------------------------------------------------ orth_rr -----
template <class T>
OrthOut orth_rr(Ctx& c, long n, int cols, T* X, int ldx, T* buf, int ldb, double drop_rel,
                const std::vector<double>* colfloor2, bool second_pass, int max_rank, T* out, int ldo,
                bool defer_rinv, bool lowp_gram) {
  OrthOut o;
  CARE_REQUIRE(out == nullptr || !second_pass, CARE_ERR_INVALID_ARG, "orth_rr: out needs one pass");
  if (cols == 0) return o;
  std::vector<double> G = gram_h<T>(c, n, cols, cols, X, ldx, X, ldx, lowp_gram);
  // column scaling; columns at or below their floor are dropped.  drop_rel < 0
  // selects the unscaled mode: pivots are compared with |drop_rel| * max_j G_jj,
  // i.e. the truncation is relative to the largest column of X (used to cut
  // factors at the accuracy of the precision that produced them).
  const bool unscaled = drop_rel < 0.0;
  double gmax = 0.0;
  for (int j = 0; j < cols; ++j) gmax = std::max(gmax, G[(size_t)j * cols + j]);
  std::vector<double> d(cols, 0.0);
  for (int j = 0; j < cols; ++j) {
    const double g = G[(size_t)j * cols + j];
    const double fl = colfloor2 ? (*colfloor2)[j] : 0.0;
    if (g > fl && g > 0.0 && std::isfinite(g)) d[j] = unscaled ? 1.0 : std::sqrt(g);
  }
  if (unscaled) drop_rel = -drop_rel * gmax;
  std::vector<double> Gs((size_t)cols * cols, 0.0);
  for (int i = 0; i < cols; ++i)
    for (int j = 0; j < cols; ++j)
      if (d[i] > 0 && d[j] > 0) Gs[(size_t)i * cols + j] = G[(size_t)i * cols + j] / (d[i] * d[j]);
  // rank-revealing pivoted Cholesky of the scaled Gram matrix: drop directions
  // whose residual norm relative to their column is below sqrt(drop_rel)
  std::vector<int> piv;
  std::vector<double> Rs;
  const int r1 = host_pivoted_cholesky(cols, Gs.data(), drop_rel, max_rank, piv, Rs);
  if (r1 == 0) return o;
  // R11 = Rs(:, piv) is upper triangular; M1 = D^{-1} P R11^{-1} (cols x r1), T1 = Rs D (r1 x cols)
  std::vector<double> R11((size_t)r1 * r1, 0.0), R11i((size_t)r1 * r1, 0.0);
  for (int i = 0; i < r1; ++i)
    for (int k = 0; k < r1; ++k) R11[(size_t)i * r1 + k] = Rs[(size_t)i * cols + piv[k]];
  host_upper_inverse(r1, R11.data(), R11i.data());
  std::vector<double> M1((size_t)cols * r1, 0.0), T1((size_t)r1 * cols, 0.0);
  for (int k = 0; k < r1; ++k) {
    const int j = piv[k];
    for (int t = 0; t < r1; ++t) M1[(size_t)j * r1 + t] = R11i[(size_t)k * r1 + t] / d[j];
  }
  for (int t = 0; t < r1; ++t)
    for (int j = 0; j < cols; ++j) T1[(size_t)t * cols + j] = Rs[(size_t)t * cols + j] * d[j];
  if (out) {
    gemm_c<T, T>(c, n, cols, r1, 1.0, X, ldx, upload(c, M1), r1, 0.0, out, ldo);
    o.rank = r1;
    o.T = std::move(T1);
    return o;
  }
  gemm_c<T, T>(c, n, cols, r1, 1.0, X, ldx, upload(c, M1), r1, 0.0, buf, ldb);
  if (!second_pass) {
    copy2d<T, T>(n, r1, buf, ldb, 1, X, ldx, 1, 1.0, c.s);
    o.rank = r1;
    o.T = std::move(T1);
    return o;
  }
  // second pass: Cholesky QR of the (now well-conditioned) basis
  std::vector<double> G2 = gram_h<T>(c, n, r1, r1, buf, ldb, buf, ldb);
  std::vector<double> R((size_t)r1 * r1);
  if (!host_cholesky_upper(r1, G2.data(), R.data())) {
    copy2d<T, T>(n, r1, buf, ldb, 1, X, ldx, 1, 1.0, c.s);
    OrthOut o2 = orth_rr<T>(c, n, r1, X, ldx, buf, ldb, drop_rel, nullptr, false, max_rank, nullptr, 0);
    o.rank = o2.rank;
    o.T.assign((size_t)o2.rank * cols, 0.0);
    for (int i = 0; i < o2.rank; ++i)
      for (int k = 0; k < r1; ++k) {
        const double t = o2.T[(size_t)i * r1 + k];
        if (t == 0.0) continue;
        for (int j = 0; j < cols; ++j) o.T[(size_t)i * cols + j] += t * T1[(size_t)k * cols + j];
      }
    return o;
  }
  // Rinv (r1 x r1, row-major) from the column-major upper factor
  std::vector<double> Rrm((size_t)r1 * r1), Rinv((size_t)r1 * r1);
  for (int a = 0; a < r1; ++a)
    for (int b = 0; b < r1; ++b) Rrm[(size_t)a * r1 + b] = R[(size_t)b * r1 + a];
  host_upper_inverse(r1, Rrm.data(), Rinv.data());
  if (defer_rinv)
    o.Rinv = Rinv;  // basis = buf * Rinv, formed by the caller's product
  else
    gemm_c<T, T>(c, n, r1, r1, 1.0, buf, ldb, upload(c, Rinv), r1, 0.0, X, ldx);
  o.rank = r1;
  o.T.assign((size_t)r1 * cols, 0.0);
#pragma omp parallel for if ((long)r1 * r1 * cols > 1000000) schedule(dynamic, 4)
  for (int i = 0; i < r1; ++i)
    for (int k = i; k < r1; ++k) {
      const double rik = R[(size_t)k * r1 + i];
      double* oi = &o.T[(size_t)i * cols];
      const double* tk = &T1[(size_t)k * cols];
      for (int j = 0; j < cols; ++j) oi[j] += rik * tk[j];
    }
  return o;
}
template OrthOut orth_rr<float>(Ctx&, long, int, float*, int, float*, int, double, const std::vector<double>*,
                                bool, int, float*, int, bool, bool);
template OrthOut orth_rr<double>(Ctx&, long, int, double*, int, double*, int, double,
                                 const std::vector<double>*, bool, int, double*, int, bool, bool);

template <class T>
std::vector<double> cgs2(Ctx& c, long n, const T* Q, int ldq, int r, T* X, int ldx, int cols) {
  std::vector<double> C((size_t)r * cols, 0.0);
  if (r == 0 || cols == 0) return C;
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<double> Ck = gram_h<T>(c, n, r, cols, Q, ldq, X, ldx);
    gemm_c<T, T>(c, n, r, cols, -1.0, Q, ldq, upload(c, Ck), cols, 1.0, X, ldx);
    for (size_t i = 0; i < C.size(); ++i) C[i] += Ck[i];
  }
  return C;
}
template std::vector<double> cgs2<float>(Ctx&, long, const float*, int, int, float*, int, int);
template std::vector<double> cgs2<double>(Ctx&, long, const double*, int, int, double*, int, int);

// --------------------------------------------------------------- Inner ----
template <class T>
void Inner<T>::alloc(Ctx& c, int n_, int m_, int bcap_, int adicap_, int hcap_) {
  n = n_; m = m_; bcap = bcap_; adicap = adicap_; hcap = hcap_;
  jacobi = c.o.precond != CARE_PRECOND_NONE;
  const int restart = c.o.krylov == CARE_KRYLOV_GMRES
                          ? std::max(2, sizeof(T) == 4 ? c.o.gmres_restart_lo : c.o.gmres_restart_hi)
                          : 0;
  const bool ilu = c.o.precond == CARE_PRECOND_ILU0 || c.o.precond == CARE_PRECOND_ILU0_EXACT;
  kw = krylov_alloc<T>(c.ar, n, jacobi, ilu ? (long)c.op_nnz : -1L, restart);
  if (c.o.krylov == CARE_KRYLOV_DENSE_LU) dw = dlu_alloc<T>(c.ar, n);
  kw.ilu_sweeps = c.o.ilu_sweeps;
  kw.tri_sweeps = c.o.tri_sweeps;
  ldm = pad_ld<T>(std::max(m, 1));
  ldw = pad_ld<T>(std::max(bcap, 1));
  ldr = pad_ld<T>(2 * (bcap + m));
  ldz = pad_ld<T>(std::max(adicap, 1));
  ldq = pad_ld<T>(std::max(hcap, 1));
  B = c.ar.get<T>((size_t)n * ldm);
  K = c.ar.get<T>((size_t)n * ldm);
  Knew = c.ar.get<T>((size_t)n * ldm);
  Kd = c.ar.get<T>((size_t)n * ldm);
  W = c.ar.get<T>((size_t)n * ldw);
  W0 = c.ar.get<T>((size_t)n * ldw);
  RHS = c.ar.get<T>((size_t)n * ldr);
  SOL = c.ar.get<T>((size_t)n * ldr);
  Z = c.ar.get<T>((size_t)n * ldz);
  Zs = c.ar.get<T>((size_t)n * ldz);
  Q = c.ar.get<T>((size_t)n * ldq);
  FQ = c.ar.get<T>((size_t)n * ldq);
  Qt = c.ar.get<T>((size_t)n * ldq);
}
template struct Inner<float>;
template struct Inner<double>;

// precision-dependent constants of the inner solves
template <class T>
static double krylov_tol(const Ctx& c) { return sizeof(T) == 4 ? c.o.krylov_tol_lo : c.o.krylov_tol_hi; }
template <class T>
static int krylov_maxit(const Ctx& c) { return sizeof(T) == 4 ? c.o.krylov_maxit_lo : c.o.krylov_maxit_hi; }
template <class T>
static double orth_drop(void) { return sizeof(T) == 4 ? 1e-5 : 1e-12; }

// Applies F = A^T - K B^T to the n x h block X (ldq) into Y (ldq).  The SpMM
// reads and writes 16-byte vectors, so blocks starting at a column offset are
// staged through the aligned scratch blocks Qt / FQ.
template <class T>
static void apply_F(Ctx& c, Inner<T>& in, bool hasK, const T* X, T* Y, int h) {
  const bool xa = ((uintptr_t)X % 16) == 0, ya = ((uintptr_t)Y % 16) == 0;
  const T* Xs = X;
  T* Ys = Y;
  if (!xa) {
    copy2d<T, T>(in.n, h, X, in.ldq, 1, in.Qt, in.ldq, 1, 1.0, c.s);
    Xs = in.Qt;
  }
  if (!ya) Ys = in.FQ;
  CARE_REQUIRE(Ys != Xs, CARE_ERR_INVALID_ARG, "apply_F: aliasing");
  spmm<T>(op_of<T>(c), cd{0.0, 0.0}, false, Xs, in.ldq, Ys, in.ldq, h, c.s);
  if (!ya) copy2d<T, T>(in.n, h, in.FQ, in.ldq, 1, Y, in.ldq, 1, 1.0, c.s);
  c.spmm_calls++;
  if (hasK) {
    std::vector<double> BtX = gram_h<T>(c, in.n, in.m, h, in.B, in.ldm, X, in.ldq);
    gemm_c<T, T>(c, in.n, in.m, h, -1.0, in.K, in.ldm, upload(c, BtX), h, 1.0, Y, in.ldq);
  }
}

struct Shift {
  double re, im;
};

// Projection shifts (Section 5: shifts generated from Krylov subspaces):
// Ritz values of F on range(S) extended by F-blocks until at least hmin
// columns; closed right half-plane values mirrored, one value per conjugate
// pair, ordered by decreasing modulus.
template <class T>
static std::vector<Shift> proj_shifts(Ctx& c, Inner<T>& in, bool hasK, const T* S, int lds, int h0) {
  const long n = in.n;
  const int hmax = in.hcap;
  // orthonormal basis of the (at most 32) dominant directions of range(S)
  // the shift basis and the projected matrix only need Ritz values of a few digits:
  // with CARE_PREC_MIXED_TF32 / _BF16 their Grams run on the tensor cores in TF32 / BF16
  OrthOut o = orth_rr<T>(c, n, h0, const_cast<T*>(S), lds, nullptr, 0, orth_drop<T>(), nullptr, false,
                         std::min(hmax / 2, 32), in.Q, in.ldq, false, true);
  int h = o.rank;
  int last0 = 0, lastw = h;
  int ext = 0;
  while (h > 0 && h < c.o.shift_hmin && ext < 4 && h + lastw <= hmax) {
    // next Krylov block F * Q(:, last block), orthogonalised against Q
    apply_F<T>(c, in, hasK, in.Q + last0, in.Q + h, lastw);
    cgs2<T>(c, n, in.Q, in.ldq, h, in.Q + h, in.ldq, lastw);
    OrthOut ob = orth_rr<T>(c, n, lastw, in.Q + h, in.ldq, in.Qt, in.ldq, orth_drop<T>() * 1e3, nullptr,
                            false, 0, nullptr, 0);
    if (ob.rank == 0) break;
    last0 = h;
    lastw = ob.rank;
    h += ob.rank;
    ++ext;
  }
  std::vector<Shift> out;
  if (h == 0) return out;
  apply_F<T>(c, in, hasK, in.Q, in.FQ, h);
  std::vector<double> Hp = gram_h<T>(c, n, h, h, in.Q, in.ldq, in.FQ, in.ldq, true);  // row-major (Q^T F Q)
  // to column-major for the host eigenvalue routine
  std::vector<double> Hc((size_t)h * h);
  for (int i = 0; i < h; ++i)
    for (int j = 0; j < h; ++j) Hc[(size_t)j * h + i] = Hp[(size_t)i * h + j];
  std::vector<double> wr(h), wi(h);
  CARE_REQUIRE(host_eigvals(h, Hc.data(), wr.data(), wi.data()), CARE_ERR_SMALL_DENSE, "eigvals (shifts)");
  // Every Ritz value in the closed right half-plane: the projection has no stable
  // direction, so the operator (A - B K^T, stable by hypothesis of Theorem 1 and of
  // K_0 = 0) is not.  Isolated right-half-plane values are mirrored below, since a
  // stable non-normal operator can have them.
  bool any_stable = false;
  for (int i = 0; i < h; ++i) any_stable |= wr[i] < 0.0;
  CARE_REQUIRE(any_stable, CARE_UNSTABLE, "every projected Ritz value has Re >= 0");
  const double imtol = sizeof(T) == 4 ? 1e-6 : 1e-10;
  for (int i = 0; i < h; ++i) {
    const double re = wr[i], im = wi[i];
    const double mod = std::hypot(re, im);
    if (!std::isfinite(mod) || mod == 0.0) continue;
    const double rn = -std::fabs(re);
    if (rn == 0.0) continue;
    if (std::fabs(im) <= imtol * mod) out.push_back({rn, 0.0});
    else if (im > 0) out.push_back({rn, im});
  }
  std::stable_sort(out.begin(), out.end(),
                   [](const Shift& a, const Shift& b) { return std::hypot(a.re, a.im) > std::hypot(b.re, b.im); });
  return out;
}

// One chunk of a shifted solve through the batch broker (batched serving mode).
template <class T>
static KrylovResult batched_solve(Ctx& c, Inner<T>& in, const OpT<T>& op, Shift p, bool cplx, int c0, int w) {
  BatchReq<T> q;
  q.n = op.n;
  q.cols = w;
  q.cplx = cplx ? 1 : 0;
  q.rp = op.rp;
  q.ci = op.ci;
  q.av = op.val;
  q.rs = op.rowsum;
  q.diag = op.diag;
  q.sre = p.re;
  q.sim = p.im;
  q.rhs = in.RHS + c0;
  q.ld_rhs = in.ldr;
  q.sol = in.SOL + c0;
  q.ld_sol = in.ldr;
  const KrylovWork<T>& k = in.kw;
  q.X = k.X; q.R = k.R; q.Rh = k.Rh; q.P = k.P; q.V = k.V; q.S = k.S; q.Tt = k.Tt; q.Ph = k.Ph; q.Sh = k.Sh;
  CARE_REQUIRE(k.Ph && k.Sh && k.Dinv, CARE_ERR_INVALID_ARG, "batched solve: Jacobi blocks missing");
  q.Dinv = k.Dinv;
  const double tol = krylov_tol<T>(c);
  q.tol2 = tol * tol;
  q.maxit = krylov_maxit<T>(c);
  return c.broker->solve<T>(q, c.s);
}

// SMW shifted solve (Section 4):  V = M_p^{-1} W + Y (I - B^T Y)^{-1} B^T M_p^{-1} W,
// Y = M_p^{-1} K, M_p = (A + p I)^T.  W: first b columns of in.W (real).
// On return V occupies the first b (complex: 2b real) columns of in.SOL.
template <class T>
static void smw_solve(Ctx& c, Inner<T>& in, Shift p, int b, bool hasK) {
  const long n = in.n;
  const bool cplx = p.im != 0.0;
  const int m = hasK ? in.m : 0;
  const int ncol = b + m;
  const int rc = cplx ? 2 * ncol : ncol;  // real columns of RHS / SOL
  if (cplx) {
    CARE_CUDA(cudaMemsetAsync(in.RHS, 0, (size_t)n * in.ldr * sizeof(T), c.s));
    copy2d<T, T>(n, b, in.W, in.ldw, 1, in.RHS, in.ldr, 2, 1.0, c.s);
    if (m) copy2d<T, T>(n, m, in.K, in.ldm, 1, in.RHS + 2 * b, in.ldr, 2, 1.0, c.s);
  } else {
    copy2d<T, T>(n, b, in.W, in.ldw, 1, in.RHS, in.ldr, 1, 1.0, c.s);
    if (m) copy2d<T, T>(n, m, in.K, in.ldm, 1, in.RHS + b, in.ldr, 1, 1.0, c.s);
  }
  const OpT<T> op = op_of<T>(c);
  const bool dense = c.o.krylov == CARE_KRYLOV_DENSE_LU;  // one factorisation serves every column
  const int chunk =
      dense ? rc : std::min(kMaxRealCols, std::max(2, (c.o.krylov_chunk > 0 ? c.o.krylov_chunk : 64) * (cplx ? 2 : 1)));
  for (int c0 = 0; c0 < rc; c0 += chunk) {
    const int w = std::min(chunk, rc - c0);
    if (!c.ke0) {
      CARE_CUDA(cudaEventCreate(&c.ke0));
      CARE_CUDA(cudaEventCreate(&c.ke1));
    }
    CARE_CUDA(cudaEventRecord(c.ke0, c.s));
    KrylovResult kr =
        c.broker ? batched_solve<T>(c, in, op, p, cplx, c0, w)
        : dense ? dense_lu_solve<T>(c.op, cd{p.re, p.im}, cplx, in.RHS + c0, in.ldr, in.SOL + c0, in.ldr, w, in.dw, c.s)
        : c.o.krylov == CARE_KRYLOV_GMRES
            ? krylov_gmres<T>(op, cd{p.re, p.im}, cplx, in.RHS + c0, in.ldr, in.SOL + c0, in.ldr, w,
                              krylov_tol<T>(c), krylov_maxit<T>(c), c.o.precond, in.kw, c.s)
            : krylov_bicgstab<T>(op, cd{p.re, p.im}, cplx, in.RHS + c0, in.ldr, in.SOL + c0, in.ldr, w,
                                 krylov_tol<T>(c), krylov_maxit<T>(c), c.o.precond, in.kw, c.s);
    CARE_CUDA(cudaEventRecord(c.ke1, c.s));
    CARE_CUDA(cudaEventSynchronize(c.ke1));  // the solve has synchronised already
    float kms = 0.f;
    CARE_CUDA(cudaEventElapsedTime(&kms, c.ke0, c.ke1));
    c.kry_ms += kms;
    c.kry_gbyte += kr.bytes * 1e-9;
    c.host_syncs += 2 + kr.iters / 4;
    c.krylov_iters += kr.iters;
    c.spmm_calls += kr.spmm;
    if (kr.unconverged) c.krylov_unconverged++;
  }
  if (!m) return;
  // capacitance: BtS (m x rc) = B^T [V0 | Y]
  std::vector<double> BtS = gram_h<T>(c, n, m, rc, in.B, in.ldm, in.SOL, in.ldr);
  auto bts = [&](int i, int j) -> cd {  // complex entry (i, j) of B^T SOL
    if (cplx) return cd{BtS[(size_t)i * rc + 2 * j], BtS[(size_t)i * rc + 2 * j + 1]};
    return cd{BtS[(size_t)i * rc + j], 0.0};
  };
  std::vector<cd> S((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      cd y = bts(i, b + j);
      S[(size_t)j * m + i] = cd{(i == j ? 1.0 : 0.0) - y.re, -y.im};
    }
  std::vector<cd> Tm((size_t)m * b);  // column-major m x b: B^T V0, overwritten by S^{-1} B^T V0
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < b; ++j) Tm[(size_t)j * m + i] = bts(i, j);
  CARE_REQUIRE(host_lu_solve_complex(m, S, Tm.data(), b), CARE_ERR_SMALL_DENSE, "SMW capacitance solve");
  // V0 += Y Tm
  if (cplx) {
    std::vector<double> E((size_t)(2 * m) * (2 * b));
    for (int k = 0; k < m; ++k)
      for (int j = 0; j < b; ++j) {
        const cd t = Tm[(size_t)j * m + k];
        E[(size_t)(2 * k) * (2 * b) + 2 * j] = t.re;
        E[(size_t)(2 * k) * (2 * b) + 2 * j + 1] = t.im;
        E[(size_t)(2 * k + 1) * (2 * b) + 2 * j] = -t.im;
        E[(size_t)(2 * k + 1) * (2 * b) + 2 * j + 1] = t.re;
      }
    gemm_c<T, T>(c, n, 2 * m, 2 * b, 1.0, in.SOL + 2 * b, in.ldr, upload(c, E), 2 * b, 1.0, in.SOL, in.ldr);
  } else {
    std::vector<double> E((size_t)m * b);
    for (int k = 0; k < m; ++k)
      for (int j = 0; j < b; ++j) E[(size_t)k * b + j] = Tm[(size_t)j * m + k].re;
    gemm_c<T, T>(c, n, m, b, 1.0, in.SOL + b, in.ldr, upload(c, E), b, 1.0, in.SOL, in.ldr);
  }
}

template <class T>
void smw_solve_public(Ctx& c, Inner<T>& in, double p_re, double p_im, int b, bool hasK) {
  smw_solve<T>(c, in, Shift{p_re, p_im}, b, hasK);
}
template void smw_solve_public<float>(Ctx&, Inner<float>&, double, double, int, bool);
template void smw_solve_public<double>(Ctx&, Inner<double>&, double, double, int, bool);

template <class T>
static double adi_norm2(Ctx& c, Inner<T>& in, int b) {
  // ||W^T W||_2 = largest eigenvalue of the b x b Gram matrix
  std::vector<double> G = gram_h<T>(c, in.n, b, b, in.W, in.ldw, in.W, in.ldw);
  const double l = host_sym_lmax(b, G.data());
  CARE_REQUIRE(std::isfinite(l), CARE_ERR_SMALL_DENSE, "largest eigenvalue (ADI norm)");
  return std::max(l, 0.0);
}

// Compresses the factor columns Z[:, col0 : col0 + ncols] (one sign group) to
// rank q: Z = Q T (rank-revealing orthonormalisation) and Z Z^T = Q (T T^T) Q^T
// = (Q L)(Q L)^T with L L^T = T T^T, written right- or left-aligned in place.
template <class T>
static int compress_part(Ctx& c, Inner<T>& in, int col0, int ncols, bool right_aligned) {
  if (ncols == 0) return 0;
  const long n = in.n;
  // unscaled truncation at the accuracy of the inner precision u_s: directions
  // whose residual column norm^2 is below (a few u_s) times the largest column
  // norm^2 carry less than that fraction of X_+- and are below what the inner
  // solve determines (the inner backward error is O(u_s), Assumption 2)
  const double drop = sizeof(T) == 4 ? -2.0e-7 : -1.0e-15;
  OrthOut o = orth_rr<T>(c, n, ncols, in.Z + col0, in.ldz, in.Zs, in.ldz, drop, nullptr, true, 0, nullptr, 0);
  const int q = o.rank;
  if (q == 0) return 0;
  std::vector<double> TT((size_t)q * q, 0.0), R((size_t)q * q);
  host_gemm_nt(q, q, ncols, o.T.data(), ncols, o.T.data(), ncols, nullptr, TT.data(), q, true);
  CARE_REQUIRE(host_cholesky_upper(q, TT.data(), R.data()), CARE_ERR_SMALL_DENSE, "compression Cholesky");
  // column-major upper R == row-major R^T = L
  gemm_c<T, T>(c, n, q, q, 1.0, in.Z + col0, in.ldz, upload(c, R), q, 0.0, in.Zs, in.ldz);
  const int dst = right_aligned ? col0 + ncols - q : col0;
  copy2d<T, T>(n, q, in.Zs, in.ldz, 1, in.Z + dst, in.ldz, 1, 1.0, c.s);
  return q;
}

// Joint compression of the two factor groups when their capacity is reached:
// X_+ - X_- = [Z_+, Z_-] N [Z_+, Z_-]^T, N = diag(I, -I), is what the refinement
// uses, and X_+, X_- are each much larger than their difference near convergence.
// The groups are widened to FP64, orthonormalised together ([Z_+, Z_-] = Q T),
// P = T N T^T is diagonalised on the device, eigenvalues below the inner
// precision's relative level (1e-8 of max|lambda| for FP32, 1e-15 for FP64) are
// dropped, and the positive / negative parts Q V_+- |Lambda_+-|^{1/2} replace the
// groups.  The truncation is then relative to the correction itself, not to X_+-.
// Returns false (nothing changed) when the FP64 blocks are too narrow.
template <class T>
static bool compress_joint(Ctx& c, Inner<T>& in, int& np, int& nm) {
  const int ny = np + nm;
  if (!in.f64a || ny > in.f64cap || ny == 0 || !c.dsm) return false;
  const long n = in.n;
  const int cap = in.adicap;
  if (np) copy2d<T, double>(n, np, in.Z, in.ldz, 1, in.f64a, in.f64ld, 1, 1.0, c.s);
  if (nm) copy2d<T, double>(n, nm, in.Z + (cap - nm), in.ldz, 1, in.f64a + np, in.f64ld, 1, 1.0, c.s);
  OrthOut O = orth_rr<double>(c, n, ny, in.f64a, in.f64ld, in.f64b, in.f64ld, 1e-14, nullptr, true, 0, nullptr, 0);
  const int q = O.rank;
  if (q == 0) {
    np = nm = 0;
    return true;
  }
  std::vector<double> TNt((size_t)ny * q);
  for (int i = 0; i < q; ++i)
    for (int j = 0; j < ny; ++j) TNt[(size_t)j * q + i] = O.T[(size_t)i * ny + j] * (j < np ? 1.0 : -1.0);
  DevSmall ds{c.dsm, c.dsm_cap, 0};
  double* Pd = dev_small_product(c, ds, q, ny, O.T, TNt);
  const size_t ew = dev_symeig_work_elems(q);
  double* ework = ds.get(ew);
  double* Vd = ds.get((size_t)q * q);
  const double rel = sizeof(T) == 4 ? 1e-8 : 1e-15;
  std::vector<double> lam;
  // The compressed FP32 factors carry each vector weighted by |lambda|^(1/2) and are only
  // FP32-accurate: weighted clustering, which splits the long run of small kept
  // eigenvalues into separate clusters.  FP64 factors keep the strict clustering.
  std::vector<int> sel = dev_symeig_select(
      q, Pd, q, lam, Vd, [rel](double l, double lmx) { return std::fabs(l) >= rel * lmx && l != 0.0; }, ework, ew,
      c.s, sizeof(T) == 4);
  c.host_syncs += 3;
  std::vector<int> pos(q, -1);
  for (int t = 0; t < (int)sel.size(); ++t) pos[sel[t]] = t;
  std::vector<int> qi;
  std::vector<double> sc;
  int rp2 = 0;
  for (int t = q - 1; t >= 0; --t)
    if (pos[t] >= 0 && lam[t] > 0) {
      qi.push_back(pos[t]);
      sc.push_back(std::sqrt(lam[t]));
      ++rp2;
    }
  for (int t = 0; t < q; ++t)
    if (pos[t] >= 0 && lam[t] < 0) {
      qi.push_back(pos[t]);
      sc.push_back(std::sqrt(-lam[t]));
    }
  const int cw = (int)qi.size(), rm2 = cw - rp2;
  double* S = ds.get((size_t)q * std::max(cw, 1));
  eig_coeffs(c, ds, q, cw, Vd, q, qi, sc, S);
  if (rp2) gemm_c<double, T>(c, n, q, rp2, 1.0, in.f64a, in.f64ld, S, cw, 0.0, in.Z, in.ldz);
  if (rm2) gemm_c<double, T>(c, n, q, rm2, 1.0, in.f64a, in.f64ld, S + rp2, cw, 0.0, in.Z + (cap - rm2), in.ldz);
  np = rp2;
  nm = rm2;
  return true;
}

template <class T>
AdiResult lradi(Ctx& c, Inner<T>& in, int b, int rp, bool hasK, double tol, int jmax, bool knew,
                int compress_end) {
  AdiResult res;
  const long n = in.n;
  const int rm = b - rp;
  CARE_REQUIRE(b <= in.bcap, CARE_ERR_RANK_CAPACITY, "LR-ADI right-hand side wider than its capacity");
  CARE_REQUIRE(rp >= 0 && rm >= 0 && (!knew || rm == 0), CARE_ERR_INVALID_ARG, "LR-ADI split");
  copy2d<T, T>(n, b, in.W0, in.ldw, 1, in.W, in.ldw, 1, 1.0, c.s);
  const double w0 = adi_norm2<T>(c, in, b);
  if (!(w0 > 0.0)) {
    res.converged = true;
    return res;
  }
  std::vector<Shift> shifts = proj_shifts<T>(c, in, hasK, in.W, in.ldw, b);
  size_t next = 0;
  int np = 0, nm = 0, j = 0;
  int last0 = -1, lastw = 0;
  double r = 1.0;
  const int cap = in.adicap;
  while (j < jmax && r > tol) {
    if (next >= shifts.size()) {
      shifts = last0 >= 0 ? proj_shifts<T>(c, in, hasK, in.Z + last0, in.ldz, lastw)
                          : proj_shifts<T>(c, in, hasK, in.W, in.ldw, b);
      next = 0;
      CARE_REQUIRE(!shifts.empty(), CARE_INNER_FAILED, "no shifts available");
    }
    const Shift p = shifts[next];
    const bool cplx = p.im != 0.0;
    const int mult = cplx ? 2 : 1;
    if (np + nm + mult * b > cap) {
      // column compression: jointly in FP64 where the session has the blocks (the
      // correction solves of care_solve), else each sign group on its own
      int np2 = np, nm2 = nm;
      if (!compress_joint<T>(c, in, np2, nm2)) {
        np2 = compress_part<T>(c, in, 0, np, false);
        nm2 = compress_part<T>(c, in, cap - nm, nm, true);
      }
      if (verbose_level() >= 2)
        fprintf(stderr, "[care]   adi compress %d+%d -> %d+%d\n", np, nm, np2, nm2);
      np = np2;
      nm = nm2;
      res.compressions++;
      last0 = -1;  // the newest block was merged; shifts restart from the residual
      if (np + nm + mult * b > cap) break;  // capacity exhausted: inexact inner solve
    }
    ++next;
    smw_solve<T>(c, in, p, b, hasK);
    const int pm0 = cap - nm - mult * rm;  // start of the new minus columns
    if (!cplx) {
      // W <- W - 2 p V;  Z <- [Z, sqrt(-2p) V]
      const double sc = std::sqrt(-2.0 * p.re);
      axpby<T>(n, b, -2.0 * p.re, in.SOL, in.ldr, 1.0, in.W, in.ldw, c.s);
      if (rp) copy2d<T, T>(n, rp, in.SOL, in.ldr, 1, in.Z + np, in.ldz, 1, sc, c.s);
      if (rm) copy2d<T, T>(n, rm, in.SOL + rp, in.ldr, 1, in.Z + pm0, in.ldz, 1, sc, c.s);
      j += 1;
    } else {
      // complex pair p, conj(p) in real arithmetic:
      // W <- W + g^2 (Re V + d Im V);  Z <- [Z, g (Re V + d Im V), g sqrt(d^2+1) Im V]
      const double g = 2.0 * std::sqrt(-p.re), d = p.re / p.im;
      const double gi = g * std::sqrt(d * d + 1.0);
      cpair_update<T>(n, b, rp, in.SOL, in.ldr, g, d, gi, in.W, in.ldw, in.Z + np, in.Z + pm0, in.ldz, c.s);
      j += 2;
    }
    if (knew) {
      // K_new += Z_blk (Z_blk^T B)
      const int add = mult * rp;
      std::vector<double> ZtB = gram_h<T>(c, n, add, in.m, in.Z + np, in.ldz, in.B, in.ldm);
      gemm_c<T, T>(c, n, add, in.m, 1.0, in.Z + np, in.ldz, upload(c, ZtB), in.m, 1.0, in.Knew, in.ldm);
    }
    if (rp) {
      last0 = np;
      lastw = mult * rp;
    } else {
      last0 = pm0;
      lastw = mult * rm;
    }
    np += mult * rp;
    nm += mult * rm;
    r = adi_norm2<T>(c, in, b) / w0;
    if (!std::isfinite(r)) CARE_THROW(CARE_NONFINITE, "LR-ADI residual not finite");
    // with left half-plane shifts the residual factor of a stable operator does not
    // grow by orders of magnitude; growth beyond 1e12 means the operator is unstable
    CARE_REQUIRE(r <= 1e12, CARE_UNSTABLE, "LR-ADI residual diverges");
    if (verbose_level() >= 2)
      fprintf(stderr, "[care]   adi j=%d p=(%.4e,%.4e) res=%.3e cols=%d+%d\n", j, p.re, p.im, r, np, nm);
  }
  // compress_end 1: each sign group on its own, only wide factors (below a few
  // hundred columns Algorithm 2's FP64 rank revealing is cheap and keeps the full
  // accuracy of X_+ - X_-).  2: the joint indefinite FP64 compression of X_+ - X_-,
  // truncated relative to the correction itself, whenever the factor is wider than
  // the right-hand side (it also drops the inner-precision noise directions that a
  // Gram-based QR in Algorithm 2 cannot resolve); each sign group on its own where
  // the session has no FP64 blocks.
  if (compress_end == 2 && np + nm > b) {
    int np2 = np, nm2 = nm;
    if (!compress_joint<T>(c, in, np2, nm2)) {
      np2 = compress_part<T>(c, in, 0, np, false);
      nm2 = compress_part<T>(c, in, cap - nm, nm, true);
    }
    np = np2;
    nm = nm2;
    res.compressions++;
  } else if (compress_end == 1 && np + nm > std::max(2 * b, 512)) {
    np = compress_part<T>(c, in, 0, np, false);
    nm = compress_part<T>(c, in, cap - nm, nm, true);
    res.compressions++;
  }
  res.np = np;
  res.nm = nm;
  res.steps = j;
  res.res = r;
  res.converged = r <= tol;
  if (verbose_level() >= 1)
    fprintf(stderr, "[care]  lradi b=%d (%d+%d) steps=%d res=%.3e cols=%d+%d compress=%d krylov_unconv=%d\n", b, rp, rm,
            j, r, np, nm, res.compressions, c.krylov_unconverged);
  return res;
}
template AdiResult lradi<float>(Ctx&, Inner<float>&, int, int, bool, double, int, bool, int);
template AdiResult lradi<double>(Ctx&, Inner<double>&, int, int, bool, double, int, bool, int);

template <class T>
NlrResult nlradi(Ctx& c, Inner<T>& in, const T* Ct, int ldct, int p, double tol_lyap, double tol_newton,
                 int newton_max, int jmax) {
  NlrResult out;
  const long n = in.n;
  bool hasK = false;
  double prev_rel = -1.0;
  CARE_CUDA(cudaMemsetAsync(in.K, 0, (size_t)n * in.ldm * sizeof(T), c.s));
  for (int i = 0; i < newton_max; ++i) {
    // right-hand side factor [C^T, K_i] (K_0 = 0: C^T only)
    copy2d<T, T>(n, p, Ct, ldct, 1, in.W0, in.ldw, 1, 1.0, c.s);
    int b = p;
    if (hasK) {
      copy2d<T, T>(n, in.m, in.K, in.ldm, 1, in.W0 + p, in.ldw, 1, 1.0, c.s);
      b += in.m;
    }
    CARE_CUDA(cudaMemsetAsync(in.Knew, 0, (size_t)n * in.ldm * sizeof(T), c.s));
    AdiResult a = lradi<T>(c, in, b, b, hasK, tol_lyap, jmax, true, 0);
    out.adi += a.steps;
    out.newton = i + 1;
    out.cols = a.np;
    // relative change of the feedback
    axpby<T>(n, in.m, 1.0, in.Knew, in.ldm, 0.0, in.Kd, in.ldm, c.s);
    axpby<T>(n, in.m, -1.0, in.K, in.ldm, 1.0, in.Kd, in.ldm, c.s);
    std::vector<double> Gd = gram_h<T>(c, n, in.m, in.m, in.Kd, in.ldm, in.Kd, in.ldm);
    std::vector<double> Gk = gram_h<T>(c, n, in.m, in.m, in.Knew, in.ldm, in.Knew, in.ldm);
    double dk = 0.0, nk = 0.0;
    for (int q = 0; q < in.m; ++q) {
      dk += Gd[(size_t)q * in.m + q];
      nk += Gk[(size_t)q * in.m + q];
    }
    const double rel = nk > 0 ? std::sqrt(dk / nk) : 0.0;
    std::swap(in.K, in.Knew);
    hasK = true;
    if (verbose_level() >= 1)
      fprintf(stderr, "[care] nlradi newton=%d adi=%d cols=%d dK=%.3e adires=%.3e\n", i + 1, a.steps, a.np,
              rel, a.res);
    if (!std::isfinite(rel)) CARE_THROW(CARE_NONFINITE, "NLR-ADI feedback not finite");
    if (rel <= tol_newton) {
      out.converged = true;
      break;
    }
    // Newton has reached the accuracy of its inner solves once the change stops
    // shrinking quadratically: further steps only add rounding noise
    if (prev_rel > 0 && rel < 1e-3 && rel > 0.5 * prev_rel) break;
    prev_rel = rel;
  }
  return out;
}
template NlrResult nlradi<float>(Ctx&, Inner<float>&, const float*, int, int, double, double, int, int);
template NlrResult nlradi<double>(Ctx&, Inner<double>&, const double*, int, int, double, double, int, int);

}  // namespace care
