// Tensor-core (tcgen05 + TMA) products: FP64-accurate sliced products and
// TF32 / BF16 products of the tall-skinny contractions (see tc.cuh).
#include <cuda_bf16.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "tc.cuh"

namespace care {
namespace {

constexpr int BM = 128;          // output rows per tile (TMEM lanes)
constexpr int BN = 64;           // output columns per tile (accumulator columns)
constexpr int ROWB = 64;         // bytes per staged operand row (64-byte swizzle)
constexpr int NSLICE = 8;        // slices of an FP64 operand
constexpr int CHUNK = 128;       // K-rows between exact flushes (FP64 mode)
constexpr int SLAB = 32768;      // K-rows (Gram) / output rows (X S) per slicing pass
constexpr int EPI_WARPS = 8;
constexpr int TC_THREADS = (EPI_WARPS + 2) * 32;
constexpr int PRODUCER_WARP = EPI_WARPS;
constexpr int MMA_WARP = EPI_WARPS + 1;
constexpr long long WAIT_NS = 2000000000LL;  // bound on any single mbarrier wait (2 s)

// error codes written to the device error word
constexpr int ERR_WAIT_FULL = 1, ERR_WAIT_EMPTY = 2, ERR_WAIT_ACC = 3, ERR_WAIT_ACCE = 4;

// ---- slice pairs of the sliced modes --------------------------------------------
// FP64 mode: pairs (a, b) with a + b <= 8 of 8 slices.  Tail pairs (a + b >= 5,
// accumulator 5) come first within every K-step so that the MMAs of a new chunk
// can start while the epilogue still drains the exact groups of the previous one;
// the exact pairs follow, grouped by a + b (accumulator a + b).
// FP32 mode: pairs with a + b <= 3 of 4 slices, all exact (accumulator a + b).
struct PairTable {
  int n;
  int a[48], b[48], acc[48], first[48];
};
constexpr PairTable make_pairs(int nsl, int smax, int sexact) {
  PairTable t{};
  int k = 0;
  for (int s = sexact + 1; s <= smax; ++s)
    for (int a = 0; a < nsl; ++a) {
      const int b = s - a;
      if (b < 0 || b >= nsl) continue;
      t.a[k] = a; t.b[k] = b; t.acc[k] = sexact + 1; t.first[k] = (k == 0); ++k;
    }
  for (int s = 0; s <= sexact && s <= smax; ++s)
    for (int a = 0; a <= s; ++a) {
      if (a >= nsl || s - a >= nsl) continue;
      t.a[k] = a; t.b[k] = s - a; t.acc[k] = s; t.first[k] = (a == 0); ++k;
    }
  t.n = k;
  return t;
}
constexpr PairTable kPairs64 = make_pairs(NSLICE, 8, 4);
constexpr PairTable kPairs32 = make_pairs(4, 3, 3);
static_assert(kPairs64.n == 43 && kPairs64.acc[28] == 0 && kPairs64.acc[27] == 5, "FP64 pairs");
static_assert(kPairs32.n == 10 && kPairs32.acc[0] == 0 && kPairs32.acc[9] == 3, "FP32 pairs");
// device copies (constant bank; the MMA loop indexes them with unrolled constants)
__constant__ PairTable c_pairs64 = make_pairs(NSLICE, 8, 4);
__constant__ PairTable c_pairs32 = make_pairs(4, 3, 3);
template <int MODE>
__device__ __forceinline__ int pair_field(int p, int f) {
  if constexpr (MODE == 0)
    return f == 0 ? c_pairs64.a[p] : f == 1 ? c_pairs64.b[p] : f == 2 ? c_pairs64.acc[p] : c_pairs64.first[p];
  else
    return f == 0 ? c_pairs32.a[p] : f == 1 ? c_pairs32.b[p] : f == 2 ? c_pairs32.acc[p] : c_pairs32.first[p];
}

// ---- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ long long gtimer() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait for the phase of parity `parity` to complete.  Gives up when the
// CTA's abort flag is set or after WAIT_NS, recording `code` in the error word.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = gtimer();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > WAIT_NS) {
      *abort_flag = 1;
      atomicCAS(err, 0, code);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(su32(dst)),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(su32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// K-major operand tile with 64-byte rows and the 64-byte swizzle: 8-row groups
// 512 bytes apart (stride byte offset), leading byte offset unused (16 B).
__device__ __forceinline__ uint64_t desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(512 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)4 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format fmt (1 BF16, 2 TF32),
// both K-major, M = 128, N = BN.
__host__ __device__ constexpr uint32_t idesc_of(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void umma(uint32_t dtm, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accum) {
  if constexpr (TF32)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
            "r"(dtm),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// ties the loaded registers to a point after tcgen05.wait::ld
__device__ __forceinline__ void reg_fence8(uint32_t (&r)[8]) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}

// exact FP32 integer (|w| < 2^22) to int32 by the 1.5 * 2^23 bias
__device__ __forceinline__ int f2i_exact(float w) { return __float_as_int(w + 12582912.0f) - 0x4B400000; }

// ---- the product kernel ---------------------------------------------------------
struct TcArgs {
  int M, N;          // valid output rows (rows of A) and columns (rows of B)
  int k_len;         // valid K of the operand maps
  int k_per_split;   // K per CTA (multiple of CHUNK)
  int tiles_m;       // tiles along M
  int sym;           // only tiles reaching the diagonal or above
  int out_mode;      // 0: FP64 partial tile store; 1: Y = alpha v + beta Y
  double* part;      // out_mode 0: part[split][M][N]
  const int* ea;     // row exponents of A (FP64 mode)
  const int* eb;     // row exponents of B
  void* Y;           // out_mode 1
  long ldy;
  int y_f32;
  double alpha, beta;
  int* err;
  int starve;        // test hook: issue no copies (the first wait then expires)
};

// MODE 0: FP64-accurate slices (8 BF16 slices, 43 pairs, 5 exact groups + tail);
// 1: TF32 (kind::tf32, FP32 operands); 2: BF16 (kind::f16, one BF16 slice);
// 3: FP32-accurate slices (4 BF16 slices, 10 pairs, all in 4 exact groups).
template <int MODE>
struct TcCfg {
  static constexpr bool SLICED = MODE == 0 || MODE == 3;
  static constexpr int NSL = MODE == 0 ? NSLICE : (MODE == 3 ? 4 : 1);
  static constexpr int NPAIR = MODE == 0 ? 43 : 10;
  static constexpr int FIRST_EXACT = MODE == 0 ? 28 : 0;
  static constexpr int NEXACT = MODE == 0 ? 5 : 4;      // exact accumulators 0 .. NEXACT-1
  static constexpr bool TAIL = MODE == 0;               // accumulator NEXACT holds the tail
  static constexpr int STAGES = MODE == 0 ? 2 : (MODE == 3 ? 4 : 8);
  static constexpr int ESZ = MODE == 1 ? 4 : 2;
  static constexpr int KEL = ROWB / ESZ;            // K elements per stage
  static constexpr int KSTEP = 32 / ESZ;            // K elements per MMA (32 bytes)
  static constexpr int A_BYTES = BM * ROWB;
  static constexpr int B_BYTES = BN * ROWB;
  static constexpr int STAGE_BYTES = NSL * (A_BYTES + B_BYTES);
  static constexpr uint32_t TCOLS = MODE == 0 ? 512 : (MODE == 3 ? 256 : 64);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
};

template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, TcArgs g) {
  using C = TcCfg<MODE>;
  constexpr bool TF32 = MODE == 1;
  const int tile = blockIdx.x, split = blockIdx.y;
  const int ti = tile % g.tiles_m, tj = tile / g.tiles_m;
  const int row0 = ti * BM, col0 = tj * BN;
  if (g.sym && col0 + BN - 1 < row0) return;  // whole tile below the diagonal (uniform per CTA)
  const int kbeg = split * g.k_per_split;
  const int kend = min(g.k_len, kbeg + g.k_per_split);
  const int nst = (kend - kbeg + C::KEL - 1) / C::KEL;  // stages (>= 1: every split has K)
  constexpr int SPC = C::SLICED ? CHUNK / C::KEL : 1 << 30;
  const int nchunks = C::SLICED ? (nst + SPC - 1) / SPC : 1;

  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::STAGES * C::STAGE_BYTES);
  uint64_t* full = bars;
  uint64_t* empty = bars + C::STAGES;
  uint64_t* accf = bars + 2 * C::STAGES;
  uint64_t* acce = accf + 1;
  uint64_t* drain = acce + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(accf, 1);
    mbar_init(acce, EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(C::TCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tmem_slot;

  if (warp == PRODUCER_WARP) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mB) : "memory");
      int stage = 0;
      uint32_t eph = 1;
      int issued = 0;
      uint32_t last_par[C::STAGES];
      for (int s = 0; s < C::STAGES; ++s) last_par[s] = 0;
      for (int it = 0; it < nst && !g.starve; ++it) {
        if (!mbar_wait(empty + stage, eph, abort_flag, g.err, ERR_WAIT_EMPTY)) break;
        mbar_arrive_tx(full + stage, C::STAGE_BYTES);
        uint8_t* st = sm + stage * C::STAGE_BYTES;
        const int kx = kbeg + it * C::KEL;
#pragma unroll
        for (int a = 0; a < C::NSL; ++a) tma_load3(st + a * C::A_BYTES, &mA, full + stage, kx, row0, a);
#pragma unroll
        for (int b = 0; b < C::NSL; ++b)
          tma_load3(st + C::NSL * C::A_BYTES + b * C::B_BYTES, &mB, full + stage, kx, col0, b);
        last_par[stage] = (uint32_t)((it / C::STAGES) & 1);
        ++issued;
        if (++stage == C::STAGES) {
          stage = 0;
          eph ^= 1;
        }
      }
      if (*abort_flag) {
        // drain the copies in flight before the CTA exits (bounded)
        for (int s = 0; s < C::STAGES && s < issued; ++s) {
          const long long t0 = gtimer();
          while (!mbar_try(full + s, last_par[s]) && gtimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_of(MODE == 1 ? 2u : 1u);
      int stage = 0;
      uint32_t fph = 0, aeph = 0;
      bool ok = true;
      for (int c = 0; c < nchunks && ok; ++c) {
        for (int st = 0; st < SPC; ++st) {
          const int it = c * SPC + st;
          if (it >= nst) break;
          if (!mbar_wait(full + stage, fph, abort_flag, g.err, ERR_WAIT_FULL)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(sm + stage * C::STAGE_BYTES);
          const uint32_t sb = sa + C::NSL * C::A_BYTES;
#pragma unroll
          for (int kk = 0; kk < C::KEL / C::KSTEP; ++kk) {
            if constexpr (C::SLICED) {
#pragma unroll
              for (int p = 0; p < C::NPAIR; ++p) {
                if (p == C::FIRST_EXACT && c > 0 && st == 0 && kk == 0) {
                  // the epilogue must have read the previous chunk's exact groups
                  if (!mbar_wait(acce, aeph, abort_flag, g.err, ERR_WAIT_ACCE)) {
                    ok = false;
                    break;
                  }
                  aeph ^= 1;
                  tc_fence_after();
                }
                const int pa = pair_field<MODE>(p, 0), pbb = pair_field<MODE>(p, 1);
                const int pacc = pair_field<MODE>(p, 2), pfirst = pair_field<MODE>(p, 3);
                const bool exact = pacc < C::NEXACT;
                const bool fresh = pfirst && kk == 0 && st == 0 && (exact || c == 0);
                umma<false>(tbase + (uint32_t)(pacc * BN), desc_sw64(sa + pa * C::A_BYTES + kk * 32),
                            desc_sw64(sb + pbb * C::B_BYTES + kk * 32), idesc, fresh ? 0u : 1u);
              }
              if (!ok) break;
            } else {
              umma<TF32>(tbase, desc_sw64(sa + kk * 32), desc_sw64(sb + kk * 32), idesc,
                         (it == 0 && kk == 0) ? 0u : 1u);
            }
          }
          if (!ok) break;
          umma_commit(empty + stage);  // frees the stage once these MMAs have read it
          if (++stage == C::STAGES) {
            stage = 0;
            fph ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(accf);  // chunk complete: the epilogue may read the accumulators
      }
      if (!ok) {
        // let the products already issued finish before TMEM is released (bounded)
        umma_commit(drain);
        const long long t0 = gtimer();
        while (!mbar_try(drain, 0) && gtimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else {
    // ---- epilogue warps: lane quadrant q, 32-column half h ----
    const int q = warp & 3, h = warp >> 2;
    const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(h * 32);
    long long acc[32];
    float tail[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      acc[j] = 0;
      tail[j] = 0.f;
    }
    uint32_t afph = 0;
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
      // warp-uniform decision: the TMEM loads below are warp-collective
      const bool got = mbar_wait(accf, afph, abort_flag, g.err, ERR_WAIT_ACC);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      afph ^= 1;
      tc_fence_after();
      const bool last = c == nchunks - 1;
      if constexpr (C::SLICED) {
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {
          uint32_t v0[8], v1[8], v2[8], v3[8], v4[8];
          tmem_ld8(tl + 0 * BN + sub * 8, v0);
          tmem_ld8(tl + 1 * BN + sub * 8, v1);
          tmem_ld8(tl + 2 * BN + sub * 8, v2);
          tmem_ld8(tl + 3 * BN + sub * 8, v3);
          if constexpr (C::NEXACT > 4) tmem_ld8(tl + 4 * BN + sub * 8, v4);
          tmem_wait_ld();
          reg_fence8(v0); reg_fence8(v1); reg_fence8(v2); reg_fence8(v3);
          if constexpr (C::NEXACT > 4) reg_fence8(v4);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // group s holds an integer times 2^-7(s+2)
            const int g0 = f2i_exact(__uint_as_float(v0[j]) * 16384.0f);             // 2^14
            const int g1 = f2i_exact(__uint_as_float(v1[j]) * 2097152.0f);           // 2^21
            const int g2 = f2i_exact(__uint_as_float(v2[j]) * 268435456.0f);         // 2^28
            const int g3 = f2i_exact(__uint_as_float(v3[j]) * 34359738368.0f);       // 2^35
            if constexpr (C::NEXACT > 4) {
              const int g4 = f2i_exact(__uint_as_float(v4[j]) * 4398046511104.0f);   // 2^42
              // units of 2^-42
              acc[sub * 8 + j] += (long long)g0 * (1LL << 28) + (long long)(g1 * 128 + g2) * (1LL << 14) +
                                  (long long)(g3 * 128 + g4);
            } else {
              // units of 2^-35
              acc[sub * 8 + j] += (long long)g0 * (1LL << 21) + (long long)(g1 * 128 + g2) * (1LL << 7) +
                                  (long long)g3;
            }
          }
        }
        if (C::TAIL && last) {
#pragma unroll
          for (int sub = 0; sub < 4; ++sub) {
            uint32_t t[8];
            tmem_ld8(tl + C::NEXACT * BN + sub * 8, t);
            tmem_wait_ld();
            reg_fence8(t);
#pragma unroll
            for (int j = 0; j < 8; ++j) tail[sub * 8 + j] = __uint_as_float(t[j]);
          }
        }
      } else {
#pragma unroll
        for (int sub = 0; sub < 4; ++sub) {
          uint32_t t[8];
          tmem_ld8(tl + sub * 8, t);
          tmem_wait_ld();
          reg_fence8(t);
#pragma unroll
          for (int j = 0; j < 8; ++j) tail[sub * 8 + j] = __uint_as_float(t[j]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (C::SLICED && !last && lane == 0) mbar_arrive(acce);
    }
    if (ok) {
      const int row = row0 + q * 32 + lane;
      if (row < g.M) {
        const int er = g.ea ? g.ea[row] : 0;
        if (g.out_mode == 0) {
          double* out = g.part + ((size_t)split * g.M + row) * (size_t)g.N;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = col0 + h * 32 + j;
            if (col >= g.N) continue;
            double v = MODE == 0 ? (double)acc[j] * 0x1p-42 + (double)tail[j]
                                 : (MODE == 3 ? (double)acc[j] * 0x1p-35 : (double)tail[j]);
            if (g.ea) v = ldexp(v, er + g.eb[col]);
            out[col] = v;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = col0 + h * 32 + j;
            if (col >= g.N) continue;
            double v = MODE == 0 ? (double)acc[j] * 0x1p-42 + (double)tail[j]
                                 : (MODE == 3 ? (double)acc[j] * 0x1p-35 : (double)tail[j]);
            if (g.ea) v = ldexp(v, er + g.eb[col]);
            v *= g.alpha;
            if (g.y_f32) {
              float* y = static_cast<float*>(g.Y) + (size_t)row * g.ldy + col;
              *y = (float)(g.beta != 0.0 ? v + g.beta * (double)*y : v);
            } else {
              double* y = static_cast<double*>(g.Y) + (size_t)row * g.ldy + col;
              *y = g.beta != 0.0 ? v + g.beta * *y : v;
            }
          }
        }
      }
    }
  }
  // all products and TMEM reads are complete (or abandoned after a bounded wait)
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(C::TCOLS) : "memory");
  }
}

// ---- slicing (FP64 / FP32 -> BF16 slices, K-major) ------------------------------------
__device__ __forceinline__ int frexp_exp(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const int E = (int)((u >> 52) & 0x7FF);
  if ((u << 1) == 0) return INT_MIN;  // +-0
  return E == 0 ? -1021 : E - 1022;   // |v| < 2^e
}

// Column exponents of a row slab: e[c] = max over rows of frexp exponents of X(r, c)
// (e starts below every FP64 exponent: the host fills it with 0x80 bytes; the
// maximum does not depend on the order of the atomics).
template <class Tin>
__global__ void k_tc_colexp(long rows, int cols, const Tin* __restrict__ X, long ldx, int* __restrict__ e) {
  __shared__ int sm[8][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  int m = INT_MIN;
  if (c < cols)
    for (long r = (long)blockIdx.y * 8 + threadIdx.y; r < rows; r += 8L * gridDim.y)
      m = max(m, frexp_exp((double)X[r * ldx + c]));
  sm[threadIdx.y][threadIdx.x] = m;
  __syncthreads();
  if (threadIdx.y == 0 && c < cols) {
#pragma unroll
    for (int y = 1; y < 8; ++y) m = max(m, sm[y][threadIdx.x]);
    if (m != INT_MIN) atomicMax(e + c, m);
  }
}

// BITS-bit fixed point of x relative to 2^e (|x| < 2^e), rounded to nearest
template <int BITS>
__device__ __forceinline__ long long fixed_point(double x, int e) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF);
  unsigned long long M = u & 0xFFFFFFFFFFFFFull;
  int Ee = E;
  if (E == 0) Ee = 1;
  else M |= 1ull << 52;
  if (M == 0) return 0;
  const int sh = Ee - 1075 + BITS - e;  // x * 2^(BITS-e) = M * 2^sh, sh <= BITS - 53
  if (sh >= 0) {
    const long long F = (long long)(M << sh);  // exact: |F| < 2^BITS
    return (u >> 63) ? -F : F;
  }
  const int r = -sh;
  if (r >= 63) return 0;
  const long long F = (long long)((M + (1ull << (r - 1))) >> r);
  return (u >> 63) ? -F : F;
}

// round-to-nearest base-2^7 digits: F = sum_a s_a 2^(7(NS-1-a)), |s_0| <= 128, |s_a| <= 64
template <int NS>
__device__ __forceinline__ void split_digits(long long F, int (&s)[NS]) {
#pragma unroll
  for (int a = 0; a < NS - 1; ++a) {
    const int sh = 7 * (NS - 1 - a);
    const long long d = (F + (1LL << (sh - 1))) >> sh;
    F -= d << sh;
    s[a] = (int)d;
  }
  s[NS - 1] = (int)F;
}

__device__ __forceinline__ uint16_t slice_bf16(int s, int a) {
  const float f = ldexpf((float)s, -7 * (a + 1));
  return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// Transposed slicing: row i of the sliced operand is column i of X (n_slab x cols,
// ldx); K index = row of X.  dst[a][i][k] (ldk), tiles of 32 columns x 64 rows.
// NS slices of 7 bits: 7 NS-bit fixed point relative to 2^e[i].
template <class Tin, int NS>
__global__ void k_tc_slice_T(long rows, int cols, const Tin* __restrict__ X, long ldx,
                             const int* __restrict__ e, uint16_t* __restrict__ dst, long ldk, long slice_stride) {
  __shared__ double tile[64][33];
  const int i0 = blockIdx.x * 32;
  const long k0 = (long)blockIdx.y * 64;
  for (int kk = threadIdx.y; kk < 64; kk += 8) {
    const long k = k0 + kk;
    const int i = i0 + threadIdx.x;
    tile[kk][threadIdx.x] = (k < rows && i < cols) ? (double)X[k * ldx + i] : 0.0;
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int i = i0 + ii;
    if (i >= cols) break;
    const int ei = e[i];
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int kk = threadIdx.x + 32 * half;
      const long k = k0 + kk;
      if (k >= rows) continue;
      int sl[NS];
      split_digits<NS>(fixed_point<7 * NS>(tile[kk][ii], ei), sl);
#pragma unroll
      for (int a = 0; a < NS; ++a) dst[a * slice_stride + (long)i * ldk + k] = slice_bf16(sl[a], a);
    }
  }
}

// Row slicing: row r of the sliced operand is row r of X (rows x cols, ldx); one
// warp per row finds the row exponent, then writes the slices dst[a][r][k].
template <class Tin, int NS>
__global__ void k_tc_slice_N(long rows, int cols, const Tin* __restrict__ X, long ldx, int* __restrict__ e,
                             uint16_t* __restrict__ dst, long ldk, long slice_stride) {
  const long warps = (long)gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (long r = (blockIdx.x * (long)blockDim.x + threadIdx.x) / 32; r < rows; r += warps) {
    const Tin* xr = X + r * ldx;
    int m = INT_MIN;
    for (int k = lane; k < cols; k += 32) m = max(m, frexp_exp((double)xr[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) e[r] = m == INT_MIN ? 0 : m;
    for (int k = lane; k < cols; k += 32) {
      int sl[NS];
      split_digits<NS>(m == INT_MIN ? 0 : fixed_point<7 * NS>((double)xr[k], m), sl);
#pragma unroll
      for (int a = 0; a < NS; ++a) dst[a * slice_stride + r * ldk + k] = slice_bf16(sl[a], a);
    }
  }
}

// all-zero columns (still at the initial fill, below any FP64 exponent): exponent 0
// (their slices are zero)
__global__ void k_tc_fix_exp(int n, int* e) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (e[i] < -4096) e[i] = 0;
}

// FP32 (rows x cols, ldx) -> K-major transposed FP32 (TF32 mode) or BF16 copy:
// dst[i][k] = X[k][i]
template <class To>
__global__ void k_tc_transpose_lowp(long rows, int cols, const float* __restrict__ X, long ldx, To* __restrict__ dst,
                                    long ldk) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.x * 32;
  const long k0 = (long)blockIdx.y * 32;
  for (int kk = threadIdx.y; kk < 32; kk += 8) {
    const long k = k0 + kk;
    const int i = i0 + threadIdx.x;
    tile[kk][threadIdx.x] = (k < rows && i < cols) ? X[k * ldx + i] : 0.f;
  }
  __syncthreads();
  for (int ii = threadIdx.y; ii < 32; ii += 8) {
    const int i = i0 + ii;
    const long k = k0 + threadIdx.x;
    if (i >= cols || k >= rows) continue;
    const float v = tile[threadIdx.x][ii];
    if constexpr (sizeof(To) == 4) dst[(long)i * ldk + k] = v;
    else dst[(long)i * ldk + k] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
  }
}

// G (+)= sum over splits of part[split][a][b]; symmetric products read entries of
// tiles that were not computed (below the diagonal band) from the mirror image.
__global__ void k_tc_reduce(int a, int b, int splits, const double* __restrict__ part, double* __restrict__ G,
                            long ldg, int sym, int accumulate) {
  const long total = (long)a * b;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int i = (int)(e / b), j = (int)(e % b);
    const bool mirror = sym && ((j / BN) * BN + BN - 1 < (i / BM) * BM);
    const long src = mirror ? (long)j * b + i : e;
    double s = 0.0;
    for (int p = 0; p < splits; ++p) s += part[(size_t)p * total + src];
    double* gp = G + (size_t)i * ldg + j;
    *gp = accumulate ? *gp + s : s;
  }
}

// ---- host side -----------------------------------------------------------------------
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn() {
  static EncodeFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 3-D map (k, row, slice) over dst[slice][row][ldk] with box (64 bytes of k, box_rows, 1)
void make_map(CUtensorMap* m, bool f32, const void* base, long k_len, long rows, int nsl, long ldk, int box_rows) {
  const int esz = f32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)k_len, (cuuint64_t)rows, (cuuint64_t)nsl};
  cuuint64_t strides[2] = {(cuuint64_t)(ldk * esz), (cuuint64_t)(ldk * esz * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(ROWB / esz), (cuuint32_t)box_rows, 1};
  cuuint32_t es[3] = {1, 1, 1};
  EncodeFn fn = encode_fn();
  CARE_REQUIRE(fn != nullptr, CARE_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const CUresult r = fn(m, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                        const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CARE_REQUIRE(r == CUDA_SUCCESS, CARE_ERR_CUDA, "cuTensorMapEncodeTiled failed");
}

int g_tc_starve = 0;

template <int MODE>
void launch_tc(const CUtensorMap& mA, const CUtensorMap& mB, TcArgs g, int tiles, int splits, cudaStream_t s) {
  g.starve = g_tc_starve;
  using C = TcCfg<MODE>;
  static std::once_flag once[64];
  int dev = 0;
  CARE_CUDA(cudaGetDevice(&dev));
  static cudaError_t attr_err[64];
  std::call_once(once[dev & 63], [&] {
    attr_err[dev & 63] = cudaFuncSetAttribute(k_tc_gemm<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  });
  CARE_CUDA(attr_err[dev & 63]);
  dim3 grid((unsigned)tiles, (unsigned)splits);
  k_tc_gemm<MODE><<<grid, TC_THREADS, C::SMEM, s>>>(mA, mB, g);
  CARE_LAUNCH();
}

long round_up(long x, long m) { return (x + m - 1) / m * m; }

}  // namespace

void tc_set_test_starve(int on) { g_tc_starve = on ? 1 : 0; }

static int g_tc_enabled = 1;
void tc_set_enabled(int on) { g_tc_enabled = on < 0 ? 0 : (on > 2 ? 2 : on); }
int tc_enabled() { return g_tc_enabled; }

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3 && encode_fn() != nullptr;
}

bool tc_f64_profitable(long k, int a, int b) {
  if (g_tc_enabled == 2) return a > 0 && b > 0;  // forced (tests)
  // the CUDA-core FP64 products are faster for narrow outputs
  return g_tc_enabled == 1 && k >= 1024 && a >= 48 && b >= 48 && (double)k * a * b >= 2.0e9;
}

size_t tc_scratch_bytes(int maxdim) {
  Arena a;
  TcScratch sc = tc_alloc(a, maxdim);
  (void)sc;
  return a.off;
}

TcScratch tc_alloc(Arena& ar, int maxdim) {
  TcScratch sc;
  const long md = std::max(maxdim, 64);
  sc.slice_bytes = (size_t)NSLICE * (size_t)md * SLAB * 2;
  sc.slices = ar.get<uint16_t>(sc.slice_bytes / 2);
  sc.expo_elems = (size_t)SLAB + (size_t)md + 64;
  sc.expo = ar.get<int>(sc.expo_elems);
  sc.part_elems = std::max<size_t>((size_t)1 << 22, (size_t)(md / 2 + 64) * (size_t)(md / 2 + 64) * 4);
  sc.part = ar.get<double>(sc.part_elems);
  sc.err = ar.get<int>(64);
  return sc;
}

int tc_check(const TcScratch& sc, cudaStream_t s) {
  if (!sc.err) return 0;
  int h = 0;
  CARE_CUDA(cudaMemcpyAsync(&h, sc.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CARE_CUDA(cudaStreamSynchronize(s));
  if (h) CARE_CUDA(cudaMemsetAsync(sc.err, 0, sizeof(int), s));
  return h;
}

// splits of a K range so that tiles * splits fills the SMs, >= 4 chunks per CTA,
// and splits * a * b partials fit
static int choose_splits(long k_len, long tiles, long ab, size_t part_elems) {
  const long sms = device_sms();
  long sp = (sms + tiles - 1) / tiles;
  sp = std::min(sp, std::max(1L, k_len / (4 * CHUNK)));
  sp = std::min(sp, std::max(1L, (long)(part_elems / (size_t)std::max(ab, 1L))));
  return (int)std::max(1L, sp);
}

// X^T Y (a x b, FP64) of FP64 (8 slices, MODE 0) or FP32 (4 slices, MODE 3) operands
template <class Tin>
static void tc_gram_sliced(long n, int a, int b, const Tin* X, int ldx, const Tin* Y, int ldy, double* G, int ldg,
                           const TcScratch& sc, int maxdim, cudaStream_t s) {
  constexpr int NS = sizeof(Tin) == 8 ? NSLICE : 4;
  if (a == 0 || b == 0) return;
  const bool sym = a == b && X == Y && ldx == ldy;
  CARE_REQUIRE(sc.ok() && a + (sym ? 0 : b) <= std::max(maxdim, 64), CARE_ERR_WORKSPACE, "tc_gram: scratch");
  CARE_REQUIRE((size_t)a * b <= sc.part_elems, CARE_ERR_WORKSPACE, "tc_gram: partials");
  const int tiles_m = (a + BM - 1) / BM, tiles_n = (b + BN - 1) / BN;
  long live = 0;
  for (int tj = 0; tj < tiles_n; ++tj)
    for (int ti = 0; ti < tiles_m; ++ti)
      if (!sym || tj * BN + BN - 1 >= ti * BM) ++live;
  if (n == 0) {
    CARE_CUDA(cudaMemsetAsync(sc.part, 0, (size_t)a * b * sizeof(double), s));
    k_tc_reduce<<<std::min<long>(((long)a * b + 255) / 256, device_sms() * 8L), 256, 0, s>>>(a, b, 1, sc.part, G,
                                                                                          ldg, 0, 0);
    CARE_LAUNCH();
    return;
  }
  int* eA = sc.expo;
  int* eB = sym ? eA : sc.expo + a;
  for (long r0 = 0; r0 < n; r0 += SLAB) {
    const long kl = std::min<long>(SLAB, n - r0);
    const long ldk = round_up(kl, 64);
    uint16_t* sA = sc.slices;
    uint16_t* sB = sym ? sA : sc.slices + (size_t)NS * a * ldk;
    // exponents and slices of the slab
    CARE_CUDA(cudaMemsetAsync(eA, 0x80, sizeof(int) * (size_t)(sym ? a : a + b), s));
    {
      dim3 blk(32, 8);
      const unsigned gy = (unsigned)std::min<long>((kl + 63) / 64, 64);
      k_tc_colexp<Tin><<<dim3((a + 31) / 32, gy), blk, 0, s>>>(kl, a, X + r0 * ldx, ldx, eA);
      CARE_LAUNCH();
      if (!sym) {
        k_tc_colexp<Tin><<<dim3((b + 31) / 32, gy), blk, 0, s>>>(kl, b, Y + r0 * ldy, ldy, eB);
        CARE_LAUNCH();
      }
      k_tc_fix_exp<<<8, 256, 0, s>>>(sym ? a : a + b, eA);
      CARE_LAUNCH();
      k_tc_slice_T<Tin, NS><<<dim3((a + 31) / 32, (unsigned)((kl + 63) / 64)), blk, 0, s>>>(
          kl, a, X + r0 * ldx, ldx, eA, sA, ldk, (long)a * ldk);
      CARE_LAUNCH();
      if (!sym) {
        k_tc_slice_T<Tin, NS><<<dim3((b + 31) / 32, (unsigned)((kl + 63) / 64)), blk, 0, s>>>(
            kl, b, Y + r0 * ldy, ldy, eB, sB, ldk, (long)b * ldk);
        CARE_LAUNCH();
      }
    }
    CUtensorMap mA, mB;
    make_map(&mA, false, sA, kl, a, NS, ldk, BM);
    make_map(&mB, false, sB, kl, b, NS, ldk, BN);
    const int splits = choose_splits(kl, live, (long)a * b, sc.part_elems);
    const long kps = round_up((kl + splits - 1) / splits, CHUNK);
    const int spl = (int)((kl + kps - 1) / kps);
    TcArgs g{};
    g.M = a; g.N = b; g.k_len = (int)kl; g.k_per_split = (int)kps; g.tiles_m = tiles_m; g.sym = sym ? 1 : 0;
    g.out_mode = 0; g.part = sc.part; g.ea = eA; g.eb = eB; g.err = sc.err;
    if constexpr (NS == NSLICE) launch_tc<0>(mA, mB, g, tiles_m * tiles_n, spl, s);
    else launch_tc<3>(mA, mB, g, tiles_m * tiles_n, spl, s);
    const int rg = (int)std::min<long>(((long)a * b + 255) / 256, device_sms() * 8L);
    k_tc_reduce<<<rg, 256, 0, s>>>(a, b, spl, sc.part, G, ldg, sym ? 1 : 0, r0 > 0 ? 1 : 0);
    CARE_LAUNCH();
  }
}

void tc_gram_f64(long n, int a, int b, const double* X, int ldx, const double* Y, int ldy, double* G, int ldg,
                 const TcScratch& sc, int maxdim, cudaStream_t s) {
  tc_gram_sliced<double>(n, a, b, X, ldx, Y, ldy, G, ldg, sc, maxdim, s);
}
void tc_gram_f32acc(long n, int a, int b, const float* X, int ldx, const float* Y, int ldy, double* G, int ldg,
                    const TcScratch& sc, int maxdim, cudaStream_t s) {
  tc_gram_sliced<float>(n, a, b, X, ldx, Y, ldy, G, ldg, sc, maxdim, s);
}

// Y = alpha X S + beta Y, X of type Tin (8 slices for FP64, 4 for FP32), S FP64
template <class Tin, class To>
void tc_gemm_ts_sliced(long n, int a, int b, double alpha, const Tin* X, int ldx, const double* S, int lds,
                       double beta, To* Y, int ldy, const TcScratch& sc, int maxdim, cudaStream_t s) {
  constexpr int NS = sizeof(Tin) == 8 ? NSLICE : 4;
  if (n == 0 || b == 0) return;
  CARE_REQUIRE(a > 0, CARE_ERR_INVALID_ARG, "tc_gemm_ts: a == 0");
  CARE_REQUIRE(sc.ok() && a + b <= std::max(maxdim, 64), CARE_ERR_WORKSPACE, "tc_gemm_ts: scratch");
  const long ldk = round_up(a, 64);
  // B operand: S^T (b rows, K = a), sliced once
  uint16_t* sB = sc.slices;
  int* eB = sc.expo + SLAB;
  CARE_CUDA(cudaMemsetAsync(eB, 0x80, sizeof(int) * (size_t)b, s));
  dim3 blk(32, 8);
  k_tc_colexp<double><<<dim3((b + 31) / 32, (unsigned)std::min<long>((a + 63) / 64, 64)), blk, 0, s>>>(a, b, S, lds,
                                                                                                     eB);
  CARE_LAUNCH();
  k_tc_fix_exp<<<8, 256, 0, s>>>(b, eB);
  CARE_LAUNCH();
  k_tc_slice_T<double, NS><<<dim3((b + 31) / 32, (unsigned)((a + 63) / 64)), blk, 0, s>>>(a, b, S, lds, eB, sB, ldk,
                                                                                          (long)b * ldk);
  CARE_LAUNCH();
  CUtensorMap mB;
  make_map(&mB, false, sB, a, b, NS, ldk, BN);
  uint16_t* sA = sc.slices + (size_t)NS * b * ldk;
  const size_t room = sc.slice_bytes / 2 - (size_t)NS * b * ldk;
  long slab = (long)(room / ((size_t)NS * ldk));
  slab = std::min<long>(slab, SLAB) / BM * BM;
  CARE_REQUIRE(slab >= BM, CARE_ERR_WORKSPACE, "tc_gemm_ts: scratch too small");
  int* eA = sc.expo;
  const int tiles_n = (b + BN - 1) / BN;
  for (long r0 = 0; r0 < n; r0 += slab) {
    const long rows = std::min(slab, n - r0);
    const int wg = (int)std::min<long>((rows + 7) / 8, device_sms() * 16L);
    k_tc_slice_N<Tin, NS><<<wg, 256, 0, s>>>(rows, a, X + r0 * ldx, ldx, eA, sA, ldk, rows * ldk);
    CARE_LAUNCH();
    CUtensorMap mA;
    make_map(&mA, false, sA, a, rows, NS, ldk, BM);
    const int tiles_m = (int)((rows + BM - 1) / BM);
    TcArgs g{};
    g.M = (int)rows; g.N = b; g.k_len = a; g.k_per_split = (int)round_up(a, CHUNK); g.tiles_m = tiles_m;
    g.sym = 0; g.out_mode = 1; g.ea = eA; g.eb = eB; g.Y = Y + r0 * ldy; g.ldy = ldy;
    g.y_f32 = sizeof(To) == 4 ? 1 : 0; g.alpha = alpha; g.beta = beta; g.err = sc.err;
    if constexpr (NS == NSLICE) launch_tc<0>(mA, mB, g, tiles_m * tiles_n, 1, s);
    else launch_tc<3>(mA, mB, g, tiles_m * tiles_n, 1, s);
  }
}

template <class To>
void tc_gemm_ts_f64(long n, int a, int b, double alpha, const double* X, int ldx, const double* S, int lds,
                    double beta, To* Y, int ldy, const TcScratch& sc, int maxdim, cudaStream_t s) {
  tc_gemm_ts_sliced<double, To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, sc, maxdim, s);
}
template void tc_gemm_ts_f64<double>(long, int, int, double, const double*, int, const double*, int, double,
                                     double*, int, const TcScratch&, int, cudaStream_t);
template void tc_gemm_ts_f64<float>(long, int, int, double, const double*, int, const double*, int, double,
                                    float*, int, const TcScratch&, int, cudaStream_t);
template <class To>
void tc_gemm_ts_f32acc(long n, int a, int b, double alpha, const float* X, int ldx, const double* S, int lds,
                       double beta, To* Y, int ldy, const TcScratch& sc, int maxdim, cudaStream_t s) {
  tc_gemm_ts_sliced<float, To>(n, a, b, alpha, X, ldx, S, lds, beta, Y, ldy, sc, maxdim, s);
}
template void tc_gemm_ts_f32acc<float>(long, int, int, double, const float*, int, const double*, int, double, float*,
                                       int, const TcScratch&, int, cudaStream_t);
template void tc_gemm_ts_f32acc<double>(long, int, int, double, const float*, int, const double*, int, double,
                                        double*, int, const TcScratch&, int, cudaStream_t);

void tc_gram_lowp(int kind, long n, int a, int b, const float* X, int ldx, const float* Y, int ldy, double* G,
                  int ldg, const TcScratch& sc, int maxdim, cudaStream_t s) {
  if (a == 0 || b == 0) return;
  CARE_REQUIRE(kind == 1 || kind == 2, CARE_ERR_INVALID_ARG, "tc_gram_lowp: kind");
  const bool sym = a == b && X == Y && ldx == ldy;
  CARE_REQUIRE(sc.ok() && a + (sym ? 0 : b) <= std::max(maxdim, 64), CARE_ERR_WORKSPACE, "tc_gram_lowp: scratch");
  CARE_REQUIRE((size_t)a * b <= sc.part_elems, CARE_ERR_WORKSPACE, "tc_gram_lowp: partials");
  const bool f32 = kind == 1;
  const int tiles_m = (a + BM - 1) / BM, tiles_n = (b + BN - 1) / BN;
  long live = 0;
  for (int tj = 0; tj < tiles_n; ++tj)
    for (int ti = 0; ti < tiles_m; ++ti)
      if (!sym || tj * BN + BN - 1 >= ti * BM) ++live;
  // slab so that the transposed copies fit the slice storage (FP32 takes 4 bytes)
  const long per_row_bytes = (long)(sym ? a : a + b) * (f32 ? 4 : 2);
  long slab = (long)(sc.slice_bytes / (size_t)per_row_bytes) / 64 * 64;
  slab = std::min<long>(slab, 4L * SLAB);
  CARE_REQUIRE(slab >= 64, CARE_ERR_WORKSPACE, "tc_gram_lowp: scratch too small");
  if (n == 0) {
    CARE_CUDA(cudaMemsetAsync(sc.part, 0, (size_t)a * b * sizeof(double), s));
    k_tc_reduce<<<std::min<long>(((long)a * b + 255) / 256, device_sms() * 8L), 256, 0, s>>>(a, b, 1, sc.part, G,
                                                                                          ldg, 0, 0);
    CARE_LAUNCH();
    return;
  }
  for (long r0 = 0; r0 < n; r0 += slab) {
    const long kl = std::min(slab, n - r0);
    const long ldk = round_up(kl, 64);
    void* dA = sc.slices;
    void* dB = sym ? dA : (void*)((char*)sc.slices + (size_t)a * ldk * (f32 ? 4 : 2));
    dim3 blk(32, 8);
    dim3 gA((a + 31) / 32, (unsigned)((kl + 31) / 32)), gB((b + 31) / 32, (unsigned)((kl + 31) / 32));
    if (f32) {
      k_tc_transpose_lowp<float><<<gA, blk, 0, s>>>(kl, a, X + r0 * ldx, ldx, (float*)dA, ldk);
      CARE_LAUNCH();
      if (!sym) {
        k_tc_transpose_lowp<float><<<gB, blk, 0, s>>>(kl, b, Y + r0 * ldy, ldy, (float*)dB, ldk);
        CARE_LAUNCH();
      }
    } else {
      k_tc_transpose_lowp<uint16_t><<<gA, blk, 0, s>>>(kl, a, X + r0 * ldx, ldx, (uint16_t*)dA, ldk);
      CARE_LAUNCH();
      if (!sym) {
        k_tc_transpose_lowp<uint16_t><<<gB, blk, 0, s>>>(kl, b, Y + r0 * ldy, ldy, (uint16_t*)dB, ldk);
        CARE_LAUNCH();
      }
    }
    CUtensorMap mA, mB;
    make_map(&mA, f32, dA, kl, a, 1, ldk, BM);
    make_map(&mB, f32, dB, kl, b, 1, ldk, BN);
    const int splits = choose_splits(kl, live, (long)a * b, sc.part_elems);
    const long kps = round_up((kl + splits - 1) / splits, CHUNK);
    const int spl = (int)((kl + kps - 1) / kps);
    TcArgs g{};
    g.M = a; g.N = b; g.k_len = (int)kl; g.k_per_split = (int)kps; g.tiles_m = tiles_m; g.sym = sym ? 1 : 0;
    g.out_mode = 0; g.part = sc.part; g.err = sc.err;
    if (f32) launch_tc<1>(mA, mB, g, tiles_m * tiles_n, spl, s);
    else launch_tc<2>(mA, mB, g, tiles_m * tiles_n, spl, s);
    const int rg = (int)std::min<long>(((long)a * b + 255) / 256, device_sms() * 8L);
    k_tc_reduce<<<rg, 256, 0, s>>>(a, b, spl, sc.part, G, ldg, sym ? 1 : 0, r0 > 0 ? 1 : 0);
    CARE_LAUNCH();
  }
}

}  // namespace care
