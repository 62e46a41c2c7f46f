// Trailing-matrix update of the mixed-precision LU on the 5th-generation tensor
// cores (paper section 2: the rank-k "delayed update" A22 -= L21 U12).
//
// Output tiles of 128 x 128 are computed with tcgen05.mma (cta_group::1,
// M = N = 128, K = 16 per instruction for 16-bit operands, 8 for TF32) into an
// FP32 accumulator in tensor memory. Operands are K-major copies (one row of K
// elements per matrix row) loaded by TMA with 128-byte swizzle. The epilogue
// scales the accumulator by 2^-eA[row] * 2^-eB[col] (exact powers of two) and
// subtracts it from the FP32 working matrix C (column-major).
// Every mbarrier wait is bounded; a wait that gives up records
// GBLA_INFO_TIMEOUT, skips the epilogue writes, drains the copies it issued and
// frees its tensor memory before returning.
#include <cuda.h>
#include <string.h>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kTcBM = 128, kTcBN = 128;
constexpr int kTcStageBytes = 128 * 128;  // one operand tile: 128 rows x 128 bytes

GBLA_DEVINL uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

GBLA_DEVINL void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

GBLA_DEVINL void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

GBLA_DEVINL bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

GBLA_DEVINL bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; a limit of 0 does not wait at all (one non-blocking test):
// try_wait may suspend the thread for a while before it answers.
GBLA_DEVINL bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return mbar_test_wait(bar, parity);
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gbla_now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (gbla_now_ns() - t0 > limit_ns) return false;
  }
  return true;
}

GBLA_DEVINL void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset); the leading
// byte offset is unused for swizzled K-major layouts (set to 1).
GBLA_DEVINL uint64_t make_sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (0 FP16, 1 BF16,
// 2 TF32), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_fmt, int M, int N) {
  return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int KIND>
GBLA_DEVINL void mma_issue(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                           uint32_t accumulate) {
  if constexpr (KIND == GBLA_PREC_TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
  }
}

GBLA_DEVINL void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

GBLA_DEVINL void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Output tile t -> (row tile, column tile): column-major over the tile grid,
// or, for the lower triangle of tiles, row by row over (i, j), j <= i.
GBLA_DEVINL void tile_coords(int t, int tilesM, int lower, int& ti, int& tj) {
  if (!lower) {
    ti = t % tilesM;
    tj = t / tilesM;
    return;
  }
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((long long)(i + 1) * (i + 2) / 2 <= t) ++i;
  while ((long long)i * (i + 1) / 2 > t) --i;
  ti = i;
  tj = t - i * (i + 1) / 2;
}

// 2^e for |e| <= 126, built from the exponent field (exact).
GBLA_DEVINL float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// ---------------------------------------------------------------------------
// Persistent, warp-specialised kernel: one CTA per SM walks the output tiles
// (tile t, t + gridDim.x, ...). Warp 0 lane 0 issues TMA loads into a 4-stage
// ring, warp 1 lane 0 issues the MMAs into one of two tensor-memory
// accumulators (2 x 128 columns), and warps 2-9 run the epilogue of tile i
// (two warps per 32-lane group of tensor memory, one per half of the columns)
// while the MMAs of tile i + 1 proceed in the other accumulator.
//   full[s]  (TMA -> MMA, transaction bytes)   empty[s] (MMA commit -> TMA)
//   tfull[b] (MMA commit -> epilogue)          tempty[b] (8 epilogue warps -> MMA)
// Every wait is bounded; a give-up sets the shared fail flag, the info word,
// and every role stops at its next check.
constexpr int kPsStages = 4;
constexpr int kPsThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kPsStageC = 32 * 64 * 4;  // one epilogue warp's 32 rows x 64 columns of FP32
constexpr int kPsSmemBytes = 2 * kPsStages * kTcStageBytes + 8 * kPsStageC + 1024 + 512;
// Waits for copies and MMAs that have already been issued (leaving the kernel
// after a failed wait) end when the hardware finishes them; a caller's tiny
// wait limit must not cut them short.
constexpr uint64_t kPsDrainFloorNs = 200000000ull;

// Epilogue through the TMA unit: the scaled, negated accumulator is staged in
// shared memory and added to C by a bulk tensor reduction (C += -D), so the
// read-modify-write of the FP32 working matrix happens in the memory system
// instead of in registers.
GBLA_DEVINL void tma_reduce_add_2d(const CUtensorMap* map, int x, int y, uint32_t src) {
  asm volatile(
      "cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(src)
      : "memory");
}
// Bring a box of C into L2 ahead of its reduction (no completion to wait for).
GBLA_DEVINL void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y)
               : "memory");
}
GBLA_DEVINL void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
GBLA_DEVINL void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
GBLA_DEVINL void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
GBLA_DEVINL void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

GBLA_DEVINL void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

struct PsArgs {
  int M, N, K, tilesM, ntiles;
  int lower;  // enumerate only the tiles (i, j) with i >= j (M == N)
  float* C;
  int ldc;
  const int* eA;
  const int* eB;
  int* info;
  uint64_t wait_ns;
};

template <int KIND, bool TMAC>
__global__ void __launch_bounds__(kPsThreads, 1)
    gemm_tc_persistent_kernel(const __grid_constant__ CUtensorMap tmA,
                              const __grid_constant__ CUtensorMap tmB,
                              const __grid_constant__ CUtensorMap tmC, PsArgs args) {
  extern __shared__ unsigned char smraw[];
  const uint32_t raw = smem_u32(smraw);
  const uint32_t sbase = (raw + 1023u) & ~1023u;
  unsigned char* sm = smraw + (sbase - raw);
  const uint32_t sA = sbase;
  const uint32_t sB = sbase + kPsStages * kTcStageBytes;
  const uint32_t sC = sbase + 2 * kPsStages * kTcStageBytes;  // 8 x kPsStageC
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * kPsStages * kTcStageBytes + 8 * kPsStageC);
  const uint32_t bar_full = smem_u32(bars);
  const uint32_t bar_empty = bar_full + 8 * kPsStages;
  const uint32_t bar_tfull = bar_full + 16 * kPsStages;
  const uint32_t bar_tempty = bar_tfull + 16;
  const uint32_t bar_drain = bar_tempty + 16;  // the MMA issuer's last commit
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * kPsStages + 5);
  volatile int* s_fail = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile int* s_issued = s_fail + 1;

  constexpr int kElem = (KIND == GBLA_PREC_TF32) ? 4 : 2;
  constexpr int kBK = 128 / kElem;
  constexpr uint32_t kIdesc =
      make_idesc(KIND == GBLA_PREC_TF32 ? 2u : (KIND == GBLA_PREC_BF16 ? 1u : 0u), kTcBM, kTcBN);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (args.K + kBK - 1) / kBK;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kPsStages; ++st) {
      mbar_init(bar_full + 8 * st, 1);
      mbar_init(bar_empty + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, 8);
    }
    mbar_init(bar_drain, 1);
    *s_fail = 0;
    *s_issued = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(2 * kTcBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    if (lane == 0) {  // TMA producer
      int it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x) {
        int ti, tj;
        tile_coords(t, args.tilesM, args.lower, ti, tj);
        const int m0 = ti * kTcBM, n0 = tj * kTcBN;
        if constexpr (TMAC) {
          // the tile's C into L2 while its MMAs run, so that the epilogue's
          // reductions find it there (8 boxes of 32 rows x 64 columns)
#pragma unroll
          for (int r = 0; r < kTcBM; r += 32)
#pragma unroll
            for (int c = 0; c < kTcBN; c += 64) tma_prefetch_2d(&tmC, m0 + r, n0 + c);
        }
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int st = it % kPsStages;
          const uint32_t ph = (uint32_t)((it / kPsStages) & 1);
          if (*s_fail || !mbar_wait_bounded(bar_empty + 8 * st, ph ^ 1u, args.wait_ns)) {
            *s_fail = 1;
            ok = false;
            break;
          }
          mbar_expect_tx(bar_full + 8 * st, 2 * kTcStageBytes);
          tma_load_2d(sA + st * kTcStageBytes, &tmA, kb * kBK, m0, bar_full + 8 * st);
          tma_load_2d(sB + st * kTcStageBytes, &tmB, kb * kBK, n0, bar_full + 8 * st);
        }
      }
      *s_issued = it;
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      int it = 0, i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < args.ntiles && ok; t += gridDim.x, ++i) {
        const int b = i & 1;
        const uint32_t u = (uint32_t)(i >> 1);
        if (*s_fail || !mbar_wait_bounded(bar_tempty + 8 * b, (u & 1u) ^ 1u, args.wait_ns)) {
          *s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * kTcBN);
        for (int kb = 0; kb < KB; ++kb, ++it) {
          const int st = it % kPsStages;
          const uint32_t ph = (uint32_t)((it / kPsStages) & 1);
          if (!mbar_wait_bounded(bar_full + 8 * st, ph, args.wait_ns)) {
            *s_fail = 1;
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = make_sdesc(sA + st * kTcStageBytes + kk * 32);
            const uint64_t bd = make_sdesc(sB + st * kTcStageBytes + kk * 32);
            mma_issue<KIND>(d, ad, bd, kIdesc, (kb > 0 || kk > 0) ? 1u : 0u);
          }
          mma_commit(bar_empty + 8 * st);
        }
        mma_commit(bar_tfull + 8 * b);
      }
      // every MMA this thread issued has finished before tensor memory is freed
      // (after a failed wait some may still be running)
      mma_commit(bar_drain);
      const uint64_t dns = args.wait_ns > kPsDrainFloorNs ? args.wait_ns : kPsDrainFloorNs;
      if (!mbar_wait_bounded(bar_drain, 0u, dns)) *s_fail = 1;
    }
  } else {  // epilogue warps 2..9: TMEM lane group warp % 4, column half (warp - 2) / 4
    const int eg = warp & 3;
    const int c_lo = ((warp - 2) >> 2) * (kTcBN / 2);
    int i = 0;
    for (int t = blockIdx.x; t < args.ntiles; t += gridDim.x, ++i) {
      const int b = i & 1;
      const uint32_t u = (uint32_t)(i >> 1);
      // the tile's scales are loaded before its accumulator is waited for, so
      // that their latency hides behind the MMAs: this lane's row, and the
      // columns c_lo + lane and c_lo + 32 + lane of this warp's half
      int ti, tj;
      tile_coords(t, args.tilesM, args.lower, ti, tj);
      const int m0 = ti * kTcBM, n0 = tj * kTcBN;
      const int row = m0 + eg * 32 + lane;
      const bool rok = row < args.M;
      const float sa = (rok && args.eA) ? pow2f(-args.eA[row]) : 1.0f;
      const int ncol = min(kTcBN, args.N - n0);
      float sbh[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int col = c_lo + 32 * h + lane;
        sbh[h] = (args.eB && col < ncol) ? pow2f(-__ldg(args.eB + n0 + col)) : 1.0f;
      }
      int bad = 0;
      if (lane == 0) bad = (!mbar_wait_bounded(bar_tfull + 8 * b, u & 1u, args.wait_ns)) || *s_fail;
      bad = __shfl_sync(0xffffffffu, bad, 0);
      if (bad) {
        *s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if constexpr (TMAC) {
        // this warp's staging area: 64 columns x 32 rows, column-major
        const int wi = warp - 2;
        const uint32_t stage = sC + wi * kPsStageC;
        float* st = reinterpret_cast<float*>(sm + 2 * kPsStages * kTcStageBytes + wi * kPsStageC);
        if (lane == 0) bulk_wait_read0();  // the previous reduction has read the area
        __syncwarp();
#pragma unroll 1
        for (int cb = c_lo; cb < c_lo + kTcBN / 2; cb += 16) {
          uint32_t v[16];
          tmem_ld16(tmem + (uint32_t)(b * kTcBN) + ((uint32_t)(eg * 32) << 16) + (uint32_t)cb, v);
          const int q = cb - c_lo;  // 0, 16, 32, 48
          const float my_sb = q < 32 ? sbh[0] : sbh[1];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float sb = __shfl_sync(0xffffffffu, my_sb, (q & 31) + j);
            st[(q + j) * 32 + lane] = -((__uint_as_float(v[j]) * sa) * sb);
          }
        }
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          tma_reduce_add_2d(&tmC, m0 + eg * 32, n0 + c_lo, stage);
          bulk_commit();
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_tempty + 8 * b);
        continue;
      }
      float* __restrict__ crow = args.C + row + (size_t)n0 * args.ldc;
#pragma unroll 1
      for (int cb = c_lo; cb < c_lo + kTcBN / 2; cb += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + (uint32_t)(b * kTcBN) + ((uint32_t)(eg * 32) << 16) + (uint32_t)cb, v);
        const int q = cb - c_lo;
        const float my_sb = q < 32 ? sbh[0] : sbh[1];
        float sbv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) sbv[j] = __shfl_sync(0xffffffffu, my_sb, (q & 31) + j);
        if (rok) {
          float cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            cv[j] = (cb + j < ncol) ? crow[(size_t)(cb + j) * args.ldc] : 0.0f;
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (cb + j < ncol) crow[(size_t)(cb + j) * args.ldc] = cv[j] - (__uint_as_float(v[j]) * sa) * sbv[j];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tempty + 8 * b);
    }
  }
  if constexpr (TMAC) {
    if (warp >= 2 && lane == 0) bulk_wait0();  // reductions done before the CTA exits
  }
  __syncthreads();
  if (*s_fail) {
    if (threadIdx.x == 0) {
      gbla_flag_timeout(args.info);
      const int issued = *s_issued;
      const uint64_t dns = args.wait_ns > kPsDrainFloorNs ? args.wait_ns : kPsDrainFloorNs;
      for (int it = (issued > kPsStages ? issued - kPsStages : 0); it < issued; ++it)
        mbar_wait_bounded(bar_full + 8 * (it % kPsStages), (uint32_t)((it / kPsStages) & 1), dns);
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(2 * kTcBN));
  }
}

// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static bool encode_kmajor(CUtensorMap* map, int kind, const void* ptr, int K, int rows, int ld) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  const int elem = kind == GBLA_PREC_TF32 ? 4 : 2;
  CUtensorMapDataType dt = kind == GBLA_PREC_TF32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                           : kind == GBLA_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * elem};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem), 128u};
  cuuint32_t estr[2] = {1u, 1u};
  CUresult r = enc(map, dt, 2, const_cast<void*>(ptr), gdim, gstride, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t launch_gemm_tc(int kind, int M, int N, int K, const void* Ak, int ldak, const void* Bk,
                           int ldbk, const int* eA, const int* eB, float* C, int ldc, int* info,
                           bool lower, cudaStream_t s, int grid_cap) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (lower && M != N) return cudaErrorInvalidValue;
  const int elem = kind == GBLA_PREC_TF32 ? 4 : 2;
  if (((size_t)ldak * elem) % 16 != 0 || ((size_t)ldbk * elem) % 16 != 0) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Ak) & 15) || (reinterpret_cast<uintptr_t>(Bk) & 15))
    return cudaErrorInvalidValue;
  CUtensorMap ta, tb;
  if (!encode_kmajor(&ta, kind, Ak, K, M, ldak)) return cudaErrorInvalidValue;
  if (!encode_kmajor(&tb, kind, Bk, K, N, ldbk)) return cudaErrorInvalidValue;
  const int tilesM = (M + kTcBM - 1) / kTcBM, tilesN = (N + kTcBN - 1) / kTcBN;
  const int ntiles = lower ? tilesM * (tilesM + 1) / 2 : tilesM * tilesN;
  PsArgs a{M, N, K, tilesM, ntiles, lower ? 1 : 0, C, ldc, eA, eB, info, wait_timeout_ns()};
  const DeviceProps& dp = device_props();
  int grid = dp.num_sms > 0 ? dp.num_sms : 1;
  if (grid_cap > 0 && grid > grid_cap) grid = grid_cap;
  if (grid > a.ntiles) grid = a.ntiles;
  // the TMA reduction needs a 16-byte aligned C and a column stride that is a
  // multiple of 16 bytes; otherwise the epilogue updates C with plain loads/stores
  CUtensorMap tc;
  memset(&tc, 0, sizeof(tc));
  bool tmac = ((reinterpret_cast<uintptr_t>(C) & 15) == 0) && (((size_t)ldc * 4) % 16 == 0);
  if (tmac) {
    EncodeTiledFn enc = get_encode();
    cuuint64_t gdim[2] = {(cuuint64_t)M, (cuuint64_t)N};
    cuuint64_t gstride[1] = {(cuuint64_t)ldc * 4};
    cuuint32_t box[2] = {32u, 64u};
    cuuint32_t estr[2] = {1u, 1u};
    tmac = enc && enc(&tc, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, C, gdim, gstride, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  switch (kind) {
#define GBLA_TC_CASE(K)                                                                         \
  case K: {                                                                                   \
    if (tmac) {                                                                               \
      cudaError_t ea = ensure_dyn_smem(gemm_tc_persistent_kernel<K, true>, (size_t)kPsSmemBytes); \
      if (ea != cudaSuccess) return ea;                                                       \
      gemm_tc_persistent_kernel<K, true><<<grid, kPsThreads, kPsSmemBytes, s>>>(ta, tb, tc, a); \
    } else {                                                                                  \
      cudaError_t ea = ensure_dyn_smem(gemm_tc_persistent_kernel<K, false>, (size_t)kPsSmemBytes); \
      if (ea != cudaSuccess) return ea;                                                       \
      gemm_tc_persistent_kernel<K, false><<<grid, kPsThreads, kPsSmemBytes, s>>>(ta, tb, tc, a); \
    }                                                                                         \
    break;                                                                                    \
  }
    GBLA_TC_CASE(GBLA_PREC_TF32)
    GBLA_TC_CASE(GBLA_PREC_BF16)
    GBLA_TC_CASE(GBLA_PREC_FP16)
#undef GBLA_TC_CASE
    default:
      return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace gbla
