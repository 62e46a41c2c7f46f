// Level-3 pieces of the blocked LU (paper section 2, "delayed updating"):
// the unit-lower triangular solve of the U row block, the fused inner step
// (solve and update inside an outer block), the SIMT rank-k update (FP64 /
// FP32), the precision conversions that feed the tensor-core update, and
// permutation helpers for the solves.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "internal.h"

namespace gbla {

// ----------------------------------------------------------------------------
// Low-precision conversion helpers (power-of-two sliver scaling).
GBLA_DEVINL int sliver_exponent(float maxabs) {
  if (!(maxabs > 0.0f)) return 0;
  int e = 14 - ilogbf(maxabs);  // maxabs * 2^e in [2^14, 2^15)
  return e > 100 ? 100 : (e < -100 ? -100 : e);
}

GBLA_DEVINL uint32_t f32_to_tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Store one scaled operand value into a K-major row `row` (K elements per
// segment). Plain kinds: row[k] = round(v). Split kinds (hi = round(v),
// lo = round(v - hi), v - hi exact in FP32): the L21 pattern (LEFT) is
// [hi | hi | lo], the U12 pattern is [hi | lo | hi], so that the three
// segment products sum to hi*hi + hi*lo + lo*hi.
template <int KIND, bool LEFT>
GBLA_DEVINL void store_lowp(void* base, size_t row, int K, int k, float v) {
  if constexpr (KIND == GBLA_PREC_BF16) {
    reinterpret_cast<__nv_bfloat16*>(base)[row + k] = __float2bfloat16_rn(v);
  } else if constexpr (KIND == GBLA_PREC_FP16) {
    reinterpret_cast<__half*>(base)[row + k] = __float2half_rn(v);
  } else if constexpr (KIND == GBLA_PREC_TF32) {
    reinterpret_cast<uint32_t*>(base)[row + k] = f32_to_tf32_rna(v);
  } else if constexpr (KIND == GBLA_PREC_FP16X3) {
    __half* b = reinterpret_cast<__half*>(base) + row;
    const __half hi = __float2half_rn(v);
    const __half lo = __float2half_rn(v - __half2float(hi));
    b[k] = hi;
    b[K + k] = LEFT ? hi : lo;
    b[2 * K + k] = LEFT ? lo : hi;
  } else {
    __nv_bfloat16* b = reinterpret_cast<__nv_bfloat16*>(base) + row;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    b[k] = hi;
    b[K + k] = LEFT ? hi : lo;
    b[2 * K + k] = LEFT ? lo : hi;
  }
}

// ----------------------------------------------------------------------------
// TRSM: B (w x N) <- L^{-1} B, L unit lower w x w. A warp owns 4 columns; row
// r = lane + 32 q (q < Q, w <= 32 Q) of each column lives in lane `lane`.
// Columns of L are staged through shared memory 32 at a time. The loop over
// those 32-row chunks is unrolled, so every register index is a constant and
// a chunk only updates the row groups at or below it.
constexpr int kTrsmCols = 32;  // columns per CTA (8 warps x 4)

template <typename Ts, typename Tc, int OUT, int Q>
__global__ void __launch_bounds__(256)
    trsm_lunit_kernel(const Ts* __restrict__ L, int ldl, Ts* __restrict__ B, int ldb, int w, int N,
                      void* __restrict__ outK, int ldk, int* __restrict__ outE) {
  extern __shared__ unsigned char smraw[];
  Tc* Ls = reinterpret_cast<Tc*>(smraw);  // [32][w]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col0 = blockIdx.x * kTrsmCols + warp * 4;
  Tc x[Q][4];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int r = lane + 32 * q;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int col = col0 + c;
      x[q][c] = (r < w && col < N) ? (Tc)B[r + (size_t)col * ldb] : (Tc)0;
    }
  }
#pragma unroll
  for (int qi = 0; qi < Q; ++qi) {
    const int i0 = 32 * qi;
    if (i0 < w) {
      __syncthreads();
      {
        // all loads of the chunk are issued before any shared-memory store
        constexpr int kPer = 4 * Q;  // 32 x (32 Q) elements over 256 threads
        Ts v[kPer];
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
          const int idx = threadIdx.x + 256 * t;
          const int cc = idx / w, r = idx - cc * w, i = i0 + cc;
          v[t] = (idx < 32 * w && i < w && r > i) ? L[r + (size_t)i * ldl] : (Ts)0;
        }
#pragma unroll
        for (int t = 0; t < kPer; ++t) {
          const int idx = threadIdx.x + 256 * t;
          if (idx < 32 * w) Ls[idx] = (Tc)v[t];
        }
      }
      __syncthreads();
      const int iend = min(32, w - i0);
      for (int ii = 0; ii < iend; ++ii) {
        Tc xi[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) xi[c] = __shfl_sync(0xffffffffu, x[qi][c], ii);
        const Tc* lcol = Ls + ii * w;
#pragma unroll
        for (int q = qi; q < Q; ++q) {
          const int r = lane + 32 * q;
          const Tc l = r < w ? lcol[r] : (Tc)0;
#pragma unroll
          for (int c = 0; c < 4; ++c) x[q][c] = fma(-l, xi[c], x[q][c]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int col = col0 + c;
    float mx = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int r = lane + 32 * q;
      if (r < w && col < N) {
        const Ts v = (Ts)x[q][c];
        B[r + (size_t)col * ldb] = v;
        if constexpr (OUT != 0) mx = fmaxf(mx, fabsf((float)v));
      }
    }
    if constexpr (OUT != 0) {
      mx = warp_max(mx);
      const int e = (OUT == GBLA_PREC_TF32) ? 0 : sliver_exponent(mx);
      if (col < N) {
        if (lane == 0) outE[col] = e;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int r = lane + 32 * q;
          if (r < w) store_lowp<OUT, false>(outK, (size_t)col * ldk, w, r, ldexpf((float)(Ts)x[q][c], e));
        }
      }
    }
  }
}

template <typename Ts, typename Tc, int Q>
static cudaError_t trsm_dispatch(const Ts* L, int ldl, Ts* B, int ldb, int w, int N, int out_kind,
                                 void* outK, int ldk, int* outE, cudaStream_t s) {
  const size_t smem = (size_t)32 * w * sizeof(Tc);
  const dim3 grid((N + kTrsmCols - 1) / kTrsmCols);
#define GBLA_TRSM_CASE(K)                                                  \
  {                                                                      \
    auto kfn = trsm_lunit_kernel<Ts, Tc, K, Q>;                          \
    cudaError_t ea = ensure_dyn_smem(kfn, smem);                         \
    if (ea != cudaSuccess) return ea;                                    \
    kfn<<<grid, 256, smem, s>>>(L, ldl, B, ldb, w, N, outK, ldk, outE);  \
    break;                                                               \
  }
  if constexpr (sizeof(Ts) == 8) {
    // the low-precision copies exist for FP32 storage only
    switch (out_kind) {
      case 0: GBLA_TRSM_CASE(0)
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (out_kind) {
      case 0: GBLA_TRSM_CASE(0)
      case GBLA_PREC_BF16: GBLA_TRSM_CASE(GBLA_PREC_BF16)
      case GBLA_PREC_FP16: GBLA_TRSM_CASE(GBLA_PREC_FP16)
      case GBLA_PREC_TF32: GBLA_TRSM_CASE(GBLA_PREC_TF32)
      case GBLA_PREC_FP16X3: GBLA_TRSM_CASE(GBLA_PREC_FP16X3)
      case GBLA_PREC_BF16X3: GBLA_TRSM_CASE(GBLA_PREC_BF16X3)
      default: return cudaErrorInvalidValue;
    }
  }
#undef GBLA_TRSM_CASE
  count_launch();
  return cudaGetLastError();
}

template <typename Ts, typename Tc>
cudaError_t launch_trsm_lunit(const Ts* L, int ldl, Ts* B, int ldb, int w, int N, int out_kind,
                              void* outK, int ldk, int* outE, cudaStream_t s) {
  if (w <= 0 || N <= 0) return cudaSuccess;
  if (w > 256) return cudaErrorInvalidValue;
  if (w <= 32) return trsm_dispatch<Ts, Tc, 1>(L, ldl, B, ldb, w, N, out_kind, outK, ldk, outE, s);
  return trsm_dispatch<Ts, Tc, 8>(L, ldl, B, ldb, w, N, out_kind, outK, ldk, outE, s);
}
template cudaError_t launch_trsm_lunit<double, double>(const double*, int, double*, int, int, int,
                                                       int, void*, int, int*, cudaStream_t);
template cudaError_t launch_trsm_lunit<float, float>(const float*, int, float*, int, int, int, int,
                                                     void*, int, int*, cudaStream_t);

// ----------------------------------------------------------------------------
// Inner step of the blocked LU, fused into one launch: U12 = L11^{-1} A12 and
// A22 -= L21 U12 for a 32-column panel. CTA (x, y) owns the 64 x 64 tile
// (x, y) of A22; it solves the 64 columns of U12 above its tile itself (a
// 32 x 32 x 64 / 2 FMA right-looking solve, small next to the tile's
// update), in the same order of operations as the separate substitution
// kernel, so the results are those of the two-kernel sequence. The last CTA
// of a column of tiles to have read A12 (one counter per column of tiles)
// writes U12 back and clears its counter, so no CTA ever reads a solved
// value as input and no CTA waits for another.
template <typename T>
__global__ void __launch_bounds__(256)
    inner_update_kernel(int M, int N, T* __restrict__ P, int lda, unsigned* __restrict__ counters) {
  constexpr int BM = 64, BN = 64, K = kPanelWidth, TM = 4, TN = 4, RX = BM / TM, RY = BN / TN;
  __shared__ T Ls[K][K + 1];   // strictly lower part of L11
  __shared__ T Us[K][BN + 1];  // A12 tile, then U12 tile
  __shared__ T As[K][BM + 1];  // L21 tile, k-major
  __shared__ int s_last;
  const int tid = threadIdx.x;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  T* A12 = P + (size_t)K * lda;
  const T* A21 = P + K;
  T* A22 = P + K + (size_t)K * lda;
  {
    // all global loads are issued before any shared-memory store
    T vl[K * K / 256], vu[K * BN / 256], va[BM * K / 256];
#pragma unroll
    for (int t = 0; t < K * K / 256; ++t) {
      const int idx = tid + 256 * t, i = idx % K, k = idx / K;
      vl[t] = i > k ? P[i + (size_t)k * lda] : (T)0;
    }
#pragma unroll
    for (int t = 0; t < K * BN / 256; ++t) {
      const int idx = tid + 256 * t, k = idx % K, n = n0 + idx / K;
      vu[t] = n < N ? A12[k + (size_t)n * lda] : (T)0;
    }
#pragma unroll
    for (int t = 0; t < BM * K / 256; ++t) {
      const int idx = tid + 256 * t, m = m0 + idx % BM, k = idx / BM;
      va[t] = m < M ? A21[m + (size_t)k * lda] : (T)0;
    }
#pragma unroll
    for (int t = 0; t < K * K / 256; ++t) {
      const int idx = tid + 256 * t;
      Ls[idx % K][idx / K] = vl[t];
    }
#pragma unroll
    for (int t = 0; t < K * BN / 256; ++t) {
      const int idx = tid + 256 * t;
      Us[idx % K][idx / K] = vu[t];
    }
#pragma unroll
    for (int t = 0; t < BM * K / 256; ++t) {
      const int idx = tid + 256 * t;
      As[idx / BM][idx % BM] = va[t];
    }
  }
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&counters[blockIdx.y], 1u) == gridDim.x - 1;
  if (tid < BN) {
    // column tid of U12: u_i -= l_ik u_k for k = 0, 1, ... (unit diagonal)
    T u[K];
#pragma unroll
    for (int k = 0; k < K; ++k) u[k] = Us[k][tid];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int i = k + 1; i < K; ++i) u[i] = fma(-Ls[i][k], u[k], u[i]);
#pragma unroll
    for (int k = 0; k < K; ++k) Us[k][tid] = u[k];
  }
  __syncthreads();
  if (s_last) {
    for (int idx = tid; idx < K * BN; idx += 256) {
      const int k = idx % K, n = n0 + idx / K;
      if (n < N) A12[k + (size_t)n * lda] = Us[k][idx / K];
    }
    if (tid == 0) counters[blockIdx.y] = 0u;
  }
  const int tx = tid % RX, ty = tid / RX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;
#pragma unroll 8
  for (int kk = 0; kk < K; ++kk) {
    T a[TM], b[TN];
#pragma unroll
    for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + i * RX];
#pragma unroll
    for (int j = 0; j < TN; ++j) b[j] = Us[kk][ty + j * RY];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int n = n0 + ty + j * RY;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + i * RX;
      if (m < M && n < N) {
        T* c = A22 + m + (size_t)n * lda;
        *c = fma((T)-1, acc[i][j], *c);
      }
    }
  }
}

template <typename T>
cudaError_t launch_inner_update(int M, int N, T* P, int lda, unsigned* counters, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const dim3 grid((M + 63) / 64, (N + 63) / 64);
  if ((int)grid.y > kInnerCounters) return cudaErrorInvalidValue;
  inner_update_kernel<T><<<grid, 256, 0, s>>>(M, N, P, lda, counters);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_inner_update<double>(int, int, double*, int, unsigned*, cudaStream_t);
template cudaError_t launch_inner_update<float>(int, int, float*, int, unsigned*, cudaStream_t);

// ----------------------------------------------------------------------------
// SIMT GEMM: C = alpha * A * op(B) + beta * C. Thread (tx, ty) owns rows
// tx + i*(BM/TM) and columns ty + j*(BN/TN) of the tile, so that the lanes of
// a warp touch consecutive rows of column-major C.
template <typename T, int BM, int BN, int BK, int TM, int TN, bool TRANSB, bool LOWER>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
    gemm_simt_kernel(int M, int N, int K, T alpha, const T* __restrict__ A, int lda,
                     const T* __restrict__ B, int ldb, T beta, T* __restrict__ C, int ldc) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int RX = BM / TM, RY = BN / TN;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  if (LOWER && m0 + BM - 1 < n0) return;  // tile strictly above the diagonal
  const int tid = threadIdx.x;
  const int tx = tid % RX, ty = tid / RX;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;
  constexpr int PA = (BM * BK + NT - 1) / NT, PB = (BN * BK + NT - 1) / NT;
  for (int k0 = 0; k0 < K; k0 += BK) {
    // all global loads of the tile pair are issued before any shared store
    T va[PA], vb[PB];
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int idx = tid + NT * t;
      const int mm = idx % BM, kk = idx / BM;
      const int m = m0 + mm, k = k0 + kk;
      va[t] = (idx < BM * BK && m < M && k < K) ? A[m + (size_t)k * lda] : (T)0;
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int idx = tid + NT * t;
      int nn, kk;
      if (TRANSB) {
        nn = idx % BN;
        kk = idx / BN;
      } else {
        kk = idx % BK;
        nn = idx / BK;
      }
      const int nidx = n0 + nn, k = k0 + kk;
      T v = (T)0;
      if (idx < BN * BK && nidx < N && k < K)
        v = TRANSB ? B[nidx + (size_t)k * ldb] : B[k + (size_t)nidx * ldb];
      vb[t] = v;
    }
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int idx = tid + NT * t;
      if (idx < BM * BK) As[idx / BM][idx % BM] = va[t];
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int idx = tid + NT * t;
      if (idx < BN * BK) {
        if (TRANSB) Bs[idx / BN][idx % BN] = vb[t];
        else Bs[idx % BK][idx / BK] = vb[t];
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tx + i * RX];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][ty + j * RY];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int n = n0 + ty + j * RY;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + tx + i * RX;
      if (m < M && n < N && (!LOWER || m >= n)) {
        T* c = C + m + (size_t)n * ldc;
        *c = (beta == (T)0) ? alpha * acc[i][j] : fma(alpha, acc[i][j], beta * *c);
      }
    }
  }
}

template <typename T>
cudaError_t launch_gemm_simt(int M, int N, int K, T alpha, const T* A, int lda, const T* B,
                             int ldb, bool transB, T beta, T* C, int ldc, bool lower,
                             cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if constexpr (sizeof(T) == 8) {
    constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    if (transB) {
      if (lower)
        gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, true><<<grid, 256, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
      else
        gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, false><<<grid, 256, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    } else {
      gemm_simt_kernel<T, BM, BN, BK, TM, TN, false, false><<<grid, 256, 0, s>>>(
          M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    }
  } else if (N <= 256 && !transB && !lower) {
    // narrow updates (the inner steps of a block column): smaller tiles, more CTAs
    constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    gemm_simt_kernel<T, BM, BN, BK, TM, TN, false, false><<<grid, 256, 0, s>>>(
        M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
  } else {
    constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8;
    dim3 grid((M + BM - 1) / BM, (N + BN - 1) / BN);
    if (transB) {
      if (lower)
        gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, true><<<grid, 256, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
      else
        gemm_simt_kernel<T, BM, BN, BK, TM, TN, true, false><<<grid, 256, 0, s>>>(
            M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    } else {
      gemm_simt_kernel<T, BM, BN, BK, TM, TN, false, false><<<grid, 256, 0, s>>>(
          M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    }
  }
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_gemm_simt<double>(int, int, int, double, const double*, int,
                                              const double*, int, bool, double, double*, int,
                                              bool, cudaStream_t);
template cudaError_t launch_gemm_simt<float>(int, int, int, float, const float*, int, const float*,
                                             int, bool, float, float*, int, bool, cudaStream_t);

// ----------------------------------------------------------------------------
// L21 (FP32, M x K column-major) -> K-major low-precision rows with one
// power-of-two exponent per row. CTA: 32 rows; shared-memory transpose.
// LEFT: the left operand's pattern for the split kinds ([hi | hi | lo]);
// otherwise the right operand's ([hi | lo | hi]).
template <int KIND, bool LEFT>
__global__ void __launch_bounds__(256)
    convert_rows_kernel(const float* __restrict__ F, int ldf, int M, int K, void* __restrict__ outK,
                        int ldk, int* __restrict__ outE) {
  __shared__ float tile[64][33];
  __shared__ float wmax[8][32];
  __shared__ int es[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m0 = blockIdx.x * 32;
  const int m = m0 + lane;
  float mx = 0.0f;
  if (m < M)
    for (int k = warp; k < K; k += 8) mx = fmaxf(mx, fabsf(F[m + (size_t)k * ldf]));
  wmax[warp][lane] = mx;
  __syncthreads();
  if (warp == 0) {
    float v = 0.0f;
#pragma unroll
    for (int q = 0; q < 8; ++q) v = fmaxf(v, wmax[q][lane]);
    const int e = (KIND == GBLA_PREC_TF32) ? 0 : sliver_exponent(v);
    es[lane] = e;
    if (m < M) outE[m] = e;
  }
  __syncthreads();
  for (int k0 = 0; k0 < K; k0 += 64) {
    for (int idx = threadIdx.x; idx < 64 * 32; idx += 256) {
      const int kk = idx >> 5, mm = idx & 31;
      const int mr = m0 + mm, k = k0 + kk;
      tile[kk][mm] = (mr < M && k < K) ? F[mr + (size_t)k * ldf] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int mm = warp * 4 + r, mr = m0 + mm;
      if (mr < M) {
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int kk = lane * 2 + t, k = k0 + kk;
          if (k < K) store_lowp<KIND, LEFT>(outK, (size_t)mr * ldk, K, k, ldexpf(tile[kk][mm], es[mm]));
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_convert_rows(const float* F, int ldf, int M, int K, int kind, void* outK,
                                int ldk, int* outE, bool right, cudaStream_t s) {
  if (M <= 0 || K <= 0) return cudaSuccess;
  dim3 grid((M + 31) / 32);
#define GBLA_CONV(KD)                                                                          \
  if (right)                                                                                   \
    convert_rows_kernel<KD, false><<<grid, 256, 0, s>>>(F, ldf, M, K, outK, ldk, outE);        \
  else                                                                                         \
    convert_rows_kernel<KD, true><<<grid, 256, 0, s>>>(F, ldf, M, K, outK, ldk, outE);
  switch (kind) {
    case GBLA_PREC_BF16: GBLA_CONV(GBLA_PREC_BF16) break;
    case GBLA_PREC_FP16: GBLA_CONV(GBLA_PREC_FP16) break;
    case GBLA_PREC_TF32: GBLA_CONV(GBLA_PREC_TF32) break;
    case GBLA_PREC_FP16X3: GBLA_CONV(GBLA_PREC_FP16X3) break;
    case GBLA_PREC_BF16X3: GBLA_CONV(GBLA_PREC_BF16X3) break;
    default:
      return cudaErrorInvalidValue;
  }
#undef GBLA_CONV
  count_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// lower: rows r >= column only (the strict upper triangle of F is left as is)
__global__ void copy_d2f_kernel(const double* __restrict__ A, int lda, float* __restrict__ F,
                                int ldf, int m, int c0, int lower) {
  const int col = blockIdx.y;
  const int r0 = lower ? c0 + col : 0;
  for (int r = r0 + blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
    F[r + (size_t)col * ldf] = (float)A[r + (size_t)col * lda];
}

cudaError_t launch_copy_d2f(const double* A, int lda, float* F, int ldf, int m, int n,
                            cudaStream_t s, bool lower) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  int bx = (m + 255) / 256;
  if (bx > 16) bx = 16;
  for (int c0 = 0; c0 < n; c0 += 65535) {
    const int nc = n - c0 < 65535 ? n - c0 : 65535;
    copy_d2f_kernel<<<dim3(bx, nc), 256, 0, s>>>(A + (size_t)c0 * lda, lda, F + (size_t)c0 * ldf,
                                                 ldf, m, c0, lower ? 1 : 0);
    count_launch();
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// perm from sequential interchanges: (P v)[i] = v[perm[i]]. One CTA takes the
// interchanges 256 at a time: swap_plan gives, in parallel, where each row
// touched by the chunk gets its value from, and the CTA applies that map to
// the running permutation (every read before any write). The permutation
// lives in shared memory when it fits, else in perm itself.
__global__ void __launch_bounds__(1024)
    ipiv_to_perm_kernel(int n, const int* __restrict__ ipiv, int* __restrict__ perm, int use_smem) {
  extern __shared__ int sp[];
  __shared__ SwapPlanShared s_plan;
  int* p = use_smem ? sp : perm;
  const int t = threadIdx.x;
  for (int i = t; i < n; i += blockDim.x) p[i] = i;
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 256) {
    const int kb = min(256, n - c0);
    if (t < kb) {
      int q = ipiv[c0 + t] - 1 - c0;
      if (q < t || q >= n - c0) q = t;  // out-of-range pivots are ignored
      s_plan.p[t] = q;
    }
    __syncthreads();
    int src_b = t, dst_o = -1, src_o = 0;
    swap_plan(s_plan, kb, t, &src_b, &dst_o, &src_o);
    int vb = 0, vo = 0;
    if (t < kb) {
      vb = p[c0 + src_b];
      if (dst_o >= 0) vo = p[c0 + src_o];
    }
    __syncthreads();
    if (t < kb) {
      p[c0 + t] = vb;
      if (dst_o >= 0) p[c0 + dst_o] = vo;
    }
    __syncthreads();
  }
  if (use_smem)
    for (int i = t; i < n; i += blockDim.x) perm[i] = p[i];
}

__global__ void iota_kernel(int n, int* __restrict__ perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

cudaError_t launch_ipiv_to_perm(int n, const int* ipiv, int* perm, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (!ipiv) {  // no interchanges: the identity
    iota_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, s>>>(n, perm);
    count_launch();
    return cudaGetLastError();
  }
  const DeviceProps& dp = device_props();
  const size_t bytes = (size_t)n * sizeof(int);
  const int use_smem = bytes + sizeof(SwapPlanShared) + 1024 <= dp.smem_optin ? 1 : 0;
  if (use_smem) {
    cudaError_t ea = ensure_dyn_smem(ipiv_to_perm_kernel, bytes);
    if (ea != cudaSuccess) return ea;
  }
  ipiv_to_perm_kernel<<<1, 1024, use_smem ? bytes : 0, s>>>(n, ipiv, perm, use_smem);
  count_launch();
  return cudaGetLastError();
}

__global__ void permute_rows_kernel(int n, int nrhs, const int* __restrict__ perm, int inverse,
                                    const double* __restrict__ src, int lds,
                                    double* __restrict__ dst, int ldd) {
  const int c = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int p = perm[i];
    if (inverse)
      dst[p + (size_t)c * ldd] = src[i + (size_t)c * lds];
    else
      dst[i + (size_t)c * ldd] = src[p + (size_t)c * lds];
  }
}

cudaError_t launch_permute_rows(int n, int nrhs, const int* perm, bool inverse, const double* src,
                                int lds, double* dst, int ldd, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  int bx = (n + 255) / 256;
  if (bx > 1024) bx = 1024;
  permute_rows_kernel<<<dim3(bx, nrhs), 256, 0, s>>>(n, nrhs, perm, inverse ? 1 : 0, src, lds, dst,
                                                     ldd);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gbla

namespace gbla {

// ----------------------------------------------------------------------------
// C (m x n) = alpha * U V^t + beta * C, U m x k, V n x k (k <= 16), FP64. The
// gradient of a solve with respect to A (-gb x^t) is this product with
// alpha = -1, beta = 0. Thread i of a CTA owns row i0 + i of 32 columns; the
// k values of its row of U stay in registers and V's 32 rows sit in shared
// memory, so every output element is written once, coalesced down a column.
constexpr int kRkRows = 256, kRkCols = 32, kRkMaxK = 16;

__global__ void __launch_bounds__(kRkRows)
    rank_k_kernel(int m, int n, int k, double alpha, const double* __restrict__ U, int ldu,
                  const double* __restrict__ V, int ldv, double beta, double* __restrict__ C,
                  int ldc) {
  __shared__ double vs[kRkCols][kRkMaxK];
  const int i = blockIdx.x * kRkRows + threadIdx.x;
  const int j0 = blockIdx.y * kRkCols;
  for (int idx = threadIdx.x; idx < kRkCols * kRkMaxK; idx += blockDim.x) {
    const int jj = idx % kRkCols, c = idx / kRkCols;
    vs[jj][c] = (j0 + jj < n && c < k) ? V[(j0 + jj) + (size_t)c * ldv] : 0.0;
  }
  __syncthreads();
  if (i >= m) return;
  double u[kRkMaxK];
#pragma unroll
  for (int c = 0; c < kRkMaxK; ++c) u[c] = c < k ? U[i + (size_t)c * ldu] : 0.0;
  const int jn = min(kRkCols, n - j0);
  for (int jj = 0; jj < jn; ++jj) {
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < kRkMaxK; ++c) acc = fma(u[c], vs[jj][c], acc);
    double* cp = C + i + (size_t)(j0 + jj) * ldc;
    *cp = beta == 0.0 ? alpha * acc : fma(alpha, acc, beta * *cp);
  }
}

cudaError_t launch_rank_k(int m, int n, int k, double alpha, const double* U, int ldu,
                          const double* V, int ldv, double beta, double* C, int ldc,
                          cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  for (int c0 = 0; c0 < k || (k == 0 && c0 == 0); c0 += kRkMaxK) {
    const int kc = k - c0 < kRkMaxK ? k - c0 : kRkMaxK;
    const double b = c0 == 0 ? beta : 1.0;
    dim3 grid((m + kRkRows - 1) / kRkRows, (n + kRkCols - 1) / kRkCols);
    rank_k_kernel<<<grid, kRkRows, 0, s>>>(m, n, kc, alpha, U + (size_t)c0 * ldu, ldu,
                                           V + (size_t)c0 * ldv, ldv, b, C, ldc);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (k == 0) break;
  }
  return cudaSuccess;
}

}  // namespace gbla
