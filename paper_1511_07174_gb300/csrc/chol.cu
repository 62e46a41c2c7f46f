// Cholesky factorisation A = L L^t of an SPD matrix (paper section 2), lower
// triangle, blocked right-looking: outer blocks of nb columns (64 .. 256,
// autotunable), each processed in 64-column steps:
//   potf2   -- the 64 x 64 diagonal block factored by one CTA in shared memory
//              (column by column: d = a_jj, stop with info = j + 1 if d <= 0,
//              l_jj = sqrt(d), l_ij = a_ij / l_jj, a_ik -= l_ij l_kj);
//   trsm    -- the rows below it: L21 = A21 L11^{-t} in two 32-column halves
//              (one thread per row, its 32 values in registers, the triangle
//              in shared memory; the second half first receives the update
//              from the first);
//   update  -- A22 -= L21 L21^t on the lower triangle (the SIMT GEMM with its
//              lower-triangle mask; tiles above the diagonal are skipped):
//              inside the outer block for its remaining columns, then once
//              per outer block (rank nb) for the trailing matrix.
// The strict upper triangle of A is never read or written.
#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kCholNb = 64;

template <typename T>
__global__ void __launch_bounds__(256)
    potf2_kernel(int kb, T* __restrict__ A, int lda, int row0, int* __restrict__ info) {
  __shared__ T D[kCholNb][kCholNb + 1];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kCholNb * kCholNb; idx += blockDim.x) {
    const int r = idx & 63, c = idx >> 6;
    D[r][c] = (r < kb && c < kb && r >= c) ? A[r + (size_t)c * lda] : (T)0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  // an earlier block that failed leaves the rest of the factor undefined; the
  // first failure stays in info
  for (int j = 0; j < kb; ++j) {
    if (tid == 0) {
      const T d = D[j][j];
      if (!(d > (T)0)) {
        s_bad = 1;
        atomicCAS(info, 0, row0 + j + 1);
      } else {
        D[j][j] = sqrt(d);
      }
    }
    __syncthreads();
    if (s_bad) break;
    const T rl = (T)1 / D[j][j];
    for (int i = j + 1 + tid; i < kb; i += blockDim.x) D[i][j] *= rl;
    __syncthreads();
    // trailing part of the block: a_ik -= l_ij l_kj for i >= k > j
    const int m = kb - j - 1;
    for (int idx = tid; idx < m * m; idx += blockDim.x) {
      const int i = j + 1 + idx % m, k = j + 1 + idx / m;
      if (i >= k) D[i][k] = fma(-D[i][j], D[k][j], D[i][k]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < kCholNb * kCholNb; idx += blockDim.x) {
    const int r = idx & 63, c = idx >> 6;
    if (r < kb && c < kb && r >= c) A[r + (size_t)c * lda] = D[r][c];
  }
}

// X L11^t = B for the M rows of B (M x kb, ldb); L11 kb x kb lower (kb <= 32),
// one thread per row with its values in registers.
constexpr int kCholTrsmW = 32;

template <typename T>
__global__ void __launch_bounds__(128)
    chol_trsm_kernel(int M, int kb, const T* __restrict__ L, int lda, T* __restrict__ B, int ldb) {
  __shared__ T Ls[kCholTrsmW][kCholTrsmW + 1];
  __shared__ T rdiag[kCholTrsmW];
  const int tid = threadIdx.x;
  for (int idx = tid; idx < kCholTrsmW * kCholTrsmW; idx += blockDim.x) {
    const int r = idx % kCholTrsmW, c = idx / kCholTrsmW;
    Ls[r][c] = (r < kb && c < kb && r >= c) ? L[r + (size_t)c * lda] : (r == c ? (T)1 : (T)0);
  }
  __syncthreads();
  if (tid < kCholTrsmW) rdiag[tid] = (T)1 / Ls[tid][tid];
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + tid;
  if (row >= M) return;
  T x[kCholTrsmW];
#pragma unroll
  for (int k = 0; k < kCholTrsmW; ++k) x[k] = k < kb ? B[row + (size_t)k * ldb] : (T)0;
#pragma unroll
  for (int j = 0; j < kCholTrsmW; ++j) {
    x[j] *= rdiag[j];
#pragma unroll
    for (int k = j + 1; k < kCholTrsmW; ++k) x[k] = fma(-x[j], Ls[k][j], x[k]);
  }
#pragma unroll
  for (int k = 0; k < kCholTrsmW; ++k)
    if (k < kb) B[row + (size_t)k * ldb] = x[k];
}

// One outer block [o0, o0 + ob) in 64-column steps: diagonal block, the
// rows below it, and the update of the rest of the outer block's columns
// (lower part). Arithmetic in T.
template <typename T>
static cudaError_t chol_outer_block(int n, T* A, int lda, int o0, int ob, int* info, cudaStream_t s) {
  for (int k0 = o0; k0 < o0 + ob; k0 += kCholNb) {
    const int kb = o0 + ob - k0 < kCholNb ? o0 + ob - k0 : kCholNb;
    T* A11 = A + k0 + (size_t)k0 * lda;
    prof_begin(KK_PANEL, s);
    potf2_kernel<T><<<1, 256, 0, s>>>(kb, A11, lda, k0, info);
    count_launch();
    prof_end(KK_PANEL, s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int m = n - k0 - kb;
    if (m <= 0) break;
    T* A21 = A11 + kb;
    // L21 = A21 L11^{-t} in 32-column halves: solve the first half, update the
    // second with it, solve the second half
    for (int h0 = 0; h0 < kb; h0 += kCholTrsmW) {
      const int hb = kb - h0 < kCholTrsmW ? kb - h0 : kCholTrsmW;
      if (h0 > 0) {
        prof_begin(KK_GEMM_SIMT, s);
        e = launch_gemm_simt<T>(m, hb, h0, (T)-1, A21, lda, A11 + h0, lda, true, (T)1,
                                A21 + (size_t)h0 * lda, lda, false, s);
        prof_end(KK_GEMM_SIMT, s);
        if (e != cudaSuccess) return e;
      }
      prof_begin(KK_TRSM, s);
      chol_trsm_kernel<T><<<(m + 127) / 128, 128, 0, s>>>(m, hb, A11 + h0 + (size_t)h0 * lda, lda,
                                                          A21 + (size_t)h0 * lda, lda);
      count_launch();
      prof_end(KK_TRSM, s);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    // the rest of the outer block's columns (lower part): rows k0 + kb .. n,
    // columns k0 + kb .. o0 + ob
    const int nrest = o0 + ob - k0 - kb;
    if (nrest > 0) {
      prof_begin(KK_GEMM_SIMT, s);
      e = launch_gemm_simt<T>(m, nrest, kb, (T)-1, A21, lda, A21, lda, true, (T)1,
                              A21 + (size_t)kb * lda, lda, true, s);
      prof_end(KK_GEMM_SIMT, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// Two-level blocking: outer blocks of nb columns (a multiple of 64, up to
// 256); inside one, 64-column steps; after the outer block, one rank-nb
// update of the trailing lower triangle.
cudaError_t launch_chol(int n, double* A, int lda, int nb, int* info, cudaStream_t s) {
  if (nb <= 0) nb = kCholNb;
  if (nb % kCholNb != 0 || nb > 256) return cudaErrorInvalidValue;
  for (int o0 = 0; o0 < n; o0 += nb) {
    const int ob = n - o0 < nb ? n - o0 : nb;
    cudaError_t e = chol_outer_block<double>(n, A, lda, o0, ob, info, s);
    if (e != cudaSuccess) return e;
    // the trailing lower triangle: rank-ob update with the outer block's L21
    const int mt = n - o0 - ob;
    if (mt > 0) {
      double* L21 = A + (o0 + ob) + (size_t)o0 * lda;
      prof_begin(KK_GEMM_SIMT, s);
      e = launch_gemm_simt<double>(mt, mt, ob, -1.0, L21, lda, L21, lda, true, 1.0,
                                   L21 + (size_t)ob * lda, lda, true, s);
      prof_end(KK_GEMM_SIMT, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// F (n x n FP32, lower triangle) <- its Cholesky factor, the trailing update
// of each outer block in the precision `prec`: FP32 SIMT, or on the tensor
// cores (lower tiles only) from a K-major low-precision copy of L21 with one
// power-of-two scale per row, which serves both operands (split kinds: a
// second copy in the right operand's [hi | lo | hi] pattern). Afterwards the
// strict upper triangle holds L^t (a mirror of the strict lower one), so that
// the backward substitution with L^t reads an upper triangle.
cudaError_t launch_chol_mixed(int n, float* F, int ldf, int nb, int prec, void* Ak, void* Bk, int ldk,
                              int* eA, int* info, cudaStream_t s) {
  if (nb % kCholNb != 0 || nb <= 0 || nb > 256) return cudaErrorInvalidValue;
  const bool tensor = prec_is_tensor(prec);
  for (int o0 = 0; o0 < n; o0 += nb) {
    const int ob = n - o0 < nb ? n - o0 : nb;
    cudaError_t e = chol_outer_block<float>(n, F, ldf, o0, ob, info, s);
    if (e != cudaSuccess) return e;
    const int mt = n - o0 - ob;
    if (mt <= 0) continue;
    float* L21 = F + (o0 + ob) + (size_t)o0 * ldf;
    float* C = L21 + (size_t)ob * ldf;
    if (tensor) {
      prof_begin(KK_CONVERT, s);
      e = launch_convert_rows(L21, ldf, mt, ob, prec, Ak, ldk, eA, false, s);
      if (e == cudaSuccess && prec_is_split(prec))
        e = launch_convert_rows(L21, ldf, mt, ob, prec, Bk, ldk, eA, true, s);
      prof_end(KK_CONVERT, s);
      if (e != cudaSuccess) return e;
      prof_begin(KK_GEMM_TC, s);
      e = launch_gemm_tc(prec_mma_kind(prec), mt, mt, prec_kmult(prec) * ob, Ak, ldk,
                         prec_is_split(prec) ? Bk : Ak, ldk, eA, eA, C, ldf, info, true, s);
      prof_end(KK_GEMM_TC, s);
    } else {
      prof_begin(KK_GEMM_SIMT, s);
      e = launch_gemm_simt<float>(mt, mt, ob, -1.0f, L21, ldf, L21, ldf, true, 1.0f, C, ldf, true, s);
      prof_end(KK_GEMM_SIMT, s);
    }
    if (e != cudaSuccess) return e;
  }
  return launch_mirror_lower(n, F, ldf, s);
}

// Strict upper triangle <- transpose of the strict lower one (32 x 32 tiles
// through shared memory: coalesced on both sides).
__global__ void mirror_lower_kernel(int n, float* __restrict__ F, int ldf) {
  __shared__ float t[32][33];
  const int bi = blockIdx.x, bj = blockIdx.y;  // tile (bi, bj) of the lower triangle, bi >= bj
  if (bi < bj) return;
  const int i0 = bi * 32, j0 = bj * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + threadIdx.x, j = j0 + r;
    t[r][threadIdx.x] = (i < n && j < n && i > j) ? F[i + (size_t)j * ldf] : 0.0f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    // element (j0 + threadIdx.x, i0 + r) of the upper triangle = (i0 + r, j0 + threadIdx.x) of the lower
    const int i = i0 + r, j = j0 + threadIdx.x;
    if (i < n && j < n && i > j) F[j + (size_t)i * ldf] = t[threadIdx.x][r];
  }
}

cudaError_t launch_mirror_lower(int n, float* F, int ldf, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int T = (n + 31) / 32;
  mirror_lower_kernel<<<dim3(T, T), dim3(32, 8), 0, s>>>(n, F, ldf);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gbla
