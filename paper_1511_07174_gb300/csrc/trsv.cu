// Forward and back substitution (paper section 2: L y = b, U x = y; and the
// transposed systems used by the gradient and by Cholesky's L^t x = y).
//
// The n rows are cut into 64-row blocks. Each CTA draws a ticket (atomic, in
// start order) that names the block it solves, so a CTA only ever waits on
// blocks owned by CTAs that started before it. For its block b it streams the
// 64 x 64 tiles M(b, q) of every earlier block q in solve order (coalesced
// loads into shared memory in either orientation), waits (bounded) for block
// q's flag, and accumulates M(b, q) x_q; then it solves its diagonal block
// in shared memory (one warp per right-hand side, lanes own rows), writes
// x_b and releases its flag. Arithmetic is FP64 whatever the storage type of
// the triangular factor (FP64 or FP32).
#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kTsBS = 64;
constexpr int kTsNR = 16;

size_t trsv_flags_count(int n) { return (size_t)((n + kTsBS - 1) / kTsBS) + 1; }

template <typename Ts, bool LOWER, bool TRANS, bool UNIT>
__global__ void __launch_bounds__(256)
    trsv_chain_kernel(int n, int nrhs, const Ts* __restrict__ T, int ldt, double* X, int ldx,
                      unsigned* flags, int* info, uint64_t wait_ns) {
  constexpr bool FWD = (LOWER != TRANS);
  __shared__ double tile[kTsBS][kTsBS + 1];
  __shared__ double xq[kTsBS][kTsNR];
  __shared__ int s_t, s_abort;
  const int tid = threadIdx.x;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  if (tid == 0) {
    s_t = (int)atomicAdd(&flags[nblk], 1u);
    s_abort = 0;
  }
  __syncthreads();
  const int t_ord = s_t;
  if (t_ord >= nblk) return;
  const int b = FWD ? t_ord : nblk - 1 - t_ord;
  const int r0 = b * kTsBS;
  const int nr = min(kTsBS, n - r0);
  const int r = tid & 63, g = tid >> 6;

  auto load_tile = [&](int c0, int nc) {
    for (int idx = tid; idx < kTsBS * kTsBS; idx += blockDim.x) {
      int rr, jj;
      if (!TRANS) {
        rr = idx & 63;
        jj = idx >> 6;
      } else {
        jj = idx & 63;
        rr = idx >> 6;
      }
      double v = 0.0;
      if (rr < nr && jj < nc)
        v = TRANS ? (double)T[(c0 + jj) + (size_t)(r0 + rr) * ldt]
                  : (double)T[(r0 + rr) + (size_t)(c0 + jj) * ldt];
      tile[rr][jj] = v;
    }
  };

  double acc[kTsNR];
#pragma unroll
  for (int c = 0; c < kTsNR; ++c) acc[c] = 0.0;

  for (int st = 0; st < t_ord; ++st) {
    const int q = FWD ? st : nblk - 1 - st;
    const int c0 = q * kTsBS;
    const int nc = min(kTsBS, n - c0);
    __syncthreads();
    load_tile(c0, nc);
    if (tid == 0) {
      if (!gbla_wait_geq(&flags[q], 1u, wait_ns)) {
        gbla_flag_timeout(info);
        s_abort = 1;
      }
      __threadfence();
    }
    __syncthreads();
    if (s_abort) return;
    for (int idx = tid; idx < kTsBS * nrhs; idx += blockDim.x) {
      const int jj = idx & 63, c = idx >> 6;
      xq[jj][c] = jj < nc ? __ldcg(&X[(c0 + jj) + (size_t)c * ldx]) : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = g * 16; jj < g * 16 + 16; ++jj) {
      const double tv = tile[r][jj];
#pragma unroll
      for (int c = 0; c < kTsNR; ++c)
        if (c < nrhs) acc[c] = fma(tv, xq[jj][c], acc[c]);
    }
  }
  // reduce the four partial sums of each row; the right-hand side of block b
  __syncthreads();
  double* part = &tile[0][0];
#pragma unroll
  for (int c = 0; c < kTsNR; ++c)
    if (c < nrhs) part[(g * kTsBS + r) * kTsNR + c] = acc[c];
  __syncthreads();
  for (int idx = tid; idx < kTsBS * nrhs; idx += blockDim.x) {
    const int rr = idx & 63, c = idx >> 6;
    double v = 0.0;
    if (rr < nr) {
      const double sum = (part[(0 * kTsBS + rr) * kTsNR + c] + part[(1 * kTsBS + rr) * kTsNR + c]) +
                         (part[(2 * kTsBS + rr) * kTsNR + c] + part[(3 * kTsBS + rr) * kTsNR + c]);
      v = __ldcg(&X[(r0 + rr) + (size_t)c * ldx]) - sum;
    }
    xq[rr][c] = v;
  }
  __syncthreads();
  load_tile(r0, nr);  // diagonal block
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  for (int c = warp; c < nrhs; c += (int)(blockDim.x >> 5)) {
    double y0 = xq[lane][c], y1 = xq[lane + 32][c];
    if (FWD) {
      for (int i = 0; i < nr; ++i) {
        double xi = __shfl_sync(0xffffffffu, i < 32 ? y0 : y1, i & 31);
        if (!UNIT) xi = xi / tile[i][i];
        if (lane == (i & 31)) {
          if (i < 32) y0 = xi;
          else y1 = xi;
        }
        if (lane > i) y0 = fma(-tile[lane][i], xi, y0);
        if (lane + 32 > i) y1 = fma(-tile[lane + 32][i], xi, y1);
      }
    } else {
      for (int i = nr - 1; i >= 0; --i) {
        double xi = __shfl_sync(0xffffffffu, i < 32 ? y0 : y1, i & 31);
        if (!UNIT) xi = xi / tile[i][i];
        if (lane == (i & 31)) {
          if (i < 32) y0 = xi;
          else y1 = xi;
        }
        if (lane < i) y0 = fma(-tile[lane][i], xi, y0);
        if (lane + 32 < i) y1 = fma(-tile[lane + 32][i], xi, y1);
      }
    }
    xq[lane][c] = y0;
    xq[lane + 32][c] = y1;
  }
  __syncthreads();
  for (int idx = tid; idx < kTsBS * nrhs; idx += blockDim.x) {
    const int rr = idx & 63, c = idx >> 6;
    if (rr < nr) X[(r0 + rr) + (size_t)c * ldx] = xq[rr][c];
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    st_release_u32(&flags[b], 1u);
  }
}

template <typename Ts>
cudaError_t launch_trsv(bool lower, bool trans, bool unit, int n, int nrhs, const Ts* T, int ldt,
                        double* X, int ldx, unsigned* flags, int* info, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  const uint64_t wait_ns = wait_timeout_ns();
  for (int c0 = 0; c0 < nrhs; c0 += kTsNR) {
    const int nc = nrhs - c0 < kTsNR ? nrhs - c0 : kTsNR;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)(nblk + 1), s);
    if (e != cudaSuccess) return e;
    double* Xc = X + (size_t)c0 * ldx;
#define GBLA_TRSV(LW, TR, UN)                                                                  \
  trsv_chain_kernel<Ts, LW, TR, UN><<<nblk, 256, 0, s>>>(n, nc, T, ldt, Xc, ldx, flags, info, \
                                                         wait_ns)
    if (lower && !trans && unit) GBLA_TRSV(true, false, true);
    else if (lower && !trans && !unit) GBLA_TRSV(true, false, false);
    else if (lower && trans && unit) GBLA_TRSV(true, true, true);
    else if (lower && trans && !unit) GBLA_TRSV(true, true, false);
    else if (!lower && !trans && unit) GBLA_TRSV(false, false, true);
    else if (!lower && !trans && !unit) GBLA_TRSV(false, false, false);
    else if (!lower && trans && unit) GBLA_TRSV(false, true, true);
    else GBLA_TRSV(false, true, false);
#undef GBLA_TRSV
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template cudaError_t launch_trsv<double>(bool, bool, bool, int, int, const double*, int, double*,
                                         int, unsigned*, int*, cudaStream_t);
template cudaError_t launch_trsv<float>(bool, bool, bool, int, int, const float*, int, double*,
                                        int, unsigned*, int*, cudaStream_t);

}  // namespace gbla

// ----------------------------------------------------------------------------
// Substitution with inverted diagonal blocks (the preconditioner apply of the
// refinement, one right-hand side). The inverse of every 64 x 64 diagonal
// block of the triangular factor is formed once per factorisation, in FP64,
// so that the per-block step of the chain is a 64 x 64 matrix-vector product
// instead of 64 dependent row eliminations. The operator applied is then a
// fixed linear map (the same for every vector), as GMRES requires.
namespace gbla {

// Dinv + b*64*64: column-major inverse of diagonal block b (zero-padded when
// the last block has fewer than 64 rows). One 64-thread CTA per block; thread
// j forms column j by substitution against e_j.
template <typename Ts, bool LOWER, bool UNIT>
__global__ void __launch_bounds__(64)
    diag_inv_kernel(int n, const Ts* __restrict__ T, int ldt, double* __restrict__ Dinv) {
  __shared__ double D[kTsBS][kTsBS + 1];
  const int b = blockIdx.x;
  const int r0 = b * kTsBS;
  const int nr = min(kTsBS, n - r0);
  const int t = threadIdx.x;
  for (int j = 0; j < kTsBS; ++j) D[t][j] = (t < nr && j < nr) ? (double)T[(r0 + t) + (size_t)(r0 + j) * ldt] : 0.0;
  __syncthreads();
  double* out = Dinv + (size_t)b * kTsBS * kTsBS + (size_t)t * kTsBS;  // column t
  double x[kTsBS];
#pragma unroll
  for (int i = 0; i < kTsBS; ++i) x[i] = 0.0;
  if (t < nr) {
    if (LOWER) {
#pragma unroll
      for (int i = 0; i < kTsBS; ++i) {
        if (i >= t && i < nr) {
          double s = (i == t) ? 1.0 : 0.0;
#pragma unroll
          for (int k = 0; k < kTsBS; ++k)
            if (k >= t && k < i) s = fma(-D[i][k], x[k], s);
          x[i] = UNIT ? s : s / D[i][i];
        }
      }
    } else {
#pragma unroll
      for (int ii = kTsBS - 1; ii >= 0; --ii) {
        if (ii <= t) {
          double s = (ii == t) ? 1.0 : 0.0;
#pragma unroll
          for (int k = 0; k < kTsBS; ++k)
            if (k > ii && k <= t) s = fma(-D[ii][k], x[k], s);
          x[ii] = UNIT ? s : s / D[ii][ii];
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < kTsBS; ++i) out[i] = x[i];
}

template <typename Ts>
cudaError_t launch_diag_inv(bool lower, bool unit, int n, const Ts* T, int ldt, double* Dinv,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  if (lower && unit) diag_inv_kernel<Ts, true, true><<<nblk, 64, 0, s>>>(n, T, ldt, Dinv);
  else if (lower) diag_inv_kernel<Ts, true, false><<<nblk, 64, 0, s>>>(n, T, ldt, Dinv);
  else if (unit) diag_inv_kernel<Ts, false, true><<<nblk, 64, 0, s>>>(n, T, ldt, Dinv);
  else diag_inv_kernel<Ts, false, false><<<nblk, 64, 0, s>>>(n, T, ldt, Dinv);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_diag_inv<float>(bool, bool, int, const float*, int, double*, cudaStream_t);
template cudaError_t launch_diag_inv<double>(bool, bool, int, const double*, int, double*, cudaStream_t);

size_t diag_inv_doubles(int n) { return (size_t)((n + kTsBS - 1) / kTsBS) * kTsBS * kTsBS; }

// One right-hand side, forward (lower factor) or backward (upper factor).
// The solution goes to X, which the launcher first fills with an all-ones bit
// pattern (a NaN that arithmetic does not produce): a block's x values
// announce themselves, so a consumer polls the 64 values it needs instead of a
// flag followed by a second load, and the producer needs no fence.
// Thread (r, g) = (tid % 64, tid / 64) keeps, in registers, elements
// (r, g + 4i), i < 16, of each 64 x 64 tile of its row block; the tile of the
// next earlier block is loaded while the current one waits for its x.
constexpr unsigned long long kXUnset = 0xffffffffffffffffull;

template <typename Ts, bool FWD>
__global__ void __launch_bounds__(256)
    trsv_inv_kernel(int n, const Ts* __restrict__ T, int ldt, const double* __restrict__ Dinv,
                    const double* __restrict__ rhs, double* X, unsigned* ticket, int* info,
                    uint64_t wait_ns) {
  extern __shared__ double smd[];
  double* dinv = smd;                  // 64 x 64, column-major
  double* xq = dinv + kTsBS * kTsBS;   // 64
  double* part = xq + kTsBS;           // 4 x 64
  double* rb = part + 4 * kTsBS;       // 64: this block's right-hand side
  __shared__ int s_t, s_abort;
  const int tid = threadIdx.x;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  if (tid == 0) {
    s_t = (int)atomicAdd(ticket, 1u);
    s_abort = 0;
  }
  __syncthreads();
  const int t_ord = s_t;
  if (t_ord >= nblk) return;
  const int b = FWD ? t_ord : nblk - 1 - t_ord;
  const int r0 = b * kTsBS;
  const int nr = min(kTsBS, n - r0);
  const int r = tid & 63, g = tid >> 6;

  // the inverse of the diagonal block and the right-hand side, needed last, are staged first
  const double* Db = Dinv + (size_t)b * kTsBS * kTsBS;
  for (int idx = tid; idx < kTsBS * kTsBS; idx += blockDim.x) dinv[idx] = Db[idx];
  if (tid < kTsBS) rb[tid] = tid < nr ? rhs[r0 + tid] : 0.0;

  auto load = [&](int st, Ts (&v)[16]) {
    const int q = FWD ? st : nblk - 1 - st;
    const int c0 = q * kTsBS;
    const int nc = min(kTsBS, n - c0);
    const Ts* base = T + (r0 + r) + (size_t)c0 * ldt;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int jj = g + 4 * i;
      v[i] = (r < nr && jj < nc) ? base[(size_t)jj * ldt] : (Ts)0;
    }
  };
  double a0 = 0.0, a1 = 0.0;
  Ts cur[16];
  if (t_ord > 0) load(0, cur);
  for (int st = 0; st < t_ord; ++st) {
    const int q = FWD ? st : nblk - 1 - st;
    const int c0 = q * kTsBS;
    const int nc = min(kTsBS, n - c0);
    Ts nxt[16];
    if (st + 1 < t_ord) load(st + 1, nxt);
    if (tid < kTsBS) {
      double v = 0.0;
      if (tid < nc) {
        const unsigned long long* px = reinterpret_cast<const unsigned long long*>(X + c0 + tid);
        unsigned long long bits;
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(px) : "memory");
        if (bits == kXUnset) {
          const uint64_t t0 = gbla_now_ns();
          do {
            asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(px) : "memory");
            if (gbla_now_ns() - t0 > wait_ns) {
              s_abort = 1;
              break;
            }
          } while (bits == kXUnset);
        }
        v = __longlong_as_double((long long)bits);
      }
      xq[tid] = v;
    }
    __syncthreads();
    if (s_abort) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
#pragma unroll
    for (int i = 0; i < 16; i += 2) {
      a0 = fma((double)cur[i], xq[g + 4 * i], a0);
      a1 = fma((double)cur[i + 1], xq[g + 4 * (i + 1)], a1);
    }
    if (st + 1 < t_ord) {
#pragma unroll
      for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
    }
    __syncthreads();  // xq is rewritten next step
  }
  part[g * kTsBS + r] = a0 + a1;
  __syncthreads();
  if (tid < kTsBS) {
    const double sum = (part[tid] + part[kTsBS + tid]) + (part[2 * kTsBS + tid] + part[3 * kTsBS + tid]);
    xq[tid] = tid < nr ? rb[tid] - sum : 0.0;
  }
  __syncthreads();
  // x_b = Dinv_b * rhs (column-major inverse)
  double y0 = 0.0, y1 = 0.0;
#pragma unroll
  for (int j = g * 16; j < g * 16 + 16; j += 2) {
    y0 = fma(dinv[r + kTsBS * j], xq[j], y0);
    y1 = fma(dinv[r + kTsBS * (j + 1)], xq[j + 1], y1);
  }
  part[g * kTsBS + r] = y0 + y1;
  __syncthreads();
  if (tid < nr) {
    const double xv = (part[tid] + part[kTsBS + tid]) + (part[2 * kTsBS + tid] + part[3 * kTsBS + tid]);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(xv);
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(X + r0 + tid), "l"(bits) : "memory");
  }
}

template <typename Ts>
cudaError_t launch_trsv_inv(bool lower, int n, const Ts* T, int ldt, const double* Dinv,
                            const double* rhs, double* X, unsigned* flags, int* info,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  // One CTA per SM: the late blocks of the chain are bound by the SM's FP64
  // rate, which two resident blocks would share. Asking for more than half
  // of an SM's shared memory keeps a second CTA off the SM; the blocks that do
  // not fit start as the early ones finish (in ticket order, so every block a
  // CTA waits for has started before it).
  const DeviceProps& dp = device_props();
  size_t smem = sizeof(double) * ((size_t)kTsBS * kTsBS + kTsBS + 4 * kTsBS + kTsBS);
  if (dp.smem_optin > 2 * smem) smem = dp.smem_optin / 2 + 1024;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(X, 0xff, sizeof(double) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  const uint64_t wait_ns = wait_timeout_ns();
  if (lower) {
    e = ensure_dyn_smem(trsv_inv_kernel<Ts, true>, smem);
    if (e != cudaSuccess) return e;
    trsv_inv_kernel<Ts, true><<<nblk, 256, smem, s>>>(n, T, ldt, Dinv, rhs, X, flags, info, wait_ns);
  } else {
    e = ensure_dyn_smem(trsv_inv_kernel<Ts, false>, smem);
    if (e != cudaSuccess) return e;
    trsv_inv_kernel<Ts, false><<<nblk, 256, smem, s>>>(n, T, ldt, Dinv, rhs, X, flags, info, wait_ns);
  }
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_trsv_inv<float>(bool, int, const float*, int, const double*,
                                            const double*, double*, unsigned*, int*, cudaStream_t);
template cudaError_t launch_trsv_inv<double>(bool, int, const double*, int, const double*,
                                             const double*, double*, unsigned*, int*, cudaStream_t);

}  // namespace gbla
