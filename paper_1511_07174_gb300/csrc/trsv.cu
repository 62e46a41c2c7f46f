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

// Right-hand sides are split over two independent chains (the columns of X
// are solved independently), each with its own flags: the FP64 work of a
// chain step halves, and two chains share the SMs without crowding them
// (measured: 16 columns as 2 x 8 beat 4 x 4 and 8 x 2; 8 columns as 2 x 4
// beat 1 x 8).
constexpr int kTsChains = 2;
static int trsv_chains(int nrhs) { return nrhs < 2 ? 1 : kTsChains; }
size_t trsv_flags_count(int n, int nrhs) {
  return (size_t)trsv_chains(nrhs) * (size_t)((n + kTsBS - 1) / kTsBS) + 1;
}

template <typename Ts, bool LOWER, bool TRANS, bool UNIT>
__global__ void __launch_bounds__(256)
    trsv_chain_kernel(int n, int ncols, int G, int C, const Ts* __restrict__ T, int ldt, double* X,
                      int ldx, unsigned* flags, int* info, uint64_t wait_ns) {
  constexpr bool FWD = (LOWER != TRANS);
  __shared__ double tile[kTsBS][kTsBS + 1];
  __shared__ double xq[kTsBS][kTsNR];
  __shared__ int s_t, s_abort;
  const int tid = threadIdx.x;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  if (tid == 0) {
    s_t = (int)atomicAdd(&flags[(size_t)C * nblk], 1u);
    s_abort = 0;
  }
  __syncthreads();
  // ticket -> (chain, position in that chain's solve order): a CTA waits only
  // for earlier positions of its own chain, which hold smaller tickets
  const int chain = s_t % C;
  const int t_ord = s_t / C;
  if (t_ord >= nblk) return;
  flags += (size_t)chain * nblk;
  X += (size_t)chain * G * ldx;
  const int nrhs = min(G, ncols - chain * G);
  if (nrhs <= 0) return;
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
  // one launch per kTsChains x kTsNR columns, split over C chains of G columns
  const int C = trsv_chains(nrhs);
  for (int c0 = 0; c0 < nrhs; c0 += C * kTsNR) {
    const int ncols = nrhs - c0 < C * kTsNR ? nrhs - c0 : C * kTsNR;
    const int G = (ncols + C - 1) / C;
    const int Cl = (ncols + G - 1) / G;  // chains that hold columns
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * ((size_t)C * nblk + 1), s);
    if (e != cudaSuccess) return e;
    double* Xc = X + (size_t)c0 * ldx;
    const int grid = Cl * nblk;
#define GBLA_TRSV(LW, TR, UN)                                                                  \
  trsv_chain_kernel<Ts, LW, TR, UN><<<grid, 256, 0, s>>>(n, ncols, G, Cl, T, ldt, Xc, ldx, flags, \
                                                         info, wait_ns)
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
// j forms column j by substitution against e_j. The same array then holds
// W (at nblk * 64 * 64) and V (at 2 nblk * 64 * 64) per block, and the
// substitution's partial-sum slots (see trsv_inv_kernel).
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

template <typename Ts, bool FWD>
__global__ void __launch_bounds__(256)
    trsv_wv_kernel(int n, const Ts* __restrict__ T, int ldt, double* __restrict__ Dinv);
// shared memory of trsv_wv_kernel: D_s (64 x 64) and one tile (64 x 65), FP64
constexpr size_t kWvSmemBytes = sizeof(double) * ((size_t)kTsBS * kTsBS + (size_t)kTsBS * (kTsBS + 1));

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
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nblk < 2) return e;
  // W_s = D_s T(s, s-1), V_s = D_s T(s, s-2) in solve order
  if (lower) {
    e = ensure_dyn_smem(trsv_wv_kernel<Ts, true>, kWvSmemBytes);
    if (e != cudaSuccess) return e;
    trsv_wv_kernel<Ts, true><<<dim3(nblk, 2), 256, kWvSmemBytes, s>>>(n, T, ldt, Dinv);
  } else {
    e = ensure_dyn_smem(trsv_wv_kernel<Ts, false>, kWvSmemBytes);
    if (e != cudaSuccess) return e;
    trsv_wv_kernel<Ts, false><<<dim3(nblk, 2), 256, kWvSmemBytes, s>>>(n, T, ldt, Dinv);
  }
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_diag_inv<float>(bool, bool, int, const float*, int, double*, cudaStream_t);
template cudaError_t launch_diag_inv<double>(bool, bool, int, const double*, int, double*, cudaStream_t);


// ---------------------------------------------------------------------------
// One right-hand side, forward (lower factor) or backward (upper factor), in
// solve order s = 0 .. nblk-1 (block b = s forward, nblk-1-s backward). With
// D_s the inverse of diagonal block s, W_s = D_s T(s, s-1) and
// V_s = D_s T(s, s-2) (both formed once, by launch_diag_inv):
//   x_s = D_s (rhs_s - sum_{t < s-2} T(s, t) x_t) - V_s x_{s-2} - W_s x_{s-1}.
// The far sum is cut into chunks of kTiChunk tiles, each done by a helper
// task that publishes its 64 partial sums; the owner task of block s adds the
// chunks in order, applies D_s, then V_s x_{s-2} and, once x_{s-1} is known,
// W_s x_{s-1}: one 64 x 64 product per block stays on the chain, and the far
// tiles of late blocks (FP64-bound) spread over many SMs.
//
// Tasks are drawn by ticket in the order (block 0: owner; block 1: owner;
// block s: helpers 0 .. h_s - 1, owner), so a task only ever waits for tasks
// with smaller tickets, which have started. Results announce themselves: X and
// the partial-sum slots start as an all-ones bit pattern (a NaN that
// arithmetic does not produce) and a consumer polls the values it needs.
// The result is a fixed linear map of rhs (the same operations in the same
// order every call), as GMRES requires.
constexpr unsigned long long kXUnset = 0xffffffffffffffffull;
constexpr int kTiChunk = 16;

__host__ __device__ inline int ti_helpers(int s) { return s >= 2 ? (s - 2 + kTiChunk - 1) / kTiChunk : 0; }

static int ti_tasks(int nblk) {
  int t = 0;
  for (int s = 0; s < nblk; ++s) t += ti_helpers(s) + 1;
  return t;
}

size_t diag_inv_doubles(int n) {
  const int nblk = (n + kTsBS - 1) / kTsBS;
  return (size_t)3 * nblk * kTsBS * kTsBS + (size_t)ti_tasks(nblk) * kTsBS;
}

// poll one announced FP64 value (bounded); false on timeout
GBLA_DEVINL bool ti_poll(const double* p, uint64_t wait_ns, double* out) {
  const unsigned long long* px = reinterpret_cast<const unsigned long long*>(p);
  unsigned long long bits;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(px) : "memory");
  if (bits == kXUnset) {
    const uint64_t t0 = gbla_now_ns();
    do {
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(bits) : "l"(px) : "memory");
      if (gbla_now_ns() - t0 > wait_ns) return false;
    } while (bits == kXUnset);
  }
  *out = __longlong_as_double((long long)bits);
  return true;
}

GBLA_DEVINL void ti_announce(double* p, double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(bits) : "memory");
}

// W_s and V_s (CTA (s, k): k = 0 -> W_s = D_s T(s, s-1), k = 1 -> V_s = D_s T(s, s-2)).

template <typename Ts, bool FWD>
__global__ void __launch_bounds__(256)
    trsv_wv_kernel(int n, const Ts* __restrict__ T, int ldt, double* __restrict__ Dinv) {
  extern __shared__ double wv_smem[];
  double* Ds = wv_smem;                                                  // column-major D_s
  double (*Tt)[kTsBS + 1] = reinterpret_cast<double (*)[kTsBS + 1]>(wv_smem + kTsBS * kTsBS);  // T(b, q)
  const int nblk = (n + kTsBS - 1) / kTsBS;
  const int s = blockIdx.x, k = blockIdx.y;
  const int sp = s - 1 - k;
  if (sp < 0) return;
  const int b = FWD ? s : nblk - 1 - s, q = FWD ? sp : nblk - 1 - sp;
  const int r0 = b * kTsBS, c0 = q * kTsBS;
  const int nr = min(kTsBS, n - r0), nc = min(kTsBS, n - c0);
  const double* D = Dinv + (size_t)b * kTsBS * kTsBS;
  for (int i = threadIdx.x; i < kTsBS * kTsBS; i += blockDim.x) {
    Ds[i] = D[i];
    const int rr = i & 63, jj = i >> 6;
    Tt[rr][jj] = (rr < nr && jj < nc) ? (double)T[(r0 + rr) + (size_t)(c0 + jj) * ldt] : 0.0;
  }
  __syncthreads();
  double* out = Dinv + (size_t)(1 + k) * nblk * kTsBS * kTsBS + (size_t)b * kTsBS * kTsBS;
  const int r = threadIdx.x & 63, g = threadIdx.x >> 6;
  for (int jj = g * 16; jj < g * 16 + 16; ++jj) {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll 8
    for (int kk = 0; kk < kTsBS; kk += 2) {
      a0 = fma(Ds[r + kTsBS * kk], Tt[kk][jj], a0);
      a1 = fma(Ds[r + kTsBS * (kk + 1)], Tt[kk + 1][jj], a1);
    }
    out[r + kTsBS * jj] = a0 + a1;
  }
}

template <typename Ts, bool FWD>
__global__ void __launch_bounds__(256)
    trsv_inv_kernel(int n, const Ts* __restrict__ T, int ldt, const double* __restrict__ Dinv,
                    const double* __restrict__ rhs, double* X, unsigned* ticket, int* info,
                    uint64_t wait_ns) {
  extern __shared__ double smd[];
  double* xq = smd;                    // 64: the x values of the current step
  double* part = xq + kTsBS;           // 4 x 64 partial sums
  double* dv = part + 4 * kTsBS;       // 64: owner's running vector
  double* mat = dv + kTsBS;            // 64 x 64: D_s, then V_s, then W_s (owner)
  __shared__ int s_t, s_abort;
  const int tid = threadIdx.x;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  const size_t nbsq = (size_t)kTsBS * kTsBS;
  double* P = const_cast<double*>(Dinv) + 3 * (size_t)nblk * nbsq;  // partial-sum slots
  // Persistent: each CTA draws tickets until they run out. A task only waits
  // for tasks with smaller tickets, drawn earlier by CTAs that are running, so
  // the grid may be smaller than the number of tasks.
  for (;;) {
  __syncthreads();  // the previous task's shared memory is no longer read
  if (tid == 0) {
    s_t = (int)atomicAdd(ticket, 1u);
    s_abort = 0;
  }
  __syncthreads();
  int t = s_t;
  // ticket -> (block s, helper c or owner), first ticket of block s
  int s = 0, first = 0;
  for (; s < nblk; ++s) {
    const int cnt = ti_helpers(s) + 1;
    if (t < first + cnt) break;
    first += cnt;
  }
  if (s >= nblk) return;
  const int c = t - first;
  const bool owner = c == ti_helpers(s);
  const int b = FWD ? s : nblk - 1 - s;
  const int r0 = b * kTsBS;
  const int nr = min(kTsBS, n - r0);
  const int r = tid & 63, g = tid >> 6;

  // y = sum over solve-order blocks s' in [lo, hi) of T(s, s') x_{s'}, into part
  // (thread (r, g): row r, columns g + 4i of each tile); the tile of the next
  // block is loaded while the current one waits for its x
  auto far_sum = [&](int lo, int hi) -> bool {
    auto load = [&](int sp, Ts (&v)[16]) {
      const int q = FWD ? sp : nblk - 1 - sp;
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
    if (lo < hi) load(lo, cur);
    for (int sp = lo; sp < hi; ++sp) {
      const int q = FWD ? sp : nblk - 1 - sp;
      const int c0 = q * kTsBS;
      const int nc = min(kTsBS, n - c0);
      Ts nxt[16];
      if (sp + 1 < hi) load(sp + 1, nxt);
      if (tid < kTsBS) {
        double v = 0.0;
        if (tid < nc && !ti_poll(X + c0 + tid, wait_ns, &v)) s_abort = 1;
        xq[tid] = v;
      }
      __syncthreads();
      if (s_abort) return false;
#pragma unroll
      for (int i = 0; i < 16; i += 2) {
        a0 = fma((double)cur[i], xq[g + 4 * i], a0);
        a1 = fma((double)cur[i + 1], xq[g + 4 * (i + 1)], a1);
      }
      if (sp + 1 < hi) {
#pragma unroll
        for (int i = 0; i < 16; ++i) cur[i] = nxt[i];
      }
      __syncthreads();  // xq is rewritten next step
    }
    part[g * kTsBS + r] = a0 + a1;
    __syncthreads();
    return true;
  };
  // part (4 x 64) -> one value per row, fixed order
  auto row_sum = [&](int rr) {
    return (part[rr] + part[kTsBS + rr]) + (part[2 * kTsBS + rr] + part[3 * kTsBS + rr]);
  };
  // part <- M (64 x 64, column-major, in mat) times xq
  auto mat_vec = [&]() {
    double a0 = 0.0, a1 = 0.0;
#pragma unroll
    for (int j = g * 16; j < g * 16 + 16; j += 2) {
      a0 = fma(mat[r + kTsBS * j], xq[j], a0);
      a1 = fma(mat[r + kTsBS * (j + 1)], xq[j + 1], a1);
    }
    part[g * kTsBS + r] = a0 + a1;
    __syncthreads();
  };
  auto load_mat = [&](const double* M) {
    for (int i = tid; i < kTsBS * kTsBS; i += blockDim.x) mat[i] = M[i];
  };
  auto wait_x = [&](int sp) -> bool {  // xq <- x of solve-order block sp
    const int q = FWD ? sp : nblk - 1 - sp;
    const int c0 = q * kTsBS;
    const int nc = min(kTsBS, n - c0);
    if (tid < kTsBS) {
      double v = 0.0;
      if (tid < nc && !ti_poll(X + c0 + tid, wait_ns, &v)) s_abort = 1;
      xq[tid] = v;
    }
    __syncthreads();
    return s_abort == 0;
  };

  if (!owner) {
    // helper: the far tiles of chunk c, published in slot t
    const int lo = c * kTiChunk, hi = min(lo + kTiChunk, s - 2);
    if (!far_sum(lo, hi)) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    if (tid < kTsBS) ti_announce(P + (size_t)t * kTsBS + tid, row_sum(tid));
    continue;
  }
  // owner of block s: rhs minus the helpers' chunks, in order
  load_mat(Dinv + (size_t)b * nbsq);
  if (tid < kTsBS) {
    double acc = tid < nr ? rhs[r0 + tid] : 0.0;
    for (int h = 0; h < c; ++h) {
      double v = 0.0;
      if (!ti_poll(P + (size_t)(first + h) * kTsBS + tid, wait_ns, &v)) s_abort = 1;
      acc -= v;
    }
    xq[tid] = tid < nr ? acc : 0.0;
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) gbla_flag_timeout(info);
    return;
  }
  mat_vec();  // D_s (rhs_s - far)
  if (tid < kTsBS) dv[tid] = row_sum(tid);
  __syncthreads();
  if (s >= 2) {
    load_mat(Dinv + nblk * nbsq * 2 + (size_t)b * nbsq);  // V_s
    if (!wait_x(s - 2)) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    mat_vec();
    if (tid < kTsBS) dv[tid] -= row_sum(tid);
    __syncthreads();
  }
  if (s >= 1) {
    load_mat(Dinv + nblk * nbsq + (size_t)b * nbsq);  // W_s
    if (!wait_x(s - 1)) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    mat_vec();
    if (tid < kTsBS) dv[tid] -= row_sum(tid);
    __syncthreads();
  }
  if (tid < nr) ti_announce(X + r0 + tid, dv[tid]);
  }
}

template <typename Ts>
cudaError_t launch_trsv_inv(bool lower, int n, const Ts* T, int ldt, const double* Dinv,
                            const double* rhs, double* X, unsigned* flags, int* info,
                            cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nblk = (n + kTsBS - 1) / kTsBS;
  const int tasks = ti_tasks(nblk);
  // The grid is persistent: as many CTAs as SMs (fewer when capped by
  // gbla_set_substitution_ctas), which the scheduler spreads one per SM, so
  // the FP64 units of an SM, which a block's chain step and the far tiles are
  // bound by, are not shared between two of them. Each CTA asks for the
  // shared memory it uses and no more, so kernels on other streams can share
  // an SM with a CTA that is waiting on the chain.
  const DeviceProps& dp = device_props();
  const size_t smem = sizeof(double) * ((size_t)kTsBS * kTsBS + 6 * kTsBS);
  int grid = dp.num_sms > 0 ? dp.num_sms : 1;
  const int cap = substitution_ctas();
  if (cap > 0 && cap < grid) grid = cap;
  if (grid > tasks) grid = tasks;
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(X, 0xff, sizeof(double) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  double* P = const_cast<double*>(Dinv) + (size_t)3 * nblk * kTsBS * kTsBS;
  e = cudaMemsetAsync(P, 0xff, sizeof(double) * (size_t)tasks * kTsBS, s);
  if (e != cudaSuccess) return e;
  const uint64_t wait_ns = wait_timeout_ns();
  if (lower) {
    e = ensure_dyn_smem(trsv_inv_kernel<Ts, true>, smem);
    if (e != cudaSuccess) return e;
    trsv_inv_kernel<Ts, true><<<grid, 256, smem, s>>>(n, T, ldt, Dinv, rhs, X, flags, info, wait_ns);
  } else {
    e = ensure_dyn_smem(trsv_inv_kernel<Ts, false>, smem);
    if (e != cudaSuccess) return e;
    trsv_inv_kernel<Ts, false><<<grid, 256, smem, s>>>(n, T, ldt, Dinv, rhs, X, flags, info, wait_ns);
  }
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_trsv_inv<float>(bool, int, const float*, int, const double*,
                                            const double*, double*, unsigned*, int*, cudaStream_t);
template cudaError_t launch_trsv_inv<double>(bool, int, const double*, int, const double*,
                                             const double*, double*, unsigned*, int*, cudaStream_t);

}  // namespace gbla
