// Panel factorisation with partial pivoting (paper section 2, the GEPP step of
// the blocked LU) and the row interchanges that go with it.
//
// Full-width panels of up to 16384 (FP32) or 4096 (FP64) rows run in one
// thread-block cluster (the cluster variant further down); the kernels
// described here take the others: an m x w panel (w <= 32) is spread over C
// cooperative CTAs, each holding a contiguous slab of R rows in the storage
// precision Ts, which is also the arithmetic precision (FP64 for the FP64
// factorisation; FP32 for the low-precision one, every operation rounded to
// FP32 as the working matrix is).
//
// Per column j:
//   1. each CTA finds its local argmax of |a_ij| over its rows i >= j
//      (warp-shuffle reduction of integer keys built from the IEEE bit
//      patterns of |a_ij|, which order like the values; ties -> lowest row);
//   2. it publishes its candidate row (and, if it owns row j, row j) and a
//      header (|v|, row) to its slot. Every 64-bit word carries a 32-bit tag
//      naming the launch and the column next to 32 bits of payload, so a
//      reader can tell a fresh word from a stale one without any fence;
//   3. thread q of every CTA polls slot q's header until it carries the
//      column's tag (bounded wait) -- the headers are the grid barrier -- and
//      the CTA reduces the C candidates to the global pivot p (same rule);
//   4. it reads the pivot row from the winner's slot (and old row j when it
//      owns row p), swaps rows j and p in its slab;
//   5. scales its multipliers l_ij = a_ij * (1 / a_jj) (i > j) and applies
//      the rank-1 update a_ik -= l_ij a_jk for k > j inside the panel.
// Slots are double-buffered by column parity: a CTA publishes column j + 2
// only after it has seen every header of column j + 1, which each CTA writes
// only after it has finished reading column j.
//
// Every panel launch also applies its interchanges to the other columns of
// the current outer block (nleft columns to the left of the panel, nright to
// its right) once its pivots are known; the columns outside the outer block
// get all the interchanges of the block at once from laswp_block_kernel,
// launched after the block's last panel. No CTA of any of these kernels waits
// for a CTA that the hardware does not schedule with it.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kPanelThreads = 256;
constexpr int kSlotRow = 4;  // words before the row words in a slot (3 header words + pad)

size_t panel_slots_doubles() { return kPanelExchangeDoubles + kInnerCounters / 2; }

typedef unsigned long long u64;

GBLA_DEVINL void st_relaxed_u64(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
GBLA_DEVINL u64 ld_relaxed_u64(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Wait (bounded) until the words at p[0..N) all carry `tag` in their upper
// halves; the N loads of one poll are independent, so a poll costs one round
// trip to L2.
template <int N>
GBLA_DEVINL bool ll_read(const u64* p, u64 tag, uint64_t wait_ns, uint32_t (&payload)[N]) {
  uint64_t t0 = 0;
  while (true) {
    u64 v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = ld_relaxed_u64(p + i);
    bool ok = true;
#pragma unroll
    for (int i = 0; i < N; ++i) ok = ok && ((v[i] & 0xffffffff00000000ull) == tag);
    if (ok) {
#pragma unroll
      for (int i = 0; i < N; ++i) payload[i] = (uint32_t)(v[i] & 0xffffffffull);
      return true;
    }
    const uint64_t now = gbla_now_ns();
    if (t0 == 0) t0 = now;
    else if (now - t0 > wait_ns) return false;
  }
}

// Pivot-search key: one 64-bit integer whose order is "larger |a|, then lower
// row index". FP32 values: (|a| bits << 32) | (2^32 - 1 - row). FP64 values
// need all 63 bits of |a|, so the row index travels beside the key.
template <typename Ts>
struct PivKey;
template <>
struct PivKey<float> {
  u64 k;
  GBLA_DEVINL PivKey() : k(0) {}
  GBLA_DEVINL static PivKey make(float a, int row) {
    PivKey p;
    p.k = ((u64)__float_as_uint(fabsf(a)) << 32) | (u64)(0xffffffffu - (unsigned)row);
    return p;
  }
  GBLA_DEVINL void merge(const PivKey& o) { k = o.k > k ? o.k : k; }
  GBLA_DEVINL void shfl_merge(int off) {
    PivKey o;
    o.k = __shfl_xor_sync(0xffffffffu, k, off);
    merge(o);
  }
  GBLA_DEVINL int row() const {
    return k ? (int)(0xffffffffu - (unsigned)(k & 0xffffffffull)) : INT_MAX;
  }
  GBLA_DEVINL bool zero_pivot() const { return (k >> 32) == 0; }
  GBLA_DEVINL bool valid() const { return k != 0; }
  GBLA_DEVINL bool same(const PivKey& o) const { return k == o.k; }
  GBLA_DEVINL void to_pair(u64& a, u64& b) const {
    a = k;
    b = 0;
  }
  GBLA_DEVINL static PivKey from_pair(u64 a, u64) {
    PivKey p;
    p.k = a;
    return p;
  }
  static constexpr int kWords = 2;
  GBLA_DEVINL void to_words(uint32_t (&w)[2]) const {
    w[0] = (uint32_t)(k & 0xffffffffull);
    w[1] = (uint32_t)(k >> 32);
  }
  GBLA_DEVINL static PivKey from_words(const uint32_t (&w)[2]) {
    PivKey p;
    p.k = ((u64)w[1] << 32) | w[0];
    return p;
  }
};
template <>
struct PivKey<double> {
  u64 k;
  int r;
  GBLA_DEVINL PivKey() : k(0), r(INT_MAX) {}
  GBLA_DEVINL static PivKey make(double a, int row) {
    PivKey p;
    p.k = (u64)__double_as_longlong(fabs(a));
    p.r = row;
    return p;
  }
  GBLA_DEVINL void merge(const PivKey& o) {
    if (o.k > k || (o.k == k && o.r < r)) {
      k = o.k;
      r = o.r;
    }
  }
  GBLA_DEVINL void shfl_merge(int off) {
    PivKey o;
    o.k = __shfl_xor_sync(0xffffffffu, k, off);
    o.r = __shfl_xor_sync(0xffffffffu, r, off);
    merge(o);
  }
  GBLA_DEVINL int row() const { return r; }
  GBLA_DEVINL bool zero_pivot() const { return k == 0; }
  GBLA_DEVINL bool valid() const { return r != INT_MAX; }
  GBLA_DEVINL bool same(const PivKey& o) const { return k == o.k && r == o.r; }
  GBLA_DEVINL void to_pair(u64& a, u64& b) const {
    a = k;
    b = (u64)(unsigned)r;
  }
  GBLA_DEVINL static PivKey from_pair(u64 a, u64 b) {
    PivKey p;
    p.k = a;
    p.r = (int)(unsigned)b;
    return p;
  }
  static constexpr int kWords = 3;
  GBLA_DEVINL void to_words(uint32_t (&w)[3]) const {
    w[0] = (uint32_t)(k & 0xffffffffull);
    w[1] = (uint32_t)(k >> 32);
    w[2] = (uint32_t)r;
  }
  GBLA_DEVINL static PivKey from_words(const uint32_t (&w)[3]) {
    PivKey p;
    p.k = ((u64)w[1] << 32) | w[0];
    p.r = (int)w[2];
    return p;
  }
};

template <typename Ts>
GBLA_DEVINL void warp_merge(PivKey<Ts>& p) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) p.shfl_merge(o);
}

// The same warp-wide argmax with the warp's integer max reduction (redux):
// the larger |a| bits first, then, among the lanes that hold them, the lower
// row. Every lane ends with the winning key. All 32 lanes must take part.
GBLA_DEVINL void warp_merge_redux(PivKey<float>& p) {
  const uint32_t hi = (uint32_t)(p.k >> 32), lo = (uint32_t)(p.k & 0xffffffffull);
  const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  const uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  p.k = ((u64)mhi << 32) | mlo;
}
GBLA_DEVINL void warp_merge_redux(PivKey<double>& p) {
  const uint32_t hi = (uint32_t)(p.k >> 32), lo = (uint32_t)(p.k & 0xffffffffull);
  const uint32_t mhi = __reduce_max_sync(0xffffffffu, hi);
  const uint32_t mlo = __reduce_max_sync(0xffffffffu, hi == mhi ? lo : 0u);
  // among equal |a|, the lowest row: the largest complement (an empty key's
  // row INT_MAX complements to the smallest value any holder can offer)
  const bool tie = hi == mhi && lo == mlo;
  const uint32_t nr = __reduce_max_sync(0xffffffffu, tie ? ~(uint32_t)p.r : 0u);
  p.k = ((u64)mhi << 32) | mlo;
  p.r = (int)~nr;
}

// ---------------------------------------------------------------------------
// Row interchanges of one panel applied to a column outside it, one warp per
// column (LAPACK laswp semantics: for l = 0 .. nw-1 in order, rows l and
// piv_l of the column are exchanged; rows relative to the panel's first row,
// piv_l >= l). Lane l holds piv_l. The plan is made once per warp: which of
// the touched rows -- the nw top rows and every distinct partner row below
// them -- ends up holding which row's old value. Applying it to a column is
// then one load and one store per touched row, the top rows coalesced.
//
// Slots: top slot t (t < nw) is row t; outside slot 32 + l is row piv_l for
// the first lane l naming a row piv_l >= nw. The plan simulates the nw
// exchanges on slot identities (ct, co: the slot whose old value ends up in
// this lane's top / outside slot).
struct LaswpPlan {
  int piv, nw, ct, co;
  bool out;  // this lane owns an outside slot
  GBLA_DEVINL void make(int piv_in, int nw_in, int lane) {
    nw = nw_in;
    piv = lane < nw ? piv_in : lane;
    const bool outside = lane < nw && piv >= nw;
    const unsigned same = __match_any_sync(0xffffffffu, outside ? piv : -1 - lane);
    const int f = __ffs(same) - 1;  // first lane naming the same outside row
    out = outside && f == lane;
    ct = lane;
    co = 32 + lane;
    for (int j = 0; j < nw; ++j) {
      const int pj = __shfl_sync(0xffffffffu, piv, j);
      const int fj = __shfl_sync(0xffffffffu, f, j);
      const bool top = pj < nw;
      const int a = __shfl_sync(0xffffffffu, ct, j);
      const int bt = __shfl_sync(0xffffffffu, ct, top ? pj : 0);
      const int bo = __shfl_sync(0xffffffffu, co, top ? 0 : fj);
      const int b = top ? bt : bo;
      if (top) {
        if (lane == pj) ct = a;
      } else if (lane == fj) {
        co = a;
      }
      if (lane == j) ct = b;
    }
  }
  // col: the column's element in the panel's first row
  template <typename T>
  GBLA_DEVINL void apply(T* col, int lane) const {
    const T vt = lane < nw ? col[lane] : (T)0;
    const T vo = out ? col[piv] : (T)0;
    store(col, lane, vt, vo);
  }
  // U columns at once: every load is issued before the first store, so the
  // loads of the U columns are in flight together
  template <typename T, int U>
  GBLA_DEVINL void apply_n(T* const (&cols)[U], int lane) const {
    T vt[U], vo[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      vt[u] = (cols[u] && lane < nw) ? cols[u][lane] : (T)0;
      vo[u] = (cols[u] && out) ? cols[u][piv] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (cols[u]) store(cols[u], lane, vt[u], vo[u]);
  }
  template <typename T>
  GBLA_DEVINL void store(T* col, int lane, T vt, T vo) const {
    const T x1 = __shfl_sync(0xffffffffu, vt, ct & 31);
    const T x2 = __shfl_sync(0xffffffffu, vo, ct & 31);
    const T y1 = __shfl_sync(0xffffffffu, vt, co & 31);
    const T y2 = __shfl_sync(0xffffffffu, vo, co & 31);
    if (lane < nw) col[lane] = ct < 32 ? x1 : x2;
    if (out) col[piv] = co < 32 ? y1 : y2;
  }
};

// The panel's interchanges on the other columns of its outer block: columns
// -nleft .. -1 and w .. w + nright - 1 relative to the panel (A = its
// top-left element), warp g of G.
template <typename Ts>
GBLA_DEVINL void panel_tail_swaps(Ts* A, int lda, int w, int nleft, int nright, const LaswpPlan& plan,
                                  int g, int G, int lane) {
  const int nt = nleft + nright;
  for (int q0 = 2 * g; q0 < nt; q0 += 2 * G) {
    Ts* cols[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int q = q0 + u;
      const long long col = q < nleft ? (long long)q - nleft : (long long)w + (q - nleft);
      cols[u] = q < nt ? A + col * lda : nullptr;
    }
    plan.apply_n<Ts, 2>(cols, lane);
  }
}

// Interchanges of one outer block (ipiv[0 .. kb), 1-based absolute rows, the
// block starting at row k0; kb <= 256) applied to columns [0, skip_lo) and
// [skip_hi, ncols) of the nrows x ncols matrix (LAPACK laswp semantics, in
// order). Every CTA first works out where each touched row's final value
// comes from (swap_plan): thread t holds at most two (destination, source)
// pairs, block row t and the partner row its interchange names last. Then,
// for a tile of columns, each thread loads the sources of its pairs in every
// column of the tile into registers, the CTA meets at a barrier, and each
// thread stores them to the destinations: a gather followed by a scatter, one
// address per element; the block's rows are consecutive lanes. Rows that keep
// their value are skipped. Columns are never shared between CTAs; no waits.
// Pivots outside [row t, nrows) are ignored.
template <typename T>
__global__ void __launch_bounds__(256)
    laswp_block_kernel(T* __restrict__ A, int lda, int ncols, int nrows, int k0, int kb,
                       const int* __restrict__ ipiv, int skip_lo, int skip_hi) {
  constexpr int LC = sizeof(T) == 4 ? 32 : 16;  // columns per tile
  __shared__ SwapPlanShared s_plan;
  const int tid = threadIdx.x;
  const int R = nrows - k0;
  if (tid < kb) {
    int p = ipiv[tid] - 1 - k0;
    if (p < tid || p >= R) p = tid;
    s_plan.p[tid] = p;
  }
  __syncthreads();
  int src_b = tid, dst_o = -1, src_o = 0;
  swap_plan(s_plan, kb, tid, &src_b, &dst_o, &src_o);
  int dr[2], sr[2];
  dr[0] = (tid < kb && src_b != tid) ? tid : -1;
  sr[0] = src_b;
  dr[1] = dst_o;
  sr[1] = src_o;
  const int skip = skip_hi - skip_lo;
  const int nfar = ncols - skip;
  const int ntiles = (nfar + LC - 1) / LC;
  T* base = A + k0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int q0 = tile * LC;
    T v[2][LC];
#pragma unroll
    for (int c = 0; c < LC; ++c) {
      const int q = q0 + c;
      const int col = q < skip_lo ? q : q + skip;
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (q < nfar && dr[u] >= 0) v[u][c] = base[(size_t)col * lda + sr[u]];
    }
    __syncthreads();  // every read of the tile's columns before any write
#pragma unroll
    for (int c = 0; c < LC; ++c) {
      const int q = q0 + c;
      const int col = q < skip_lo ? q : q + skip;
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (q < nfar && dr[u] >= 0) base[(size_t)col * lda + dr[u]] = v[u][c];
    }
  }
}

template <typename T>
cudaError_t launch_laswp_block(T* A, int lda, int ncols, int nrows, int k0, int kb, const int* ipiv,
                               int skip_lo, int skip_hi, cudaStream_t s) {
  const int nfar = ncols - (skip_hi - skip_lo);
  if (nfar <= 0 || kb <= 0) return cudaSuccess;
  if (kb > 256) return cudaErrorInvalidValue;
  const DeviceProps& dp = device_props();
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, laswp_block_kernel<T>, 256, 0) !=
          cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  constexpr int LC = sizeof(T) == 4 ? 32 : 16;
  const int ntiles = (nfar + LC - 1) / LC;
  int grid = per_sm * (dp.num_sms > 0 ? dp.num_sms : 1);
  if (grid > ntiles) grid = ntiles;
  laswp_block_kernel<T><<<grid, 256, 0, s>>>(A, lda, ncols, nrows, k0, kb, ipiv, skip_lo, skip_hi);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_laswp_block<double>(double*, int, int, int, int, int, const int*, int,
                                                int, cudaStream_t);
template cudaError_t launch_laswp_block<float>(float*, int, int, int, int, int, const int*, int, int,
                                               cudaStream_t);

// ---------------------------------------------------------------------------
// Interchanges of the columns left of each outer block, applied once after
// the last block instead of block by block: a column of block b needs the
// interchanges of every later block c > b on its rows q >= k_{b+1}. With
// sigma_c the map "row q receives the old value of row sigma_c(q)" of block
// c's interchanges (the identity outside the rows they touch), the final value
// of row q comes from row tau_b(q) = sigma_{b+1}(sigma_{b+2}(...(q))).
//
// left_perm_kernel (one CTA): sigma_c is formed from block c's interchanges by
// swap_plan and written into an identity array in shared memory;
// tau is composed from the last block backwards, tau <- sigma_c o tau, and
// tau_{c-1} is stored for every block c >= 1 (rows >= k_c; the rest of the
// row range is not read). Pivots outside [row, n) are ignored, as everywhere.
__global__ void __launch_bounds__(1024)
    left_perm_kernel(int n, int nb, const int* __restrict__ ipiv, int* __restrict__ tau,
                     int* __restrict__ snaps) {
  extern __shared__ int lp_D[];  // n entries
  __shared__ SwapPlanShared s_plan;
  const int tid = threadIdx.x;
  for (int q = tid; q < n; q += blockDim.x) {
    lp_D[q] = q;
    tau[q] = q;
  }
  __syncthreads();
  const int nblk = (n + nb - 1) / nb;
  for (int c = nblk - 1; c >= 1; --c) {
    const int k0 = c * nb, kb = min(nb, n - k0);
    if (tid < kb) {
      int p = ipiv[k0 + tid] - 1 - k0;
      if (p < tid || p >= n - k0) p = tid;
      s_plan.p[tid] = p;
    }
    __syncthreads();
    int src_b = tid, dst_o = -1, src_o = 0;
    swap_plan(s_plan, kb, tid, &src_b, &dst_o, &src_o);
    if (tid < kb) {
      lp_D[k0 + tid] = k0 + src_b;
      if (dst_o >= 0) lp_D[k0 + dst_o] = k0 + src_o;
    }
    __syncthreads();
    int* snap = snaps + (size_t)(c - 1) * n;
    for (int q = k0 + tid; q < n; q += blockDim.x) {
      const int v = lp_D[tau[q]];
      tau[q] = v;
      snap[q] = v;
    }
    __syncthreads();
    // back to the identity on the rows block c touched
    if (tid < kb) {
      lp_D[k0 + tid] = k0 + tid;
      if (dst_o >= 0) lp_D[k0 + dst_o] = k0 + dst_o;
    }
    __syncthreads();
  }
}

// left_gather_kernel: CTA x = column x of blocks 0 .. nblk-2; rows
// [k_{b+1}, n) of the column are staged in shared memory and written back
// through tau_b (coalesced loads and stores).
template <typename T>
__global__ void __launch_bounds__(256)
    left_gather_kernel(T* __restrict__ A, int lda, int n, int nb, const int* __restrict__ snaps) {
  extern __shared__ double lg_smem[];
  T* seg = reinterpret_cast<T*>(lg_smem);
  const int col = blockIdx.x;
  const int b = col / nb;
  const int r0 = (b + 1) * nb;
  const int len = n - r0;
  if (len <= 0) return;
  T* a = A + (size_t)col * lda + r0;
  const int* tb = snaps + (size_t)b * n + r0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) seg[i] = a[i];
  __syncthreads();
  for (int i = threadIdx.x; i < len; i += blockDim.x) a[i] = seg[tb[i] - r0];
}

size_t left_perm_ints(int n, int nb) {
  const int nblk = (n + nb - 1) / nb;
  return nblk >= 2 ? (size_t)n * (size_t)nblk : 0;  // tau + (nblk - 1) snapshots
}

template <typename T>
bool left_deferred_fits(int n, int nb) {
  const DeviceProps& dp = device_props();
  return (size_t)n * sizeof(int) <= dp.smem_optin && (size_t)n * sizeof(T) <= dp.smem_optin &&
         n > nb;
}
template bool left_deferred_fits<double>(int, int);
template bool left_deferred_fits<float>(int, int);

template <typename T>
cudaError_t launch_left_interchanges(T* A, int lda, int n, int nb, const int* ipiv, int* work,
                                     cudaStream_t s) {
  const int nblk = (n + nb - 1) / nb;
  if (nblk < 2) return cudaSuccess;
  int* tau = work;
  int* snaps = work + n;
  const size_t sm_d = (size_t)n * sizeof(int);
  cudaError_t e = ensure_dyn_smem(left_perm_kernel, sm_d);
  if (e != cudaSuccess) return e;
  left_perm_kernel<<<1, 1024, sm_d, s>>>(n, nb, ipiv, tau, snaps);
  count_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm_g = (size_t)(n - nb) * sizeof(T);
  e = ensure_dyn_smem(left_gather_kernel<T>, sm_g);
  if (e != cudaSuccess) return e;
  left_gather_kernel<T><<<(nblk - 1) * nb, 256, sm_g, s>>>(A, lda, n, nb, snaps);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_left_interchanges<double>(double*, int, int, int, const int*, int*,
                                                      cudaStream_t);
template cudaError_t launch_left_interchanges<float>(float*, int, int, int, const int*, int*,
                                                     cudaStream_t);

// The exchange area holds two parities of slots for up to kPanelMaxSms CTAs;
// the launcher never uses more CTAs than that.
static_assert(kPanelExchangeDoubles == (size_t)2 * (kPanelMaxSms + 1) * kPanelSlotW,
              "exchange area sized for kPanelMaxSms CTAs");

template <typename Ts>
__global__ void __launch_bounds__(kPanelThreads)
    panel_kernel(Ts* __restrict__ A, int lda, int m, int w, int row0, int R,
                 int* __restrict__ ipiv, int* __restrict__ info, double* __restrict__ slots_d,
                 unsigned tag_base, uint64_t wait_ns, int nleft, int nright) {
  typedef PivKey<Ts> Key;
  constexpr int KW = Key::kWords;
  extern __shared__ double smem[];
  Ts* slab = reinterpret_cast<Ts*>(smem);       // [w][R], column-major slab
  Ts* prow = slab + (size_t)w * R;              // pivot row (w)
  Ts* rj = prow + kPanelWidth;                  // old row j (w)
  // raw storage: a __shared__ object is never constructed
  __shared__ alignas(16) unsigned char s_wk_raw[sizeof(Key) * (kPanelThreads / 32)];
  __shared__ alignas(16) unsigned char s_key_raw[sizeof(Key)];
  Key* s_wk = reinterpret_cast<Key*>(s_wk_raw);
  Key& s_key = *reinterpret_cast<Key*>(s_key_raw);
  __shared__ Ts s_rp;
  __shared__ int s_abort;

  u64* slots = reinterpret_cast<u64*>(slots_d);
  const int C = gridDim.x;
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int rbeg = c * R;
  const int rcnt = max(0, min(R, m - rbeg));
  u64* rowj_buf = slots + (size_t)2 * C * kPanelSlotW;

  for (int k = 0; k < w; ++k)
    for (int r = tid; r < rcnt; r += blockDim.x)
      slab[k * R + r] = A[(size_t)k * lda + rbeg + r];
  if (tid == 0) s_abort = 0;
  // pivots start as "no interchange", so that an aborted launch leaves only
  // in-range row indices behind for the kernels that follow
  if (c == 0)
    for (int j = tid; j < min(w, m); j += blockDim.x) ipiv[j] = row0 + j + 1;
  __syncthreads();

  const int jend = min(w, m);
  int my_piv = lane;  // lane l: the partner row of column l
  for (int j = 0; j < jend; ++j) {
    const int par = j & 1;
    const u64 tag = (u64)(tag_base | (unsigned)(j + 1)) << 32;
    // 1. local argmax over own rows with panel row >= j
    Key bk;
    for (int r = tid; r < rcnt; r += blockDim.x)
      if (rbeg + r >= j) bk.merge(Key::make(slab[j * R + r], rbeg + r));
    warp_merge<Ts>(bk);
    if (lane == 0) s_wk[warp] = bk;
    __syncthreads();
    if (warp == 0) {
      bk = lane < nwarps ? s_wk[lane] : Key();
      warp_merge<Ts>(bk);
      if (lane == 0) s_key = bk;
    }
    __syncthreads();
    // 2. publish: candidate row and row j as tagged 32-bit halves, header last
    u64* myslot = slots + ((size_t)par * C + c) * kPanelSlotW;
    const Key lk = s_key;
    const int lb = lk.row();
    if (tid < 2 * w) {
      const int k = tid >> 1;
      if (lb != INT_MAX) {
        const u64 bits = (u64)__double_as_longlong((double)slab[k * R + (lb - rbeg)]);
        st_relaxed_u64(myslot + kSlotRow + tid,
                       tag | ((tid & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      }
      if (j >= rbeg && j < rbeg + rcnt) {
        const u64 bits = (u64)__double_as_longlong((double)slab[k * R + (j - rbeg)]);
        st_relaxed_u64(rowj_buf + par * kPanelSlotW + tid,
                       tag | ((tid & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      }
    }
    if (tid == 0) {
      uint32_t hw[KW];
      lk.to_words(hw);
#pragma unroll
      for (int i = 0; i < KW; ++i) st_relaxed_u64(myslot + i, tag | hw[i]);
    }
    // 3. thread q polls header q; block-wide argmax of the C candidates
    bk = Key();
    bool ok = true;
    for (int q = tid; q < C; q += blockDim.x) {
      uint32_t hw[KW];
      ok = ll_read<KW>(slots + ((size_t)par * C + q) * kPanelSlotW, tag, wait_ns, hw);
      if (!ok) break;
      bk.merge(Key::from_words(hw));
    }
    if (!ok) s_abort = 1;
    warp_merge<Ts>(bk);
    if (lane == 0) s_wk[warp] = bk;
    __syncthreads();
    if (s_abort) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    if (warp == 0) {
      bk = lane < nwarps ? s_wk[lane] : Key();
      warp_merge<Ts>(bk);
      if (lane == 0) s_key = bk;
    }
    __syncthreads();
    const Key gk = s_key;
    const int p = gk.row();
    if (lane == j) my_piv = p;
    const int cw = p / R;  // the CTA that owns row p published it
    const bool own_j = (j >= rbeg && j < rbeg + rcnt);
    const bool own_p = (p >= rbeg && p < rbeg + rcnt);
    // 4. pivot row from the winner's slot; old row j when this CTA owns row p
    if (warp < 2) {  // whole warps, so that the pair shuffles see every lane
      const bool act = tid < 2 * w;
      const u64* wrow = slots + ((size_t)par * C + cw) * kPanelSlotW + kSlotRow;
      uint32_t half[1] = {0};
      bool okr = act ? ll_read<1>(wrow + tid, tag, wait_ns, half) : true;
      uint32_t other = __shfl_xor_sync(0xffffffffu, half[0], 1);
      if (act && (tid & 1) == 0) {
        const double v = __longlong_as_double((long long)(((u64)other << 32) | half[0]));
        prow[tid >> 1] = (Ts)v;
        if ((tid >> 1) == j) s_rp = v != 0.0 ? (Ts)1 / (Ts)v : (Ts)0;
      }
      if (p != j && own_p) {
        if (act) okr = ll_read<1>(rowj_buf + par * kPanelSlotW + tid, tag, wait_ns, half) && okr;
        other = __shfl_xor_sync(0xffffffffu, half[0], 1);
        if (act && (tid & 1) == 0)
          rj[tid >> 1] = (Ts)__longlong_as_double((long long)(((u64)other << 32) | half[0]));
      }
      if (!okr) s_abort = 1;
    }
    if (c == 0 && tid == 0) {
      ipiv[j] = row0 + p + 1;
      if (gk.zero_pivot()) atomicCAS(info, 0, row0 + j + 1);
    }
    __syncthreads();
    if (s_abort) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    if (p != j && tid < w) {
      if (own_j) slab[tid * R + (j - rbeg)] = prow[tid];
      if (own_p) slab[tid * R + (p - rbeg)] = rj[tid];
    }
    __syncthreads();
    // 5. scale by the reciprocal pivot and rank-1 update of own rows below it
    //    (the pivot row is held in registers; the k loop is unrolled)
    const Ts rp = s_rp;
    const bool nz = prow[j] != (Ts)0;
    Ts pr[kPanelWidth];
#pragma unroll
    for (int k = 0; k < kPanelWidth; ++k) pr[k] = k < w ? prow[k] : (Ts)0;
    for (int r = tid; r < rcnt; r += blockDim.x) {
      if (rbeg + r > j) {
        Ts l = slab[j * R + r];
        if (nz) {
          l = l * rp;
          slab[j * R + r] = l;
        }
#pragma unroll
        for (int k = 0; k < kPanelWidth; ++k)
          if (k > j && k < w) slab[k * R + r] = fma(-l, pr[k], slab[k * R + r]);
      }
    }
    __syncthreads();
  }
  for (int k = 0; k < w; ++k)
    for (int r = tid; r < rcnt; r += blockDim.x)
      A[(size_t)k * lda + rbeg + r] = slab[k * R + r];
  if (nleft + nright > 0) {
    LaswpPlan plan;
    plan.make(my_piv, jend, lane);
    panel_tail_swaps<Ts>(A, lda, w, nleft, nright, plan, c * nwarps + warp, C * nwarps, lane);
  }
}

// Register-resident variant: thread t of a CTA holds rows t, t + 256, ...
// (RPT rows) of its slab, all kPanelWidth columns, in registers; the column
// loop is unrolled so every register index is a constant. Same exchange
// protocol and same arithmetic as panel_kernel; used when a CTA's slab has at
// most 256 * RPT rows.
template <typename Ts, int RPT>
__global__ void __launch_bounds__(kPanelThreads, 1)
    panel_reg_kernel(Ts* __restrict__ A, int lda, int m, int w, int row0, int R,
                     int* __restrict__ ipiv, int* __restrict__ info, double* __restrict__ slots_d,
                     unsigned tag_base, uint64_t wait_ns, int nleft, int nright) {
  typedef PivKey<Ts> Key;
  constexpr int KW = Key::kWords;
  constexpr int W = kPanelWidth;
  __shared__ Ts prow[W], rj[W], crow[W], jrow[W];
  // raw storage: a __shared__ object is never constructed
  __shared__ alignas(16) unsigned char s_wk_raw[sizeof(Key) * (kPanelThreads / 32)];
  __shared__ alignas(16) unsigned char s_key_raw[sizeof(Key)];
  Key* s_wk = reinterpret_cast<Key*>(s_wk_raw);
  Key& s_key = *reinterpret_cast<Key*>(s_key_raw);
  __shared__ Ts s_rp;
  __shared__ int s_abort;

  u64* slots = reinterpret_cast<u64*>(slots_d);
  const int C = gridDim.x;
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int nwarps = blockDim.x >> 5;
  const int rbeg = c * R;
  const int rcnt = max(0, min(R, m - rbeg));
  u64* rowj_buf = slots + (size_t)2 * C * kPanelSlotW;

  Ts a[RPT][W];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + kPanelThreads * i;
#pragma unroll
    for (int k = 0; k < W; ++k)
      a[i][k] = (r < rcnt && k < w) ? A[(size_t)k * lda + rbeg + r] : (Ts)0;
  }
  if (tid == 0) s_abort = 0;
  if (c == 0)
    for (int j = tid; j < min(w, m); j += blockDim.x) ipiv[j] = row0 + j + 1;
  __syncthreads();

  const int jend = min(w, m);
  int my_piv = lane;  // lane l: the partner row of column l
#pragma unroll
  for (int j = 0; j < W; ++j) {
    if (j < jend) {
      const int par = j & 1;
      const u64 tag = (u64)(tag_base | (unsigned)(j + 1)) << 32;
      // 1. local argmax
      Key bk;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = tid + kPanelThreads * i;
        if (r < rcnt && rbeg + r >= j) bk.merge(Key::make(a[i][j], rbeg + r));
      }
      warp_merge<Ts>(bk);
      if (lane == 0) s_wk[warp] = bk;
      __syncthreads();
      if (warp == 0) {
        bk = lane < nwarps ? s_wk[lane] : Key();
        warp_merge<Ts>(bk);
        if (lane == 0) s_key = bk;
      }
      __syncthreads();
      // 2. publish: the owners of the local candidate row and of row j copy
      //    them to shared memory; 64 threads per row then write the tagged
      //    halves in parallel; thread 0 writes the header
      u64* myslot = slots + ((size_t)par * C + c) * kPanelSlotW;
      const Key lk = s_key;
      const int lb = lk.row();
      const bool have_j = (j >= rbeg && j < rbeg + rcnt);
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = tid + kPanelThreads * i;
        if (lb != INT_MAX && r == lb - rbeg) {
#pragma unroll
          for (int k = 0; k < W; ++k) crow[k] = a[i][k];
        }
        if (have_j && r == j - rbeg) {
#pragma unroll
          for (int k = 0; k < W; ++k) jrow[k] = a[i][k];
        }
      }
      __syncthreads();
      if (tid < 2 * w && lb != INT_MAX) {
        const u64 bits = (u64)__double_as_longlong((double)crow[tid >> 1]);
        st_relaxed_u64(myslot + kSlotRow + tid, tag | ((tid & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      } else if (tid >= 64 && tid < 64 + 2 * w && have_j) {
        const int t = tid - 64;
        const u64 bits = (u64)__double_as_longlong((double)jrow[t >> 1]);
        st_relaxed_u64(rowj_buf + par * kPanelSlotW + t, tag | ((t & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      }
      if (tid == 0) {
        uint32_t hw[KW];
        lk.to_words(hw);
#pragma unroll
        for (int i = 0; i < KW; ++i) st_relaxed_u64(myslot + i, tag | hw[i]);
      }
      // 3. poll the C headers; block-wide argmax
      bk = Key();
      bool ok = true;
      for (int q = tid; q < C; q += blockDim.x) {
        uint32_t hw[KW];
        ok = ll_read<KW>(slots + ((size_t)par * C + q) * kPanelSlotW, tag, wait_ns, hw);
        if (!ok) break;
        bk.merge(Key::from_words(hw));
      }
      if (!ok) s_abort = 1;
      warp_merge<Ts>(bk);
      if (lane == 0) s_wk[warp] = bk;
      __syncthreads();
      if (s_abort) {
        if (tid == 0) gbla_flag_timeout(info);
        return;
      }
      if (warp == 0) {
        bk = lane < nwarps ? s_wk[lane] : Key();
        warp_merge<Ts>(bk);
        if (lane == 0) s_key = bk;
      }
      __syncthreads();
      const Key gk = s_key;
      const int p = gk.row();
      if (lane == j) my_piv = p;
      const int cw = p / R;
      const bool own_p = (p >= rbeg && p < rbeg + rcnt);
      // 4. pivot row (and old row j for the owner of row p)
      if (warp < 2) {
        const bool act = tid < 2 * w;
        const u64* wrow = slots + ((size_t)par * C + cw) * kPanelSlotW + kSlotRow;
        uint32_t half[1] = {0};
        bool okr = act ? ll_read<1>(wrow + tid, tag, wait_ns, half) : true;
        uint32_t other = __shfl_xor_sync(0xffffffffu, half[0], 1);
        if (act && (tid & 1) == 0) {
          const double v = __longlong_as_double((long long)(((u64)other << 32) | half[0]));
          prow[tid >> 1] = (Ts)v;
          if ((tid >> 1) == j) s_rp = v != 0.0 ? (Ts)1 / (Ts)v : (Ts)0;
        }
        if (p != j && own_p) {
          if (act) okr = ll_read<1>(rowj_buf + par * kPanelSlotW + tid, tag, wait_ns, half) && okr;
          other = __shfl_xor_sync(0xffffffffu, half[0], 1);
          if (act && (tid & 1) == 0)
            rj[tid >> 1] = (Ts)__longlong_as_double((long long)(((u64)other << 32) | half[0]));
        }
        if (!okr) s_abort = 1;
      }
      if (c == 0 && tid == 0) {
        ipiv[j] = row0 + p + 1;
        if (gk.zero_pivot()) atomicCAS(info, 0, row0 + j + 1);
      }
      if (tid >= kPanelWidth * 2 && tid < kPanelWidth * 2 + kPanelWidth)  // pad columns >= w
        if (tid - 2 * kPanelWidth >= w) prow[tid - 2 * kPanelWidth] = (Ts)0;
      __syncthreads();
      if (s_abort) {
        if (tid == 0) gbla_flag_timeout(info);
        return;
      }
      // 5. swap rows j and p, scale, rank-1 update (registers)
      const Ts rp = s_rp;
      const bool nz = prow[j] != (Ts)0;
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int r = tid + kPanelThreads * i;
        if (r < rcnt) {
          const int gi = rbeg + r;
          if (p != j && gi == j) {
#pragma unroll
            for (int k = 0; k < W; ++k) a[i][k] = prow[k];
          } else if (p != j && gi == p) {
#pragma unroll
            for (int k = 0; k < W; ++k) a[i][k] = rj[k];
          }
          if (gi > j) {
            Ts l = a[i][j];
            if (nz) {
              l = l * rp;
              a[i][j] = l;
            }
#pragma unroll
            for (int k = j + 1; k < W; ++k) a[i][k] = fma(-l, prow[k], a[i][k]);
          }
        }
      }
      __syncthreads();  // prow / rj / s_key are rewritten in the next column
    }
  }
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int r = tid + kPanelThreads * i;
#pragma unroll
    for (int k = 0; k < W; ++k)
      if (r < rcnt && k < w) A[(size_t)k * lda + rbeg + r] = a[i][k];
  }
  if (nleft + nright > 0) {
    LaswpPlan plan;
    plan.make(my_piv, jend, lane);
    panel_tail_swaps<Ts>(A, lda, w, nleft, nright, plan, c * nwarps + warp, C * nwarps, lane);
  }
}

// ---------------------------------------------------------------------------
// Cluster variant. The panel rows are spread over the CL CTAs (CL <= 16) of
// one thread-block cluster -- the whole grid, scheduled together by the
// hardware -- RPT (1 or 2) rows per thread, all kPanelWidth columns in
// registers; the three argmax levels (thread -> warp -> CTA -> cluster) use
// the warp's integer max reduction. The per-column exchange stays inside the
// cluster: every CTA pushes its candidate (pivot key + row) into the shared
// memory of every CTA of the cluster with a bulk copy, completing bytes on
// the receiver's mbarrier, and CTA 0 pushes old row j the same way; each CTA
// then waits on its own mbarrier alone and reduces the CL candidates locally.
// Nothing goes through global memory.
//
// Buffers are double-buffered by column parity. A CTA pushes column j + 2
// only after it has received every CTA's column j + 1 message, and each CTA
// sends that message only after it has finished reading its column j
// buffers; a CTA re-arms the mbarrier of column j + 2 before it sends its own
// column j + 1 message, so the transaction count is always armed before any
// byte of that column can arrive. Hence, whenever a CTA stops, copies can be
// on their way into it for at most the two columns its two mbarriers are
// armed for.
//
// Leaving. Whether the panel finished or a wait gave up, every CTA tells
// every other how many columns it pushed (shared-memory stores across the
// cluster, made visible by a cluster barrier). From those counts a CTA knows
// exactly how many bytes will still arrive for each armed column; it
// completes the bytes that never will on its own mbarrier, waits (bounded)
// for the phase to finish -- i.e. for every copy in flight into it to land --
// and only then meets the others at a second cluster barrier. After that no
// copy reads or writes the shared memory of any CTA of the cluster, so all
// may exit.
constexpr int kClMax = 16;

template <typename Ts>
struct alignas(16) ClMsg {
  u64 k;                 // pivot key words (PivKey::to_pair)
  u64 r;
  Ts v[kPanelWidth];     // the candidate row
};

GBLA_DEVINL uint32_t cl_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
GBLA_DEVINL uint32_t cl_mapa(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// Bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to
// another CTA's, completing the bytes on that CTA's mbarrier.
GBLA_DEVINL void cl_bulk_push(uint32_t rdst, uint32_t src, uint32_t bytes, uint32_t rbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          rdst),
      "r"(src), "r"(bytes), "r"(rbar)
      : "memory");
}
GBLA_DEVINL void cl_store_remote_u32(uint32_t raddr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(raddr), "r"(v) : "memory");
}
GBLA_DEVINL void cl_fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
GBLA_DEVINL void cl_mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
GBLA_DEVINL void cl_mbar_arm(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// Count `bytes` as arrived on this CTA's mbarrier (bytes that no copy will bring).
GBLA_DEVINL void cl_mbar_complete_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
GBLA_DEVINL bool cl_mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
GBLA_DEVINL bool cl_mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity. A limit of 0 does not wait
// at all (one non-blocking test), so that "give up at once" is what it says:
// try_wait may itself suspend the thread for a while before it answers.
GBLA_DEVINL bool cl_mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (limit_ns == 0) return cl_mbar_test(bar, parity);
  if (cl_mbar_try(bar, parity)) return true;
  const uint64_t t0 = gbla_now_ns();
  while (!cl_mbar_try(bar, parity))
    if (gbla_now_ns() - t0 > limit_ns) return false;
  return true;
}
GBLA_DEVINL uint32_t cl_nctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
GBLA_DEVINL uint32_t cl_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
GBLA_DEVINL void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Correctly rounded reciprocal (the value 1 / x rounds to, as the division
// gives it, in fewer instructions).
GBLA_DEVINL float rcp_rn(float x) { return __frcp_rn(x); }
GBLA_DEVINL double rcp_rn(double x) { return __drcp_rn(x); }

template <typename Ts, int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
    panel_cluster_kernel(Ts* __restrict__ A, int lda, int m, int row0, int* __restrict__ ipiv,
                         int* __restrict__ info, uint64_t wait_ns, int nleft, int nright, int CL) {
  typedef PivKey<Ts> Key;
  constexpr int W = kPanelWidth;
  constexpr int NW = NT / 32;
  __shared__ ClMsg<Ts> s_warp[2][NW];                  // each warp's winner (key + row)
  __shared__ ClMsg<Ts> s_recv[2][kClMax];              // candidates pushed by the cluster
  __shared__ alignas(16) Ts s_rowj[2][W];              // row j staged by its owner
  __shared__ alignas(16) Ts s_rowj_recv[2][W];         // row j pushed by CTA 0
  __shared__ alignas(8) u64 s_bar[2];
  __shared__ unsigned s_pushed[kClMax];                // columns each CTA pushed (for leaving)

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // pivots start as "no interchange" before anything can fail, so that an
  // aborted launch leaves only in-range row indices behind
  if (blockIdx.x == 0 && tid < W) ipiv[tid] = row0 + tid + 1;
  // every shared-memory address below is mapped into CTAs 0 .. CL - 1 of this
  // cluster: a launch whose cluster is not the CL-CTA grid (never made by this
  // library's launcher) touches no other CTA and reports a failed wait
  if (cl_nctarank() != (uint32_t)CL || cl_ctarank() != blockIdx.x || gridDim.x != (unsigned)CL) {
    if (tid == 0) gbla_flag_timeout(info);
    return;
  }
  const int c = blockIdx.x;  // rank in the cluster
  const int g0 = c * NT * RPT + tid;  // panel row of this thread's row i: g0 + i * NT
  const uint32_t kExpect = (uint32_t)(CL * sizeof(ClMsg<Ts>) + W * sizeof(Ts));

  Ts a[RPT][W];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int gi = g0 + i * NT;
#pragma unroll
    for (int k = 0; k < W; ++k) a[i][k] = gi < m ? A[(size_t)k * lda + gi] : (Ts)0;
  }
  const uint32_t bar[2] = {cl_smem_u32(&s_bar[0]), cl_smem_u32(&s_bar[1])};
  if (tid == 0) {
    cl_mbar_init(bar[0], 1);
    cl_mbar_init(bar[1], 1);
    cl_mbar_arm(bar[0], kExpect);
    cl_mbar_arm(bar[1], kExpect);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  cl_sync();  // every mbarrier initialised and armed before the first push

  int my_fail = 0;             // this thread's wait gave up
  bool aborted = false;        // uniform over the CTA
  int npushed = 0;             // columns this CTA pushed (uniform)
  int armed[2] = {0, 1};       // thread 0: the column each mbarrier is armed for
  int my_piv = lane;           // lane l: the partner row of column l
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const int par = j & 1;
    // 1. candidate of this thread (ties -> lower row), warp argmax; the
    //    winning lane stages its key and row; thread j of CTA 0 (which owns
    //    panel row j) stages row j
    Key bk;
    int ib = 0;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gi = g0 + i * NT;
      if (gi < m && gi >= j) {
        const Key ki = Key::make(a[i][j], gi);
        if (!bk.valid()) {
          bk = ki;
          ib = i;
        } else {
          Key t = bk;
          t.merge(ki);
          if (!t.same(bk)) {
            bk = ki;
            ib = i;
          }
        }
      }
    }
    Key wk = bk;
    warp_merge_redux(wk);
    ClMsg<Ts>& mine = s_warp[par][warp];
    // A thread whose wait of column j - 1 gave up stages nothing: only a
    // completed column j - 1 proves that every copy of column j - 2 (which
    // read this buffer) has landed. The CTA stops at the barrier below.
    if (my_fail) {
    } else if (bk.valid() && bk.same(wk)) {
      bk.to_pair(mine.k, mine.r);
#pragma unroll
      for (int i = 0; i < RPT; ++i)
        if (i == ib) {
          if constexpr (sizeof(Ts) == 4) {
#pragma unroll
            for (int q = 0; q < W / 4; ++q)
              reinterpret_cast<float4*>(mine.v)[q] =
                  make_float4(a[i][4 * q], a[i][4 * q + 1], a[i][4 * q + 2], a[i][4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < W / 2; ++q)
              reinterpret_cast<double2*>(mine.v)[q] = make_double2(a[i][2 * q], a[i][2 * q + 1]);
          }
        }
      cl_fence_proxy_async();  // the bulk copies read the staged message
    } else if (lane == 0 && !wk.valid()) {
      Key().to_pair(mine.k, mine.r);
      cl_fence_proxy_async();
    }
    if (c == 0 && tid == j && !my_fail) {
      if constexpr (sizeof(Ts) == 4) {
#pragma unroll
        for (int q = 0; q < W / 4; ++q)
          reinterpret_cast<float4*>(s_rowj[par])[q] =
              make_float4(a[0][4 * q], a[0][4 * q + 1], a[0][4 * q + 2], a[0][4 * q + 3]);
      } else {
#pragma unroll
        for (int q = 0; q < W / 2; ++q)
          reinterpret_cast<double2*>(s_rowj[par])[q] = make_double2(a[0][2 * q], a[0][2 * q + 1]);
      }
      cl_fence_proxy_async();
    }
    // one decision for the whole CTA: a wait of an earlier column gave up
    if (__syncthreads_or(my_fail)) {
      aborted = true;
      break;
    }
    // 2. warp 0: the CTA's winner (its staged message; a CTA without
    //    candidates has every warp's entry empty and sends entry 0), one bulk
    //    copy per CTA of the cluster; warp 1 of CTA 0: row j, likewise
    if (warp == 0) {
      Key ck;
      if (lane < NW) ck = Key::from_pair(s_warp[par][lane].k, s_warp[par][lane].r);
      Key mk = ck;
      warp_merge_redux(mk);
      const unsigned bal = __ballot_sync(0xffffffffu, lane < NW && mk.valid() && ck.same(mk));
      const int ww = bal ? __ffs(bal) - 1 : 0;
      if (lane < CL)
        cl_bulk_push(cl_mapa(cl_smem_u32(&s_recv[par][c]), lane), cl_smem_u32(&s_warp[par][ww]),
                     (uint32_t)sizeof(ClMsg<Ts>), cl_mapa(bar[par], lane));
    } else if (warp == 1 && c == 0) {
      if (lane < CL)
        cl_bulk_push(cl_mapa(cl_smem_u32(s_rowj_recv[par]), lane), cl_smem_u32(s_rowj[par]),
                     (uint32_t)(W * sizeof(Ts)), cl_mapa(bar[par], lane));
    }
    npushed = j + 1;
    // 3. wait for the CL candidates and row j; every warp reduces them
    if (!cl_mbar_wait(bar[par], (uint32_t)((j >> 1) & 1), wait_ns)) {
      my_fail = 1;
    } else {
      if (tid == 0 && j + 2 < W) {
        cl_mbar_arm(bar[par], kExpect);
        armed[par] = j + 2;
      }
      Key q;
      Ts qv = (Ts)0;
      if (lane < CL) {
        q = Key::from_pair(s_recv[par][lane].k, s_recv[par][lane].r);
        qv = s_recv[par][lane].v[j];
      }
      // each lane forms the reciprocal of its candidate's pivot while the
      // warp reduces the keys; the winner's is then broadcast
      const Ts qr = qv != (Ts)0 ? rcp_rn(qv) : (Ts)0;
      Key g = q;
      warp_merge_redux(g);
      const unsigned bal = __ballot_sync(0xffffffffu, lane < CL && q.same(g));
      const int cw = bal ? __ffs(bal) - 1 : 0;
      const int p = g.row();
      // a winner outside rows j .. m-1 cannot come from a completed exchange;
      // it is treated as a failed wait and never reaches ipiv
      const bool pok = p >= j && p < m;
      if (!pok) my_fail = 1;
      if (lane == j) my_piv = pok ? p : j;
      const Ts* prow = s_recv[par][cw].v;
      const Ts pv = __shfl_sync(0xffffffffu, qv, cw);
      const Ts rp = __shfl_sync(0xffffffffu, qr, cw);
      if (c == 0 && tid == 0 && pok) {
        ipiv[j] = row0 + p + 1;
        if (g.zero_pivot()) atomicCAS(info, 0, row0 + j + 1);
      }
      // 4. interchange rows j and p, scale by the reciprocal pivot, rank-1
      //    update (the same operations, in the same order, as the other
      //    panel kernels)
      bool below[RPT];
      Ts lm[RPT];
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int gi = g0 + i * NT;
        below[i] = false;
        lm[i] = (Ts)0;
        if (gi < m) {
          // one source row for the interchange, so that only one row of
          // shared-memory loads is live at a time
          const Ts* src = (p != j && gi == j) ? prow : ((p != j && gi == p) ? s_rowj_recv[par] : nullptr);
          if (src) {
#pragma unroll
            for (int k = 0; k < W; ++k) a[i][k] = src[k];
          }
          if (gi > j) {
            Ts l = a[i][j];
            if (pv != (Ts)0) {
              l = l * rp;
              a[i][j] = l;
            }
            below[i] = true;
            lm[i] = l;
          }
        }
      }
      // the pivot row is read 16 bytes at a time, once for all rows of the thread
      constexpr int VE = 16 / (int)sizeof(Ts);
#pragma unroll
      for (int qv4 = (j + 1) / VE; qv4 < W / VE; ++qv4) {
        Ts pk[VE];
        if constexpr (sizeof(Ts) == 4) {
          const float4 v = reinterpret_cast<const float4*>(prow)[qv4];
          pk[0] = v.x;
          pk[1] = v.y;
          pk[2] = v.z;
          pk[3] = v.w;
        } else {
          const double2 v = reinterpret_cast<const double2*>(prow)[qv4];
          pk[0] = v.x;
          pk[1] = v.y;
        }
#pragma unroll
        for (int e = 0; e < VE; ++e) {
          const int k = VE * qv4 + e;
          if (k > j) {
#pragma unroll
            for (int i = 0; i < RPT; ++i)
              if (below[i]) a[i][k] = fma(-lm[i], pk[e], a[i][k]);
          }
        }
      }
    }
  }
  if (!aborted) aborted = __syncthreads_or(my_fail) != 0;  // a wait of the last column
  if (!aborted) {
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gi = g0 + i * NT;
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (gi < m) A[(size_t)k * lda + gi] = a[i][k];
    }
    if (nleft + nright > 0) {
      LaswpPlan plan;
      plan.make(my_piv, W, lane);
      panel_tail_swaps<Ts>(A, lda, W, nleft, nright, plan, c * NW + warp, CL * NW, lane);
    }
  } else if (tid == 0) {
    gbla_flag_timeout(info);
  }
  // Leaving (see above): publish the push count (top bit: this CTA stopped
  // early) to every CTA. When no CTA stopped early, every copy of the launch
  // has been waited for by its receiver, so the barrier that makes the counts
  // visible is the last one. Otherwise each CTA drains the two armed columns
  // of its mbarriers, then all meet at a final cluster barrier.
  if (tid < CL)
    cl_store_remote_u32(cl_mapa(cl_smem_u32(&s_pushed[c]), tid),
                        (unsigned)npushed | (aborted ? 0x80000000u : 0u));
  cl_sync();
  bool any_stopped = false;
  for (int q = 0; q < CL; ++q) any_stopped = any_stopped || (s_pushed[q] & 0x80000000u) != 0;
  if (!any_stopped) return;  // the same decision in every CTA of the cluster
  if (tid == 0) {
    // every copy counted here has been issued and lands within microseconds;
    // the floor keeps a tiny caller wait limit from cutting the drain short
    const uint64_t drain_ns = wait_ns > 200000000ull ? wait_ns : 200000000ull;
    bool drained = true;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int col = armed[b];
      uint32_t coming = 0;
      for (int q = 0; q < CL; ++q)
        if ((int)(s_pushed[q] & 0x7fffffffu) > col) coming += (uint32_t)sizeof(ClMsg<Ts>);
      if ((int)(s_pushed[0] & 0x7fffffffu) > col) coming += (uint32_t)(W * sizeof(Ts));
      if (coming < kExpect) cl_mbar_complete_tx(bar[b], kExpect - coming);
      drained = cl_mbar_wait(bar[b], (uint32_t)((col >> 1) & 1), drain_ns) && drained;
    }
    if (!drained) gbla_flag_timeout(info);
  }
  __syncthreads();
  cl_sync();
}

template <typename Ts, int NT, int RPT>
static cudaError_t launch_panel_cluster_nt(Ts* A, int lda, int m, int row0, int* ipiv, int* info,
                                           uint64_t wait_ns, int nleft, int nright, int CL,
                                           cudaStream_t s) {
  // once per device: allow clusters of 16 and look up whether a cluster of
  // each size can be resident, so that a launch that cannot be placed is
  // never attempted
  static int max_clusters[64][kClMax + 1];
  static bool init[64] = {false};
  const int dev = device_props().device;
  if (dev < 0 || dev >= 64) return cudaErrorNotSupported;
  if (!init[dev]) {
    cudaError_t e = cudaFuncSetAttribute(panel_cluster_kernel<Ts, NT, RPT>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cudaErrorNotSupported;
    }
    for (int i = 0; i <= kClMax; ++i) max_clusters[dev][i] = -1;
    init[dev] = true;
  }
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  if (max_clusters[dev][CL] < 0) {
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3((unsigned)CL);
    q.blockDim = dim3(NT);
    q.attrs = at;
    q.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, panel_cluster_kernel<Ts, NT, RPT>, &q) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    max_clusters[dev][CL] = n;
  }
  if (max_clusters[dev][CL] < 1) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)CL);  // one cluster: the whole grid
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, panel_cluster_kernel<Ts, NT, RPT>, A, lda, m, row0, ipiv, info,
                            wait_ns, nleft, nright, CL);
}

// Cluster launch shape for a full-width panel of m >= 32 rows: NT threads
// per CTA (128, 256 or 512) with RPT rows each (2 only for FP32 panels of
// more than 8192 rows) and CL = the power of two >= m / (NT * RPT) CTAs. An
// FP64 row takes twice the registers, so FP64 stays at <= 256 threads.
// Returns cudaErrorNotSupported, with nothing enqueued, for a narrower or
// taller panel or when the device cannot hold the cluster.
template <typename Ts>
static cudaError_t launch_panel_cluster(Ts* A, int lda, int m, int w, int row0, int* ipiv,
                                        int* info, uint64_t wait_ns, int nleft, int nright,
                                        cudaStream_t s) {
  constexpr int kMaxNt = sizeof(Ts) == 4 ? 512 : 256;
  constexpr int kMaxRpt = sizeof(Ts) == 4 ? 2 : 1;
  if (w != kPanelWidth || m < kPanelWidth) return cudaErrorNotSupported;
  int NT = 128;
  while (NT < kMaxNt && (long long)NT * kClMax < m) NT *= 2;
  const int RPT = (long long)NT * kClMax >= m ? 1 : 2;
  if (RPT > kMaxRpt || (long long)NT * RPT * kClMax < m) return cudaErrorNotSupported;
  const int need = (m + NT * RPT - 1) / (NT * RPT);
  int CL = 1;
  while (CL < need) CL *= 2;
  if (RPT == 2) {
    if constexpr (sizeof(Ts) == 4)
      return launch_panel_cluster_nt<Ts, 512, 2>(A, lda, m, row0, ipiv, info, wait_ns, nleft, nright, CL, s);
    return cudaErrorNotSupported;
  }
  switch (NT) {
    case 128:
      return launch_panel_cluster_nt<Ts, 128, 1>(A, lda, m, row0, ipiv, info, wait_ns, nleft, nright, CL, s);
    case 256:
      return launch_panel_cluster_nt<Ts, 256, 1>(A, lda, m, row0, ipiv, info, wait_ns, nleft, nright, CL, s);
    default:
      if constexpr (sizeof(Ts) == 4)
        return launch_panel_cluster_nt<Ts, 512, 1>(A, lda, m, row0, ipiv, info, wait_ns, nleft, nright, CL, s);
      return cudaErrorNotSupported;
  }
}

template <typename Ts>
cudaError_t launch_panel(Ts* A, int lda, int m, int w, int row0, int* ipiv, int* info,
                         double* slots, unsigned panel_index, int nleft, int nright,
                         cudaStream_t s) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  if (w > kPanelWidth || nleft < 0 || nright < 0) return cudaErrorInvalidValue;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return cudaErrorNoDevice;
  const uint64_t wait_ns = wait_timeout_ns();
  {
    const cudaError_t ec =
        launch_panel_cluster<Ts>(A, lda, m, w, row0, ipiv, info, wait_ns, nleft, nright, s);
    if (ec != cudaErrorNotSupported) return ec;
  }
  // Panels taller than one cluster holds: up to 64 CTAs exchanging through
  // global memory, all resident together (a cooperative launch). Up to 64
  // CTAs: the exchange round per column gets slower with the number of CTAs
  // polling each other's headers, faster than the per-CTA share of the
  // rank-1 update grows (measured at m = 16384: 3.96 us per column with 64
  // CTAs, 4.79 us with 152).
  const int kMinRows = 64, kMaxCtas = 64;
  const int max_ctas = dp.num_sms < kPanelMaxSms ? dp.num_sms : kPanelMaxSms;
  int C = (m + kMinRows - 1) / kMinRows;
  if (C > kMaxCtas) C = kMaxCtas;
  if (C > max_ctas) C = max_ctas;
  if (C < 1) C = 1;
  int R = (m + C - 1) / C;
  if (R > 2 * kPanelThreads) {  // more CTAs before leaving the register-resident kernel
    C = (m + 2 * kPanelThreads - 1) / (2 * kPanelThreads);
    if (C > max_ctas) C = max_ctas;
    R = (m + C - 1) / C;
  }
  C = (m + R - 1) / R;
  unsigned tag_base = (panel_index + 1u) << 6;
  uint64_t wns = wait_ns;
  void* args[] = {&A, &lda, &m, &w, &row0, &R, &ipiv, &info, &slots, &tag_base, &wns, &nleft, &nright};
  count_launch();
  if (R <= kPanelThreads)
    return cudaLaunchCooperativeKernel((const void*)panel_reg_kernel<Ts, 1>, dim3(C),
                                       dim3(kPanelThreads), args, 0, s);
  if (R <= 2 * kPanelThreads)
    return cudaLaunchCooperativeKernel((const void*)panel_reg_kernel<Ts, 2>, dim3(C),
                                       dim3(kPanelThreads), args, 0, s);
  // very tall panels: shared-memory slab
  size_t smem = ((size_t)w * R + 2 * kPanelWidth) * sizeof(Ts) + 16;
  if (smem > dp.smem_optin) return cudaErrorInvalidValue;
  cudaError_t ea = ensure_dyn_smem(panel_kernel<Ts>, smem);
  if (ea != cudaSuccess) return ea;
  return cudaLaunchCooperativeKernel((const void*)panel_kernel<Ts>, dim3(C), dim3(kPanelThreads),
                                     args, smem, s);
}

template cudaError_t launch_panel<double>(double*, int, int, int, int, int*, int*, double*,
                                          unsigned, int, int, cudaStream_t);
template cudaError_t launch_panel<float>(float*, int, int, int, int, int*, int*, double*,
                                         unsigned, int, int, cudaStream_t);

}  // namespace gbla
