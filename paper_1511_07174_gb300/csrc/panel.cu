// Panel factorisation with partial pivoting (paper section 2, the GEPP step of
// the blocked LU). Full-width panels of up to 16384 (FP32) or 4096 (FP64)
// rows run in one thread-block cluster (the cluster variant further down);
// the kernels described here take the others: an m x w panel (w <= 32) is
// spread over C cooperative CTAs,
// each holding a contiguous slab of R rows in shared memory in the storage
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
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kPanelThreads = 256;
constexpr int kSlotRow = 4;  // words before the row words in a slot (3 header words + pad)

size_t panel_slots_doubles() { return kPanelExchangeDoubles + kPanelWidth + kInnerCounters / 2; }

typedef unsigned long long u64;

// Word offset of the pivot log in the exchange area (after 2 * (kMaxSms + 1)
// slots); the host sizes the area with the same bound.
constexpr int kPanelMaxSms = 256;
GBLA_DEVINL size_t panel_pivlog_offset() { return (size_t)2 * (kPanelMaxSms + 1) * kPanelSlotW; }

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

// Interchange role of the panel launch: the last S CTAs apply each column's
// row interchange (rows j0 + j and j0 + p) to every column of the matrix
// outside the panel, as soon as CTA 0 has logged the pivot of column j. They
// only read the exchange (never publish), so they cannot slow the panel down;
// each thread always owns the same columns, so program order keeps the
// interchanges of one column in sequence.
template <typename Ts>
GBLA_DEVINL void swapper_role(Ts* __restrict__ Aall, int lda, int ncols, int j0, int w, int jend,
                              int sidx, int S, const u64* __restrict__ pivlog, unsigned tag_base,
                              int* __restrict__ info, uint64_t wait_ns) {
  __shared__ int s_sp, s_sabort;
  const int other = ncols - w;
  const int per = (other + S - 1) / S;
  const int cbeg = sidx * per, cend = min(other, cbeg + per);
  for (int j = 0; j < jend; ++j) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const u64 tag = (u64)(tag_base | (unsigned)(j + 1)) << 32;
      uint32_t pl[1] = {0};
      s_sabort = ll_read<1>(pivlog + j, tag, wait_ns, pl) ? 0 : 1;
      s_sp = (int)pl[0];
    }
    __syncthreads();
    if (s_sabort) {
      if (threadIdx.x == 0) gbla_flag_timeout(info);
      return;
    }
    const int p = s_sp;
    if (p == j) continue;
    for (int q = cbeg + (int)threadIdx.x; q < cend; q += blockDim.x) {
      const int col = q < j0 ? q : q + w;
      Ts* a = Aall + (size_t)col * lda;
      const Ts x = a[j0 + j];
      a[j0 + j] = a[j0 + p];
      a[j0 + p] = x;
    }
  }
}

template <typename Ts>
__global__ void __launch_bounds__(kPanelThreads)
    panel_kernel(Ts* __restrict__ A, int lda, int m, int w, int row0, int R,
                 int* __restrict__ ipiv, int* __restrict__ info, double* __restrict__ slots_d,
                 unsigned tag_base, uint64_t wait_ns, int ncols, int S) {
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
  const int C = gridDim.x - S;  // panel CTAs; the last S CTAs apply the interchanges
  if ((int)blockIdx.x >= C) {
    swapper_role<Ts>(A - (size_t)row0 - (size_t)row0 * lda, lda, ncols, row0, w, min(w, m),
                     (int)blockIdx.x - C, S,
                     reinterpret_cast<const u64*>(slots_d) + panel_pivlog_offset(), tag_base, info,
                     wait_ns);
    return;
  }
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
      if (S > 0)
        st_relaxed_u64(slots + panel_pivlog_offset() + j, tag | (u64)(unsigned)p);
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
                     unsigned tag_base, uint64_t wait_ns, int ncols, int S) {
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
  const int C = gridDim.x - S;  // panel CTAs; the last S CTAs apply the interchanges
  if ((int)blockIdx.x >= C) {
    swapper_role<Ts>(A - (size_t)row0 - (size_t)row0 * lda, lda, ncols, row0, w, min(w, m),
                     (int)blockIdx.x - C, S,
                     reinterpret_cast<const u64*>(slots_d) + panel_pivlog_offset(), tag_base, info,
                     wait_ns);
    return;
  }
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
      if (S > 0)
        st_relaxed_u64(slots + panel_pivlog_offset() + j, tag | (u64)(unsigned)p);
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
}

// ---------------------------------------------------------------------------
// Cluster variant. The panel rows are spread over the CL CTAs (CL <= 16) of
// one thread-block cluster, RPT (1 or 2) rows per thread, all kPanelWidth
// columns in registers; the three argmax levels (thread -> warp -> CTA ->
// cluster) use the warp's integer max reduction. The per-column exchange stays inside the cluster: every CTA
// pushes its candidate (pivot key + row) into the shared memory of every CTA
// of the cluster with st.async, completing bytes on the receiver's mbarrier,
// and CTA 0 pushes old row j the same way; each CTA then waits on its own
// mbarrier alone and reduces the CL candidates locally. Nothing goes through
// global memory except the pivot log read by the interchange CTAs, which form
// further clusters of the same cooperative launch.
//
// Buffers are double-buffered by column parity. A CTA pushes column j + 2
// only after it has received every CTA's column j + 1 message, and each CTA
// sends that message only after it has finished reading its column j
// buffers; a CTA re-arms the mbarrier of column j + 2 before it sends its own
// column j + 1 message, so the transaction count is always armed before any
// byte of that column can arrive.
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
GBLA_DEVINL bool cl_mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
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

template <typename Ts, int NT, int RPT>
__global__ void __launch_bounds__(NT, 1)
    panel_cluster_kernel(Ts* __restrict__ A, int lda, int m, int row0,
                         int* __restrict__ ipiv, int* __restrict__ info,
                         double* __restrict__ slots_d, unsigned tag_base, uint64_t wait_ns,
                         int ncols, int CL) {
  typedef PivKey<Ts> Key;
  constexpr int W = kPanelWidth;
  constexpr int NW = NT / 32;
  __shared__ ClMsg<Ts> s_warp[2][NW];                  // each warp's winner (key + row)
  __shared__ ClMsg<Ts> s_recv[2][kClMax];              // candidates pushed by the cluster
  __shared__ alignas(16) Ts s_rowj[2][W];              // row j staged by its owner
  __shared__ alignas(16) Ts s_rowj_recv[2][W];         // row j pushed by CTA 0
  __shared__ alignas(8) u64 s_bar[2];
  __shared__ int s_abort;

  const u64* pivlog_r = reinterpret_cast<const u64*>(slots_d) + panel_pivlog_offset();
  const int S = (int)gridDim.x - CL;
  if ((int)blockIdx.x >= CL) {
    swapper_role<Ts>(A - (size_t)row0 - (size_t)row0 * lda, lda, ncols, row0, W, W,
                     (int)blockIdx.x - CL, S, pivlog_r, tag_base, info, wait_ns);
    return;
  }
  u64* pivlog = reinterpret_cast<u64*>(slots_d) + panel_pivlog_offset();
  // every shared-memory address below is mapped into CTAs 0 .. CL - 1 of this
  // cluster: a launch whose clusters are not CL CTAs wide (never made by this
  // library's launcher) does no exchange at all and reports a failed wait
  if (cl_nctarank() != (uint32_t)CL || cl_ctarank() != blockIdx.x) {
    if (threadIdx.x == 0) gbla_flag_timeout(info);
    return;
  }
  const int c = blockIdx.x;  // rank in the panel cluster (cluster 0)
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
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
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // pivots start as "no interchange", so that an aborted launch leaves only
  // in-range row indices behind for the kernels that follow
  if (c == 0 && tid < W) ipiv[tid] = row0 + tid + 1;
  cl_sync();  // every mbarrier initialised and armed before the first push

  bool aborted = false;
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
    if (bk.valid() && bk.same(wk)) {
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
    if (c == 0 && tid == j) {
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
    __syncthreads();
    if (s_abort) {
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
    // 3. wait for the CL candidates and row j; every warp reduces them
    const bool ok = cl_mbar_wait(bar[par], (uint32_t)((j >> 1) & 1), wait_ns);
    if (!ok) {
      s_abort = 1;
    } else {
      if (tid == 0 && j + 2 < W) cl_mbar_arm(bar[par], kExpect);
      Key q;
      Ts qv = (Ts)0;
      if (lane < CL) {
        q = Key::from_pair(s_recv[par][lane].k, s_recv[par][lane].r);
        qv = s_recv[par][lane].v[j];
      }
      // each lane forms the reciprocal of its candidate's pivot while the
      // warp reduces the keys; the winner's is then broadcast
      const Ts qr = qv != (Ts)0 ? (Ts)1 / qv : (Ts)0;
      Key g = q;
      warp_merge_redux(g);
      const unsigned bal = __ballot_sync(0xffffffffu, lane < CL && q.same(g));
      const int cw = bal ? __ffs(bal) - 1 : 0;
      const int p = g.row();
      const Ts* prow = s_recv[par][cw].v;
      const Ts pv = __shfl_sync(0xffffffffu, qv, cw);
      const Ts rp = __shfl_sync(0xffffffffu, qr, cw);
      if (c == 0 && tid == 0) {
        ipiv[j] = row0 + p + 1;
        if (S > 0)
          st_relaxed_u64(pivlog + j, ((u64)(tag_base | (unsigned)(j + 1)) << 32) | (u64)(unsigned)p);
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
  if (!aborted) {
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int gi = g0 + i * NT;
#pragma unroll
      for (int k = 0; k < W; ++k)
        if (gi < m) A[(size_t)k * lda + gi] = a[i][k];
    }
  } else if (tid == 0) {
    gbla_flag_timeout(info);
  }
  // no CTA leaves while a peer may still write into its shared memory
  cl_sync();
  if (aborted) {
    const uint64_t t0 = gbla_now_ns();
    while (gbla_now_ns() - t0 < 20000) {
    }
  }
}

template <typename Ts, int NT, int RPT>
static cudaError_t launch_panel_cluster_nt(Ts* A, int lda, int m, int row0, int* ipiv,
                                           int* info, double* slots, unsigned tag_base,
                                           uint64_t wait_ns, int ncols, int CL, int S,
                                           cudaStream_t s) {
  // once per device: allow clusters of 16 and look up how many clusters of
  // each size can be resident, so that a launch that cannot be co-resident
  // is never attempted
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
  if (max_clusters[dev][CL] < 0) {
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3((unsigned)CL);
    q.blockDim = dim3(NT);
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = (unsigned)CL;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, panel_cluster_kernel<Ts, NT, RPT>, &q) != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    max_clusters[dev][CL] = n;
  }
  if (max_clusters[dev][CL] < 1 + S / CL) return cudaErrorNotSupported;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CL + S));
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeCooperative;
  at[1].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  count_launch();
  return cudaLaunchKernelEx(&cfg, panel_cluster_kernel<Ts, NT, RPT>, A, lda, m, row0, ipiv, info,
                            slots, tag_base, wait_ns, ncols, CL);
}

// Cluster launch shape for a full-width panel of m >= 32 rows: NT threads
// per CTA (128, 256 or 512) with RPT rows each (2 only for FP32 panels of
// more than 8192 rows), CL = the power of two >= m / (NT * RPT), and enough
// interchange CTAs (a multiple of CL, at most 64) for about one column per
// thread. An FP64 row takes twice the registers, so FP64 stays at <= 256
// threads.
// Returns cudaErrorNotSupported, with nothing enqueued, for a narrower or
// taller panel or when the device cannot hold the launch.
template <typename Ts>
static cudaError_t launch_panel_cluster(Ts* A, int lda, int m, int w, int row0, int* ipiv,
                                        int* info, double* slots, unsigned tag_base,
                                        uint64_t wait_ns, int ncols, cudaStream_t s) {
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
  const int other = ncols - w;
  int S = 0;
  if (other > 0) {
    S = (other + NT - 1) / NT;
    if (S > 64) S = 64;
    S = ((S + CL - 1) / CL) * CL;
  }
  if (RPT == 2) {
    if constexpr (sizeof(Ts) == 4)
      return launch_panel_cluster_nt<Ts, 512, 2>(A, lda, m, row0, ipiv, info, slots, tag_base, wait_ns, ncols, CL, S, s);
    return cudaErrorNotSupported;
  }
  switch (NT) {
    case 128:
      return launch_panel_cluster_nt<Ts, 128, 1>(A, lda, m, row0, ipiv, info, slots, tag_base, wait_ns, ncols, CL, S, s);
    case 256:
      return launch_panel_cluster_nt<Ts, 256, 1>(A, lda, m, row0, ipiv, info, slots, tag_base, wait_ns, ncols, CL, S, s);
    default:
      if constexpr (sizeof(Ts) == 4)
        return launch_panel_cluster_nt<Ts, 512, 1>(A, lda, m, row0, ipiv, info, slots, tag_base, wait_ns, ncols, CL, S, s);
      return cudaErrorNotSupported;
  }
}

template <typename Ts>
cudaError_t launch_panel(Ts* A, int lda, int m, int w, int row0, int* ipiv, int* info,
                         double* slots, unsigned panel_index, int ncols, cudaStream_t s) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  if (w > kPanelWidth) return cudaErrorInvalidValue;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return cudaErrorNoDevice;
  {
    const cudaError_t ec = launch_panel_cluster<Ts>(A, lda, m, w, row0, ipiv, info, slots,
                                                    (panel_index + 1u) << 6, wait_timeout_ns(),
                                                    ncols, s);
    if (ec != cudaErrorNotSupported) return ec;
  }
  // Panels taller than one cluster holds: up to 64 CTAs exchanging through
  // global memory. Up to 64 CTAs: the exchange round per column gets slower with the number
  // of CTAs polling each other's headers, faster than the per-CTA share of
  // the rank-1 update grows (measured at m = 16384: 3.96 us per column with
  // 64 CTAs, 4.79 us with 152).
  const int kMinRows = 64, kMaxCtas = 64;
  int C = (m + kMinRows - 1) / kMinRows;
  if (C > kMaxCtas) C = kMaxCtas;
  if (C > dp.num_sms) C = dp.num_sms;
  if (C < 1) C = 1;
  int R = (m + C - 1) / C;
  if (R > 2 * kPanelThreads) {  // more CTAs before leaving the register-resident kernel
    C = (m + 2 * kPanelThreads - 1) / (2 * kPanelThreads);
    if (C > dp.num_sms) C = dp.num_sms;
    R = (m + C - 1) / C;
  }
  C = (m + R - 1) / R;
  // interchange CTAs: enough that each owns ~512 of the other columns, while
  // the whole grid stays co-resident (one CTA per SM)
  int S = 0;
  if (ncols > w) {
    S = (ncols - w + 511) / 512;
    if (S > 32) S = 32;
    if (S > dp.num_sms - C) S = dp.num_sms - C;
    if (S < 1) S = 0;  // no room: caller must apply the interchanges itself
  }
  if (S == 0 && ncols > w) return cudaErrorInvalidConfiguration;
  uint64_t wait_ns = wait_timeout_ns();
  unsigned tag_base = (panel_index + 1u) << 6;
  void* args[] = {&A, &lda, &m, &w, &row0, &R, &ipiv, &info, &slots, &tag_base, &wait_ns, &ncols, &S};
  count_launch();
  if (R <= kPanelThreads)
    return cudaLaunchCooperativeKernel((const void*)panel_reg_kernel<Ts, 1>, dim3(C + S),
                                       dim3(kPanelThreads), args, 0, s);
  if (R <= 2 * kPanelThreads)
    return cudaLaunchCooperativeKernel((const void*)panel_reg_kernel<Ts, 2>, dim3(C + S),
                                       dim3(kPanelThreads), args, 0, s);
  // very tall panels: shared-memory slab
  size_t smem = ((size_t)w * R + 2 * kPanelWidth) * sizeof(Ts) + 16;
  if (smem > dp.smem_optin) return cudaErrorInvalidValue;
  cudaError_t ea = ensure_dyn_smem(panel_kernel<Ts>, smem);
  if (ea != cudaSuccess) return ea;
  return cudaLaunchCooperativeKernel((const void*)panel_kernel<Ts>, dim3(C + S), dim3(kPanelThreads),
                                     args, smem, s);
}

template cudaError_t launch_panel<double>(double*, int, int, int, int, int*, int*, double*,
                                          unsigned, int, cudaStream_t);
template cudaError_t launch_panel<float>(float*, int, int, int, int, int*, int*, double*,
                                         unsigned, int, cudaStream_t);

}  // namespace gbla
