// Panel factorisation with partial pivoting (paper section 2, the GEPP step of
// the blocked LU): an m x w panel (w <= 32) is spread over C cooperative CTAs,
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

size_t panel_slots_doubles() {
  const DeviceProps& p = device_props();
  int c = p.num_sms > 0 ? p.num_sms : 160;
  (void)c;
  return (size_t)2 * (256 + 1) * kPanelSlotW + kPanelWidth;  // slots for <= 256 SMs + pivot log
}

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
  __shared__ Key s_wk[kPanelThreads / 32];
  __shared__ Key s_key;
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
  __shared__ Key s_wk[kPanelThreads / 32];
  __shared__ Key s_key;
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

template <typename Ts>
cudaError_t launch_panel(Ts* A, int lda, int m, int w, int row0, int* ipiv, int* info,
                         double* slots, unsigned panel_index, int ncols, cudaStream_t s) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  if (w > kPanelWidth) return cudaErrorInvalidValue;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return cudaErrorNoDevice;
  // Up to 64 CTAs: the exchange round per column gets slower with the number
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
