// Panel factorisation with partial pivoting (paper section 2, the GEPP step of
// the blocked LU): an m x w panel (w <= 32) is spread over C cooperative CTAs,
// each holding a contiguous slab of R rows in shared memory, in FP64.
//
// Per column j:
//   1. each CTA finds its local argmax of |a_ij| over its rows i >= j
//      (warp-shuffle reduction on the IEEE bit patterns of |a_ij|, which
//      order like the values; ties -> lowest row index);
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
  return (size_t)(2 * (c + 1)) * kPanelSlotW;
}

typedef unsigned long long u64;

GBLA_DEVINL void st_relaxed_u64(u64* p, u64 v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
GBLA_DEVINL u64 ld_relaxed_u64(const u64* p) {
  u64 v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Wait (bounded) until the word at p carries `tag` in its upper half.
GBLA_DEVINL bool ll_read(const u64* p, u64 tag, uint64_t wait_ns, uint32_t* payload) {
  u64 v = ld_relaxed_u64(p);
  if ((v & 0xffffffff00000000ull) != tag) {
    const uint64_t t0 = gbla_now_ns();
    while (true) {
      v = ld_relaxed_u64(p);
      if ((v & 0xffffffff00000000ull) == tag) break;
      if (gbla_now_ns() - t0 > wait_ns) return false;
    }
  }
  *payload = (uint32_t)(v & 0xffffffffull);
  return true;
}

// key order: larger |v| bits first, then lower row index
GBLA_DEVINL void key_merge(u64& bk, int& bi, int& bc, u64 k, int i, int cq) {
  if (k > bk || (k == bk && i < bi)) {
    bk = k;
    bi = i;
    bc = cq;
  }
}
GBLA_DEVINL void warp_key_argmax(u64& bk, int& bi, int& bc) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 k = __shfl_xor_sync(0xffffffffu, bk, o);
    const int i = __shfl_xor_sync(0xffffffffu, bi, o);
    const int cq = __shfl_xor_sync(0xffffffffu, bc, o);
    key_merge(bk, bi, bc, k, i, cq);
  }
}

template <typename Ts>
__global__ void __launch_bounds__(kPanelThreads)
    panel_kernel(Ts* __restrict__ A, int lda, int m, int w, int row0, int R,
                 int* __restrict__ ipiv, int* __restrict__ info, double* __restrict__ slots_d,
                 unsigned tag_base, uint64_t wait_ns) {
  extern __shared__ double smem[];
  double* slab = smem;                          // [w][R], column-major slab
  double* prow = slab + (size_t)w * R;          // pivot row (w)
  double* rj = prow + kPanelWidth;              // old row j (w)
  __shared__ u64 s_wk[kPanelThreads / 32];
  __shared__ int s_wi[kPanelThreads / 32], s_wc[kPanelThreads / 32];
  __shared__ u64 s_pk;
  __shared__ double s_rp;
  __shared__ int s_p, s_cw, s_abort;

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
      slab[k * R + r] = (double)A[(size_t)k * lda + rbeg + r];
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
    u64 bk = 0;
    int bi = INT_MAX, bc = c;
    for (int r = tid; r < rcnt; r += blockDim.x) {
      const int gi = rbeg + r;
      if (gi >= j) key_merge(bk, bi, bc, (u64)__double_as_longlong(fabs(slab[j * R + r])), gi, c);
    }
    warp_key_argmax(bk, bi, bc);
    if (lane == 0) {
      s_wk[warp] = bk;
      s_wi[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
      bk = lane < nwarps ? s_wk[lane] : 0;
      bi = lane < nwarps ? s_wi[lane] : INT_MAX;
      warp_key_argmax(bk, bi, bc);
      if (lane == 0) {
        s_pk = bk;
        s_p = bi;
      }
    }
    __syncthreads();
    // 2. publish: candidate row and row j as tagged 32-bit halves, header last
    u64* myslot = slots + ((size_t)par * C + c) * kPanelSlotW;
    const int lb = s_p;
    if (tid < 2 * w) {
      const int k = tid >> 1;
      if (lb != INT_MAX) {
        const u64 bits = (u64)__double_as_longlong(slab[k * R + (lb - rbeg)]);
        st_relaxed_u64(myslot + kSlotRow + tid, tag | ((tid & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      }
      if (j >= rbeg && j < rbeg + rcnt) {
        const u64 bits = (u64)__double_as_longlong(slab[k * R + (j - rbeg)]);
        st_relaxed_u64(rowj_buf + par * kPanelSlotW + tid,
                       tag | ((tid & 1) ? (bits >> 32) : (bits & 0xffffffffull)));
      }
    }
    if (tid == 0) {
      const u64 kb = s_pk;
      st_relaxed_u64(myslot + 0, tag | (kb & 0xffffffffull));
      st_relaxed_u64(myslot + 1, tag | (kb >> 32));
      st_relaxed_u64(myslot + 2, tag | (u64)(unsigned)lb);
    }
    // 3. thread q polls header q; block-wide argmax of the C candidates
    bk = 0;
    bi = INT_MAX;
    bc = 0;
    bool ok = true;
    for (int q = tid; q < C; q += blockDim.x) {
      const u64* h = slots + ((size_t)par * C + q) * kPanelSlotW;
      uint32_t lo, hi, ix;
      ok = ll_read(h + 0, tag, wait_ns, &lo) && ll_read(h + 1, tag, wait_ns, &hi) &&
           ll_read(h + 2, tag, wait_ns, &ix);
      if (!ok) break;
      key_merge(bk, bi, bc, ((u64)hi << 32) | lo, (int)ix, q);
    }
    if (!ok) s_abort = 1;
    warp_key_argmax(bk, bi, bc);
    if (lane == 0) {
      s_wk[warp] = bk;
      s_wi[warp] = bi;
      s_wc[warp] = bc;
    }
    __syncthreads();
    if (s_abort) {
      if (tid == 0) gbla_flag_timeout(info);
      return;
    }
    if (warp == 0) {
      bk = lane < nwarps ? s_wk[lane] : 0;
      bi = lane < nwarps ? s_wi[lane] : INT_MAX;
      bc = lane < nwarps ? s_wc[lane] : 0;
      warp_key_argmax(bk, bi, bc);
      if (lane == 0) {
        s_pk = bk;
        s_p = bi;
        s_cw = bc;
      }
    }
    __syncthreads();
    const int p = s_p;
    const int cw = s_cw;
    const bool own_j = (j >= rbeg && j < rbeg + rcnt);
    const bool own_p = (p >= rbeg && p < rbeg + rcnt);
    // 4. pivot row from the winner's slot; old row j when this CTA owns row p
    if (warp < 2) {  // whole warps, so that the pair shuffles see every lane
      const bool act = tid < 2 * w;
      const u64* wrow = slots + ((size_t)par * C + cw) * kPanelSlotW + kSlotRow;
      uint32_t half = 0;
      bool okr = act ? ll_read(wrow + tid, tag, wait_ns, &half) : true;
      uint32_t other = __shfl_xor_sync(0xffffffffu, half, 1);
      if (act && (tid & 1) == 0) {
        const double v = __longlong_as_double((long long)(((u64)other << 32) | half));
        prow[tid >> 1] = v;
        if ((tid >> 1) == j) s_rp = v != 0.0 ? 1.0 / v : 0.0;
      }
      if (p != j && own_p) {
        if (act) okr = ll_read(rowj_buf + par * kPanelSlotW + tid, tag, wait_ns, &half) && okr;
        other = __shfl_xor_sync(0xffffffffu, half, 1);
        if (act && (tid & 1) == 0)
          rj[tid >> 1] = __longlong_as_double((long long)(((u64)other << 32) | half));
      }
      if (!okr) s_abort = 1;
    }
    if (c == 0 && tid == 0) {
      ipiv[j] = row0 + p + 1;
      if (s_pk == 0) atomicCAS(info, 0, row0 + j + 1);
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
    const double rp = s_rp;
    const bool nz = prow[j] != 0.0;
    for (int r = tid; r < rcnt; r += blockDim.x) {
      if (rbeg + r > j) {
        double l = slab[j * R + r];
        if (nz) {
          l = l * rp;
          slab[j * R + r] = l;
        }
        for (int k = j + 1; k < w; ++k) slab[k * R + r] = fma(-l, prow[k], slab[k * R + r]);
      }
    }
    __syncthreads();
  }
  for (int k = 0; k < w; ++k)
    for (int r = tid; r < rcnt; r += blockDim.x)
      A[(size_t)k * lda + rbeg + r] = (Ts)slab[k * R + r];
}

template <typename Ts>
cudaError_t launch_panel(Ts* A, int lda, int m, int w, int row0, int* ipiv, int* info,
                         double* slots, unsigned panel_index, cudaStream_t s) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  if (w > kPanelWidth) return cudaErrorInvalidValue;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return cudaErrorNoDevice;
  const int kMinRows = 64;
  int C = (m + kMinRows - 1) / kMinRows;
  if (C > dp.num_sms) C = dp.num_sms;
  if (C < 1) C = 1;
  int R = (m + C - 1) / C;
  C = (m + R - 1) / R;
  size_t smem = ((size_t)w * R + 2 * kPanelWidth) * sizeof(double);
  if (smem > dp.smem_optin) return cudaErrorInvalidValue;
  cudaError_t ea = ensure_dyn_smem(panel_kernel<Ts>, smem);
  if (ea != cudaSuccess) return ea;
  uint64_t wait_ns = wait_timeout_ns();
  unsigned tag_base = (panel_index + 1u) << 6;
  void* args[] = {&A, &lda, &m, &w, &row0, &R, &ipiv, &info, &slots, &tag_base, &wait_ns};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)panel_kernel<Ts>, dim3(C), dim3(kPanelThreads),
                                     args, smem, s);
}

template cudaError_t launch_panel<double>(double*, int, int, int, int, int*, int*, double*,
                                          unsigned, cudaStream_t);
template cudaError_t launch_panel<float>(float*, int, int, int, int, int*, int*, double*,
                                         unsigned, cudaStream_t);

}  // namespace gbla
