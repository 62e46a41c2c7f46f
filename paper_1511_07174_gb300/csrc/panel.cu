// Panel factorisation with partial pivoting (paper section 2, the GEPP step of
// the blocked LU): an m x w panel (w <= 32) is spread over C cooperative CTAs,
// each holding a contiguous slab of R rows in shared memory, in FP64.
//
// Per column j (one grid barrier per column):
//   1. each CTA finds its local argmax of |a_ij| over its rows i >= j
//      (warp-shuffle reduction; ties -> lowest row index);
//   2. it publishes (|v|, row, the whole candidate row) to a global slot, and
//      the CTA that owns row j publishes row j;
//   3. grid barrier (bounded wait);
//   4. every CTA reduces the C slots to the global pivot p (same tie rule),
//      reads the pivot row from the winner's slot and swaps rows j and p in
//      its own slab (no second barrier: both rows were published in step 2);
//   5. scales its multipliers l_ij = a_ij / a_jj (division, i > j) and applies
//      the rank-1 update a_ik -= l_ij a_jk for k > j inside the panel.
// Slots are double-buffered by column parity: a CTA can only overwrite the
// parity-(j) slots after the barrier of column j+1, which every CTA reaches
// only after it has finished reading them.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kPanelThreads = 256;

size_t panel_slots_doubles() {
  const DeviceProps& p = device_props();
  int c = p.num_sms > 0 ? p.num_sms : 160;
  return (size_t)(2 * (c + 1)) * kPanelSlotW;
}

template <typename Ts>
__global__ void __launch_bounds__(kPanelThreads)
    panel_kernel(Ts* __restrict__ A, int lda, int m, int w, int row0, int R,
                 int* __restrict__ ipiv, int* __restrict__ info, double* __restrict__ slots,
                 unsigned* __restrict__ counter, uint64_t wait_ns) {
  extern __shared__ double smem[];
  double* slab = smem;                          // [w][R], column-major slab
  double* prow = slab + (size_t)w * R;          // pivot row (w)
  double* rj = prow + kPanelWidth;              // old row j (w)
  __shared__ double s_wv[kPanelThreads / 32];
  __shared__ int s_wi[kPanelThreads / 32];
  __shared__ double s_pv;
  __shared__ int s_p, s_cw, s_abort;

  const int C = gridDim.x;
  const int c = blockIdx.x;
  const int tid = threadIdx.x;
  const int rbeg = c * R;
  const int rcnt = max(0, min(R, m - rbeg));
  double* rowj_buf = slots + (size_t)2 * C * kPanelSlotW;

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
    // 1. local argmax over own rows with panel row >= j
    double bv = -1.0;
    int bi = INT_MAX;
    for (int r = tid; r < rcnt; r += blockDim.x) {
      int gi = rbeg + r;
      if (gi >= j) argmax_merge(bv, bi, fabs(slab[j * R + r]), gi);
    }
    warp_argmax(bv, bi);
    if ((tid & 31) == 0) {
      s_wv[tid >> 5] = bv;
      s_wi[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid < 32) {
      const int nw = blockDim.x >> 5;
      double v = tid < nw ? s_wv[tid] : -1.0;
      int i = tid < nw ? s_wi[tid] : INT_MAX;
      warp_argmax(v, i);
      if (tid == 0) {
        s_pv = v;
        s_p = i;
      }
    }
    __syncthreads();
    // 2. publish the local candidate (and row j if owned)
    double* myslot = slots + ((size_t)par * C + c) * kPanelSlotW;
    const int lb = s_p;
    if (tid == 0) {
      myslot[0] = s_pv;
      myslot[1] = (double)lb;
    }
    if (tid < w && lb != INT_MAX) myslot[2 + tid] = slab[tid * R + (lb - rbeg)];
    if (j >= rbeg && j < rbeg + rcnt && tid < w)
      rowj_buf[par * kPanelSlotW + tid] = slab[tid * R + (j - rbeg)];
    __syncthreads();
    // 3. grid barrier
    if (tid == 0) {
      __threadfence();
      atomicAdd(counter, 1u);
      bool ok = gbla_wait_geq(counter, (unsigned)(j + 1) * (unsigned)C, wait_ns);
      __threadfence();
      if (!ok) {
        gbla_flag_timeout(info);
        s_abort = 1;
      }
    }
    __syncthreads();
    if (s_abort) return;
    // 4. global argmax over the published candidates
    if (tid < 32) {
      double v = -1.0;
      int i = INT_MAX, cw = 0;
      for (int q = tid; q < C; q += 32) {
        const double* s = slots + ((size_t)par * C + q) * kPanelSlotW;
        double sv = __ldcg(s);
        int si = (int)__ldcg(s + 1);
        if (sv > v || (sv == v && si < i)) {
          v = sv;
          i = si;
          cw = q;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        int c2 = __shfl_xor_sync(0xffffffffu, cw, o);
        if (v2 > v || (v2 == v && i2 < i)) {
          v = v2;
          i = i2;
          cw = c2;
        }
      }
      if (tid == 0) {
        s_pv = v;
        s_p = i;
        s_cw = cw;
      }
    }
    __syncthreads();
    const int p = s_p;
    const int cw = s_cw;
    const bool own_j = (j >= rbeg && j < rbeg + rcnt);
    const bool own_p = (p >= rbeg && p < rbeg + rcnt);
    if (tid < w) {
      prow[tid] = __ldcg(slots + ((size_t)par * C + cw) * kPanelSlotW + 2 + tid);
      if (p != j && own_p) rj[tid] = __ldcg(rowj_buf + par * kPanelSlotW + tid);
    }
    if (c == 0 && tid == 0) {
      ipiv[j] = row0 + p + 1;
      if (s_pv == 0.0) atomicCAS(info, 0, row0 + j + 1);
    }
    __syncthreads();
    // swap rows j and p inside the slabs
    if (p != j && tid < w) {
      if (own_j) slab[tid * R + (j - rbeg)] = prow[tid];
      if (own_p) slab[tid * R + (p - rbeg)] = rj[tid];
    }
    __syncthreads();
    // 5. scale and rank-1 update of own rows below the pivot
    const double piv = prow[j];
    for (int r = tid; r < rcnt; r += blockDim.x) {
      if (rbeg + r > j) {
        double l = slab[j * R + r];
        if (piv != 0.0) {
          l = l / piv;
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
                         double* slots, unsigned* counter, cudaStream_t s) {
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
  void* args[] = {&A, &lda, &m, &w, &row0, &R, &ipiv, &info, &slots, &counter, &wait_ns};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)panel_kernel<Ts>, dim3(C), dim3(kPanelThreads),
                                     args, smem, s);
}

template cudaError_t launch_panel<double>(double*, int, int, int, int, int*, int*, double*,
                                          unsigned*, cudaStream_t);
template cudaError_t launch_panel<float>(float*, int, int, int, int, int*, int*, double*,
                                         unsigned*, cudaStream_t);

}  // namespace gbla
