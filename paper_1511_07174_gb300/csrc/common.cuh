// Shared device helpers for the gbla kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gbla.h"

#define GBLA_DEVINL __device__ __forceinline__

// Nanosecond wall clock of the GPU; used to bound every inter-CTA wait.
GBLA_DEVINL uint64_t gbla_now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

GBLA_DEVINL unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

GBLA_DEVINL void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

GBLA_DEVINL int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Record the first device-side failure in the caller's info word: the
// timeout code only replaces a zero (a numerical info already set stays).
GBLA_DEVINL void gbla_flag_timeout(int* info) {
  if (info) atomicCAS(info, 0, GBLA_INFO_TIMEOUT);
}

// Spin until *p >= target or the wait exceeds limit_ns. Returns true on
// success. One thread per CTA calls it.
GBLA_DEVINL bool gbla_wait_geq(const unsigned* p, unsigned target, uint64_t limit_ns) {
  if (ld_acquire_u32(p) >= target) return true;
  uint64_t t0 = gbla_now_ns();
  while (true) {
    if (ld_acquire_u32(p) >= target) return true;
    if (gbla_now_ns() - t0 > limit_ns) return false;
    __nanosleep(32);
  }
}

template <typename T>
GBLA_DEVINL T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
GBLA_DEVINL T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  return v;
}

// (|value|, index) argmax: larger magnitude wins, ties go to the lower index.
GBLA_DEVINL void argmax_merge(double& bv, int& bi, double v, int i) {
  if (v > bv || (v == bv && i < bi)) {
    bv = v;
    bi = i;
  }
}

GBLA_DEVINL void warp_argmax(double& bv, int& bi) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v = __shfl_xor_sync(0xffffffffu, bv, o);
    int i = __shfl_xor_sync(0xffffffffu, bi, o);
    argmax_merge(bv, bi, v, i);
  }
}

// Final sources of the rows touched by kb <= 256 sequential interchanges
// (row t <-> row p_t for t = 0 .. kb - 1 in order, p_t >= t, rows relative to
// the block's first row), worked out by the threads t < kb in parallel. With
// pre(t) the value row t holds just before interchange t:
//   pre(t) = pre(i) for the last i < t with p_i = t, else row t's own value;
//   row t ends with pre(t) if p_t = t, else with what row p_t held just
//   before interchange t: pre(i) for the last i < t with p_i = p_t, else p_t's
//   own value;
//   a partner row x >= kb ends with pre(i) for the last interchange i naming it.
// pre follows the chains t -> i (i < t) to a row that kept its own value,
// found by pointer jumping (8 rounds cover chains of 256). Every thread of the
// CTA must call it (it contains barriers); s.p must already hold the p_t.
struct SwapPlanShared {
  int p[256];
  int J[2][256];
};

// Thread t < kb: *src_b = the row whose original value ends in row t; when t
// is the last interchange naming a partner row p_t >= kb, *dst_o = p_t and
// *src_o its source, else *dst_o = -1.
GBLA_DEVINL void swap_plan(SwapPlanShared& s, int kb, int t, int* src_b, int* dst_o, int* src_o) {
  int last_to = -1, prev_same = -1;
  bool later = false;
  const int pt = t < kb ? s.p[t] : -1;
  if (t < kb) {
    for (int i = 0; i < kb; ++i) {
      const int q = s.p[i];
      if (i < t) {
        if (q == t) last_to = i;
        if (q == pt) prev_same = i;
      } else if (i > t && q == pt) {
        later = true;
      }
    }
    s.J[0][t] = last_to < 0 ? t : last_to;
  }
  __syncthreads();
  int cur = 0;
#pragma unroll 1
  for (int r = 0; r < 8; ++r) {
    if (t < kb) s.J[cur ^ 1][t] = s.J[cur][s.J[cur][t]];
    __syncthreads();
    cur ^= 1;
  }
  *dst_o = -1;
  if (t < kb) {
    const int pre_t = s.J[cur][t];
    *src_b = pt == t ? pre_t : (prev_same >= 0 ? s.J[cur][prev_same] : pt);
    if (pt >= kb && !later) {
      *dst_o = pt;
      *src_o = pre_t;
    }
  }
}
