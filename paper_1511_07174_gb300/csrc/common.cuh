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
