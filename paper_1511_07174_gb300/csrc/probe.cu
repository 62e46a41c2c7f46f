// Arithmetic-rate probes: the FP64 and FP32 fused multiply-add throughput of
// the whole GPU, measured with a kernel of independent FMA chains. They give
// the ALU-bound kernels of this library (the FP64 factorisations and
// substitutions, the batched solver) a denominator measured on the device
// they run on, instead of a library GEMM's rate or a nominal figure.
#include "internal.h"

namespace gbla {

constexpr int kProbeChains = 8;     // independent FMA chains per thread
constexpr int kProbeThreads = 256;

// Each thread runs kProbeChains chains x = x * m + c for `iters` steps. The
// multiplier is just below one, so the values stay finite; the sum is stored
// only when it equals a value it cannot reach, which keeps the chains live
// without any global traffic.
template <typename T>
__global__ void __launch_bounds__(kProbeThreads)
    fma_probe_kernel(int iters, T m, T c, T* __restrict__ sink) {
  T x[kProbeChains];
#pragma unroll
  for (int u = 0; u < kProbeChains; ++u) x[u] = (T)(threadIdx.x + u) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) x[u] = fma(x[u], m, c);
  }
  T s = (T)0;
#pragma unroll
  for (int u = 0; u < kProbeChains; ++u) s += x[u];
  if (s == (T)-1) sink[0] = s;
}

template <typename T>
static cudaError_t run_probe(int iters, double* tflops, cudaStream_t s) {
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return cudaErrorNoDevice;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel<T>,
                                                                kProbeThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int grid = per_sm * dp.num_sms;
  cudaEvent_t a = nullptr, b = nullptr;
  if ((e = cudaEventCreate(&a)) != cudaSuccess) return e;
  if ((e = cudaEventCreate(&b)) != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  const T m = (T)0.9999999, c = (T)1e-7;
  // one untimed launch first (clocks up, code loaded), then the timed one
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, s>>>(iters / 8 + 1, m, c, nullptr);
  count_launch();
  cudaEventRecord(a, s);
  fma_probe_kernel<T><<<grid, kProbeThreads, 0, s>>>(iters, m, c, nullptr);
  count_launch();
  cudaEventRecord(b, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return e;
  const double flops = 2.0 * kProbeChains * (double)iters * kProbeThreads * (double)grid;
  *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  return cudaSuccess;
}

}  // namespace gbla

using namespace gbla;

extern "C" int gbla_fma_peak(int precision, int iters, double* tflops, gbla_stream_t stream) {
  api_clear_error();
  if (precision != 0 && precision != 1) return -1;
  if (iters < 1) return -2;
  if (!tflops) return -3;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = precision == 0 ? run_probe<double>(iters, tflops, s)
                                       : run_probe<float>(iters, tflops, s);
  return api_cuda_status(e, "fma probe", "probe.cu", __LINE__);
}
