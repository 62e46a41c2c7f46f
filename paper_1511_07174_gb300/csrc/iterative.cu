// Building blocks of the library's standalone Krylov solvers (paper section 2:
// the non-stationary methods GMRES and BiCGSTAB next to the direct solvers):
// inner products with a fixed reduction order, and the vector updates of
// BiCGSTAB. Every scalar of the recurrence (rho, alpha, omega, the inner
// products) stays in a device-side state record: the update kernels form
// alpha, beta and omega from it themselves, so one iteration needs no host
// round trip except the residual-norm read that decides when to stop.
#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kDotThreads = 256;
constexpr int kDotMaxCtas = 512;

// Slice of the n elements that CTA c of C owns (fixed, so sums do not depend on timing).
GBLA_DEVINL void dot_slice(int n, int C, int c, int& i0, int& i1) {
  const int per = (n + C - 1) / C;
  i0 = c * per;
  i1 = min(n, i0 + per);
}

// part[k * C + c] = sum over CTA c's slice of x_k[i] * y_k[i], for K pairs.
template <int K>
__global__ void __launch_bounds__(kDotThreads)
    dot_partial_kernel(int n, const double* __restrict__ x0, const double* __restrict__ y0,
                       const double* __restrict__ x1, const double* __restrict__ y1,
                       double* __restrict__ part) {
  __shared__ double red[K][kDotThreads / 32];
  const int C = gridDim.x, c = blockIdx.x;
  int i0, i1;
  dot_slice(n, C, c, i0, i1);
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    acc[0] = fma(x0[i], y0[i], acc[0]);
    if constexpr (K > 1) acc[1] = fma(x1[i], y1[i], acc[1]);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[k][warp] = v;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0.0;
    for (int w = 0; w < kDotThreads / 32; ++w) s += red[threadIdx.x][w];
    part[threadIdx.x * C + c] = s;
  }
}

// out_k = sum_c part[k * C + c], in CTA order (one thread per product).
__global__ void dot_finish_kernel(int C, int K, const double* __restrict__ part, double* out0,
                                  double* out1) {
  const int k = threadIdx.x;
  if (k >= K) return;
  double s = 0.0;
  for (int c = 0; c < C; ++c) s += part[k * C + c];
  *(k == 0 ? out0 : out1) = s;
}

size_t dot_part_doubles() { return (size_t)2 * kDotMaxCtas; }

cudaError_t launch_dots(int n, int K, const double* x0, const double* y0, const double* x1,
                        const double* y1, double* part, double* out0, double* out1,
                        cudaStream_t s) {
  if (K < 1 || K > 2) return cudaErrorInvalidValue;
  int C = (n + 4 * kDotThreads - 1) / (4 * kDotThreads);
  if (C > kDotMaxCtas) C = kDotMaxCtas;
  if (C < 1) C = 1;
  if (K == 1)
    dot_partial_kernel<1><<<C, kDotThreads, 0, s>>>(n, x0, y0, nullptr, nullptr, part);
  else
    dot_partial_kernel<2><<<C, kDotThreads, 0, s>>>(n, x0, y0, x1, y1, part);
  dot_finish_kernel<<<1, 32, 0, s>>>(C, K, part, out0, out1);
  count_launch(2);
  return cudaGetLastError();
}

// ---- BiCGSTAB vector updates (the state's scalars are read, never raced:
// each kernel stores only fields that no thread of the same launch reads).
GBLA_DEVINL double safe_div(double a, double b) { return b != 0.0 ? a / b : 0.0; }

// p = r + beta (p - omega v), beta = (rho' / rho) (alpha / omega)
__global__ void bcg_p_kernel(int n, const double* __restrict__ r, const double* __restrict__ v,
                             double* __restrict__ p, const BcgState* st) {
  const double beta = safe_div(st->rho_new, st->rho) * safe_div(st->alpha, st->omega);
  const double om = st->omega;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    p[i] = fma(beta, fma(-om, v[i], p[i]), r[i]);
}

// alpha = rho' / (r~, v); s = r - alpha v
__global__ void bcg_s_kernel(int n, const double* __restrict__ r, const double* __restrict__ v,
                             double* __restrict__ s, BcgState* st) {
  const double alpha = safe_div(st->rho_new, st->rv);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    s[i] = fma(-alpha, v[i], r[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->alpha = alpha;
    if (st->rho_new == 0.0 || st->rv == 0.0) st->status = 1;  // breakdown
  }
}

// omega = (t, s) / (t, t); x += alpha p^ + omega s^; r = s - omega t; rho = rho'
__global__ void bcg_xr_kernel(int n, double* __restrict__ x, const double* __restrict__ ph,
                              const double* __restrict__ sh, const double* __restrict__ s,
                              const double* __restrict__ t, double* __restrict__ r, BcgState* st) {
  const double alpha = st->alpha;
  const double omega = safe_div(st->ts, st->tt);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    x[i] = fma(omega, sh[i], fma(alpha, ph[i], x[i]));
    r[i] = fma(-omega, t[i], s[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->omega = omega;
    st->rho = st->rho_new;
    if (st->tt == 0.0) st->status = st->status ? st->status : 2;  // t = 0: s solved it, or a breakdown
  }
}

__global__ void bcg_init_kernel(BcgState* st) {
  st->rho = st->alpha = st->omega = 1.0;
  st->rho_new = st->rv = st->ts = st->tt = st->rr = 0.0;
  st->status = 0;
}

static int vec_grid(int n) {
  int bx = (n + 255) / 256;
  return bx > 1024 ? 1024 : (bx < 1 ? 1 : bx);
}

cudaError_t launch_bcg_init(BcgState* st, cudaStream_t s) {
  bcg_init_kernel<<<1, 1, 0, s>>>(st);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_bcg_p(int n, const double* r, const double* v, double* p, const BcgState* st,
                         cudaStream_t s) {
  bcg_p_kernel<<<vec_grid(n), 256, 0, s>>>(n, r, v, p, st);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_bcg_s(int n, const double* r, const double* v, double* sv, BcgState* st,
                         cudaStream_t s) {
  bcg_s_kernel<<<vec_grid(n), 256, 0, s>>>(n, r, v, sv, st);
  count_launch();
  return cudaGetLastError();
}
cudaError_t launch_bcg_xr(int n, double* x, const double* ph, const double* sh, const double* sv,
                          const double* t, double* r, BcgState* st, cudaStream_t s) {
  bcg_xr_kernel<<<vec_grid(n), 256, 0, s>>>(n, x, ph, sh, sv, t, r, st);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gbla
