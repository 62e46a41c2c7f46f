// FP64 residual, norms and the GMRES building blocks (paper section 2: GMRES
// with Gram-Schmidt orthogonalisation and restarts; here the inner solver of
// iterative refinement).
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kResRows = 256;   // rows per CTA (one thread per row)
constexpr int kResCols = 512;   // columns per CTA

size_t residual_work_doubles(int n, int nrhs) {
  const size_t chunks = (size_t)((n + kResCols - 1) / kResCols);
  return chunks * (size_t)(n > 0 ? n : 1) * (size_t)(nrhs > 0 ? nrhs : 1);
}

// part[chunk][c][i] = sum_{j in chunk} A[i, j] X[j, c]   (ABS: |A[i, j]|, X unused).
// NR is the number of right-hand sides of this pass (compile time, so the
// accumulators stay in registers); two interleaved accumulators per sum keep
// two independent FMA chains in flight.
template <bool ABS, int NR>
__global__ void __launch_bounds__(kResRows)
    matvec_partial_kernel(int n, const double* __restrict__ A, int lda,
                          const double* __restrict__ X, int ldx, double* __restrict__ part) {
  __shared__ double xs[kResCols][NR];
  const int i = blockIdx.x * kResRows + threadIdx.x;
  const int chunk = blockIdx.y;
  const int j0 = chunk * kResCols;
  const int nc = min(kResCols, n - j0);
  if (!ABS) {
    for (int idx = threadIdx.x; idx < kResCols * NR; idx += blockDim.x) {
      const int jj = idx % kResCols, c = idx / kResCols;
      xs[jj][c] = jj < nc ? X[(j0 + jj) + (size_t)c * ldx] : 0.0;
    }
    __syncthreads();
  }
  if (i >= n) return;
  double acc0[NR], acc1[NR];
#pragma unroll
  for (int c = 0; c < NR; ++c) acc0[c] = acc1[c] = 0.0;
  const double* a = A + i + (size_t)j0 * lda;
  int jj = 0;
#pragma unroll 4
  for (; jj + 1 < nc; jj += 2) {
    const double v0 = __ldg(a + (size_t)jj * lda);
    const double v1 = __ldg(a + (size_t)(jj + 1) * lda);
    if (ABS) {
      acc0[0] += fabs(v0);
      acc1[0] += fabs(v1);
    } else {
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        acc0[c] = fma(v0, xs[jj][c], acc0[c]);
        acc1[c] = fma(v1, xs[jj + 1][c], acc1[c]);
      }
    }
  }
  if (jj < nc) {
    const double v0 = __ldg(a + (size_t)jj * lda);
    if (ABS) {
      acc0[0] += fabs(v0);
    } else {
#pragma unroll
      for (int c = 0; c < NR; ++c) acc0[c] = fma(v0, xs[jj][c], acc0[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NR; ++c) part[((size_t)chunk * NR + c) * n + i] = acc0[c] + acc1[c];
}

// R[i, c] = B[i, c] - sum_chunk part (or + sum when B == nullptr), fixed order.
__global__ void residual_finish_kernel(int n, int nrhs, int chunks, const double* __restrict__ part,
                                       const double* __restrict__ B, int ldb, double* __restrict__ R,
                                       int ldr) {
  const int c = blockIdx.y;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[((size_t)k * nrhs + c) * n + i];
    R[i + (size_t)c * ldr] = B ? B[i + (size_t)c * ldb] - s : s;
  }
}

cudaError_t launch_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                            const double* B, int ldb, double* R, int ldr, double* work,
                            cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const int chunks = (n + kResCols - 1) / kResCols;
  for (int c0 = 0; c0 < nrhs;) {
    const int left = nrhs - c0;
    const int nc = left >= 8 ? 8 : (left >= 4 ? 4 : (left >= 2 ? 2 : 1));
    dim3 grid((n + kResRows - 1) / kResRows, chunks);
    const double* Xc = X + (size_t)c0 * ldx;
    switch (nc) {
      case 8: matvec_partial_kernel<false, 8><<<grid, kResRows, 0, s>>>(n, A, lda, Xc, ldx, work); break;
      case 4: matvec_partial_kernel<false, 4><<<grid, kResRows, 0, s>>>(n, A, lda, Xc, ldx, work); break;
      case 2: matvec_partial_kernel<false, 2><<<grid, kResRows, 0, s>>>(n, A, lda, Xc, ldx, work); break;
      default: matvec_partial_kernel<false, 1><<<grid, kResRows, 0, s>>>(n, A, lda, Xc, ldx, work); break;
    }
    int bx = (n + 255) / 256;
    if (bx > 512) bx = 512;
    residual_finish_kernel<<<dim3(bx, nc), 256, 0, s>>>(
        n, nc, chunks, work, B ? B + (size_t)c0 * ldb : nullptr, ldb, R + (size_t)c0 * ldr, ldr);
    count_launch(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    c0 += nc;
  }
  return cudaSuccess;
}

__global__ void __launch_bounds__(1024)
    rowsum_max_kernel(int n, int chunks, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double wm[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[(size_t)k * n + i];
    m = fmax(m, s);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0.0;
    v = warp_max(v);
    if (threadIdx.x == 0) out[0] = v;
  }
}

cudaError_t launch_row_abs_sum_max(int n, const double* A, int lda, double* work, double* anorm,
                                   cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(anorm, 0, sizeof(double), s);
  const int chunks = (n + kResCols - 1) / kResCols;
  dim3 grid((n + kResRows - 1) / kResRows, chunks);
  matvec_partial_kernel<true, 1><<<grid, kResRows, 0, s>>>(n, A, lda, nullptr, 0, work);
  rowsum_max_kernel<<<1, 1024, 0, s>>>(n, chunks, work, anorm);
  count_launch(2);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(1024)
    backward_error_finish_kernel(int n, const double* __restrict__ R, int ldr,
                                 const double* __restrict__ X, int ldx,
                                 const double* __restrict__ anorm, double* __restrict__ beta) {
  __shared__ double wr[32], wx[32];
  const int c = blockIdx.x;
  double rm = 0.0, xm = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    rm = fmax(rm, fabs(R[i + (size_t)c * ldr]));
    xm = fmax(xm, fabs(X[i + (size_t)c * ldx]));
  }
  rm = warp_max(rm);
  xm = warp_max(xm);
  if ((threadIdx.x & 31) == 0) {
    wr[threadIdx.x >> 5] = rm;
    wx[threadIdx.x >> 5] = xm;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool ok = threadIdx.x < (blockDim.x >> 5);
    double a = ok ? wr[threadIdx.x] : 0.0, b = ok ? wx[threadIdx.x] : 0.0;
    a = warp_max(a);
    b = warp_max(b);
    if (threadIdx.x == 0) {
      const double den = anorm[0] * b;
      beta[c] = den > 0.0 ? a / den : (a > 0.0 ? __longlong_as_double(0x7ff0000000000000ll) : 0.0);
    }
  }
}

cudaError_t launch_backward_error_finish(int n, int nrhs, const double* R, int ldr, const double* X,
                                         int ldx, const double* anorm, double* beta,
                                         cudaStream_t s) {
  if (nrhs <= 0) return cudaSuccess;
  backward_error_finish_kernel<<<nrhs, 1024, 0, s>>>(n, R, ldr, X, ldx, anorm, beta);
  count_launch();
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// One Arnoldi step with modified Gram-Schmidt, cooperative over C CTAs that
// each own a contiguous slice of rows:
//   for i = 0..j: h_ij = v_i . w; w -= h_ij v_i      (one grid barrier each)
//   h_{j+1,j} = ||w||_2;  v_{j+1} = w / h_{j+1,j}
// then (CTA 0) the previous Givens rotations are applied to column j of H, a
// new rotation zeroes h_{j+1,j}, g is updated and |g_{j+1}| is stored in
// st->res. With j = -1 the call only normalises: v_0 = w / ||w||, g_0 = ||w||.
// Partial sums go through per-CTA slots and are added in CTA order, so the
// result does not depend on timing.
struct GmresState {
  double res;      // |g_{j+1}| after the step (or ||w|| for j = -1)
  double pad;
};

constexpr int kMgsThreads = 256;

__device__ double mgs_block_sum(double v, double* red) {
  v = warp_sum(v);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(kMgsThreads)
    mgs_step_kernel(int n, int j, int ldv, double* __restrict__ V, const double* __restrict__ w_in,
                    double* __restrict__ H, int ldh, double* __restrict__ cs, double* __restrict__ sn,
                    double* __restrict__ g, GmresState* st, double* __restrict__ slots,
                    unsigned* __restrict__ counter, int* info, uint64_t wait_ns) {
  extern __shared__ double wsl[];  // this CTA's slice of w
  __shared__ double red[kMgsThreads / 32];
  __shared__ double s_h;
  __shared__ int s_abort;
  const int C = gridDim.x, c = blockIdx.x;
  const int S = (n + C - 1) / C;
  const int i0 = c * S;
  const int cnt = max(0, min(S, n - i0));
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) wsl[t] = w_in[i0 + t];
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  unsigned phase = 0;
  auto grid_sum = [&](double local) -> bool {
    // slot parity by phase; returns false on timeout
    double bs = mgs_block_sum(local, red);
    const int par = phase & 1;
    if (threadIdx.x == 0) {
      slots[par * C + c] = bs;
      __threadfence();
      atomicAdd(counter, 1u);
      bool ok = gbla_wait_geq(counter, (phase + 1) * (unsigned)C, wait_ns);
      __threadfence();
      if (!ok) {
        gbla_flag_timeout(info);
        s_abort = 1;
      } else {
        double tot = 0.0;
        for (int q = 0; q < C; ++q) tot += __ldcg(&slots[par * C + q]);
        s_h = tot;
      }
    }
    __syncthreads();
    ++phase;
    return s_abort == 0;
  };
  for (int i = 0; i <= j; ++i) {
    const double* vi = V + (size_t)i * ldv + i0;
    double loc = 0.0;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) loc = fma(vi[t], wsl[t], loc);
    if (!grid_sum(loc)) return;
    const double h = s_h;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) wsl[t] = fma(-h, vi[t], wsl[t]);
    if (c == 0 && threadIdx.x == 0) H[i + (size_t)j * ldh] = h;
    __syncthreads();
  }
  double loc = 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) loc = fma(wsl[t], wsl[t], loc);
  if (!grid_sum(loc)) return;
  const double nrm = sqrt(s_h);
  double* vn = V + (size_t)(j + 1) * ldv + i0;
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) vn[t] = nrm > 0.0 ? wsl[t] * inv : 0.0;
  if (c == 0 && threadIdx.x == 0) {
    if (j < 0) {
      g[0] = nrm;
      st->res = nrm;
    } else {
      double* hc = H + (size_t)j * ldh;
      hc[j + 1] = nrm;
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * hc[i] + sn[i] * hc[i + 1];
        hc[i + 1] = -sn[i] * hc[i] + cs[i] * hc[i + 1];
        hc[i] = t;
      }
      const double rho = hypot(hc[j], hc[j + 1]);
      double cj = 1.0, sj = 0.0;
      if (rho != 0.0) {
        cj = hc[j] / rho;
        sj = hc[j + 1] / rho;
      }
      cs[j] = cj;
      sn[j] = sj;
      hc[j] = rho;
      hc[j + 1] = 0.0;
      g[j + 1] = -sj * g[j];
      g[j] = cj * g[j];
      st->res = fabs(g[j + 1]);
    }
  }
}

cudaError_t launch_mgs_step(int n, int j, double* V, int ldv, const double* w, double* H, int ldh,
                            double* cs, double* sn, double* g, void* st, double* slots,
                            unsigned* counter, int* info, cudaStream_t s) {
  const DeviceProps& dp = device_props();
  int C = (n + 255) / 256;
  if (C > dp.num_sms) C = dp.num_sms;
  if (C < 1) C = 1;
  const int S = (n + C - 1) / C;
  const size_t smem = (size_t)S * sizeof(double);
  if (smem > dp.smem_optin) return cudaErrorInvalidValue;
  cudaError_t ea = ensure_dyn_smem(mgs_step_kernel, smem);
  if (ea != cudaSuccess) return ea;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  GmresState* stp = static_cast<GmresState*>(st);
  uint64_t wait_ns = wait_timeout_ns();
  void* args[] = {&n, &j, &ldv, &V, &w, &H, &ldh, &cs, &sn, &g, &stp, &slots, &counter, &info, &wait_ns};
  count_launch();
  return cudaLaunchCooperativeKernel((const void*)mgs_step_kernel, dim3(C), dim3(kMgsThreads), args,
                                     smem, s);
}

size_t mgs_slots_doubles() {
  const DeviceProps& dp = device_props();
  return (size_t)2 * (dp.num_sms > 0 ? dp.num_sms : 160);
}

// x += V(:, 0:k) y with y = R^{-1} g(0:k), R the k x k upper triangle of the
// rotated Hessenberg matrix. Every CTA re-solves the small triangle (k <= 128)
// in shared memory, then updates its rows of x.
__global__ void __launch_bounds__(256)
    gmres_update_kernel(int n, int k, const double* __restrict__ V, int ldv,
                        const double* __restrict__ H, int ldh, const double* __restrict__ g,
                        double* __restrict__ x) {
  __shared__ double y[128];
  if (threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; --i) {
      double sacc = g[i];
      for (int t = i + 1; t < k; ++t) sacc -= H[i + (size_t)t * ldh] * y[t];
      y[i] = sacc / H[i + (size_t)i * ldh];
    }
  }
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int t = 0; t < k; ++t) acc = fma(V[i + (size_t)t * ldv], y[t], acc);
    x[i] += acc;
  }
}

// out = a x + b y (FP64 vectors; out may alias x or y).
__global__ void axpby_kernel(int n, double a, const double* x, double b, const double* y,
                             double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = fma(a, x[i], b * y[i]);
}

cudaError_t launch_axpby(int n, double a, const double* x, double b, const double* y, double* out,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int bx = (n + 255) / 256;
  if (bx > 1024) bx = 1024;
  axpby_kernel<<<bx, 256, 0, s>>>(n, a, x, b, y, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_gmres_update(int n, int k, const double* V, int ldv, const double* H, int ldh,
                                const double* g, double* x, cudaStream_t s) {
  if (n <= 0 || k <= 0) return cudaSuccess;
  if (k > 128) return cudaErrorInvalidValue;
  int bx = (n + 255) / 256;
  if (bx > 1024) bx = 1024;
  gmres_update_kernel<<<bx, 256, 0, s>>>(n, k, V, ldv, H, ldh, g, x);
  count_launch();
  return cudaGetLastError();
}

}  // namespace gbla
