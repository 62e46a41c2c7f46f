// Batched LU with partial pivoting and solve for many small systems of uneven
// size in one persistent launch (paper section 2 -- factor, then forward and
// back substitution -- applied to every system of the batch), and the same
// for Cholesky (further down).
//
// A fixed grid (SMs x CTAs per SM) pulls system indices from an atomic
// counter in the caller's order (largest first balances the tail). One CTA
// takes one whole system at a time:
//   * the matrix is copied into shared memory when it fits (n <= smem limit),
//     otherwise it is factored in place in global memory (L2-resident);
//   * unblocked right-looking GEPP: block-wide argmax of |a_ij| (ties to the
//     lowest row), interchange across all columns, scaling by the reciprocal
//     of the pivot, rank-1 update of the trailing block;
//   * the right-hand sides are copied to shared memory, permuted, and solved
//     by forward (unit L) and back (U) substitution;
//   * the factors, pivots, solutions and info are written back.
// Nothing here waits on another CTA.
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace gbla {

constexpr int kBatchMaxRhs = 4;

// solve_only: the matrices already hold L\U and ipiv the pivots (a previous
// factor-only launch); only the right-hand sides are solved and written.
template <typename T>
__global__ void batched_lu_kernel(int batch, const int* __restrict__ nv, T* const* __restrict__ Av,
                                  const int* __restrict__ ldav, int* const* __restrict__ ipivv,
                                  const int* __restrict__ nrhsv, T* const* __restrict__ Bv,
                                  const int* __restrict__ ldbv, int* __restrict__ infov,
                                  const int* __restrict__ order, unsigned* __restrict__ counter,
                                  int smem_n, int solve_only) {
  extern __shared__ unsigned char smraw[];
  T* sA = reinterpret_cast<T*>(smraw);                        // smem_n x smem_n (ld = smem_n)
  T* sB = sA + (size_t)smem_n * smem_n;                       // smem_n x kBatchMaxRhs
  __shared__ int s_idx, s_p;
  __shared__ T s_rp;
  __shared__ double s_wv[32];
  __shared__ int s_wi[32];
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nth >> 5;

  while (true) {
    if (tid == 0) s_idx = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= batch) break;
    const int sys = order ? order[idx] : idx;
    const int n = nv[sys];
    const int nrhs = min(nrhsv ? nrhsv[sys] : 0, kBatchMaxRhs);
    T* gA = Av[sys];
    const int glda = ldav[sys];
    int* piv = ipivv[sys];
    const bool in_smem = n <= smem_n;
    T* a = in_smem ? sA : gA;
    const int ld = in_smem ? smem_n : glda;
    if (in_smem)
      for (int e = tid; e < n * n; e += nth) {
        const int r = e % n, c = e / n;
        sA[r + c * smem_n] = gA[r + (size_t)c * glda];
      }
    int info = 0;
    __syncthreads();
    for (int j = 0; j < (solve_only ? 0 : n); ++j) {
      // argmax of |a_ij|, i >= j
      double bv = -1.0;
      int bi = INT_MAX;
      for (int i = j + tid; i < n; i += nth) argmax_merge(bv, bi, fabs((double)a[i + (size_t)j * ld]), i);
      warp_argmax(bv, bi);
      if (lane == 0) {
        s_wv[warp] = bv;
        s_wi[warp] = bi;
      }
      __syncthreads();
      if (warp == 0) {
        double v = lane < nw ? s_wv[lane] : -1.0;
        int i = lane < nw ? s_wi[lane] : INT_MAX;
        warp_argmax(v, i);
        if (lane == 0) {
          s_p = i;
          piv[j] = i + 1;
          const T pv = a[i + (size_t)j * ld];
          s_rp = pv != (T)0 ? (T)1 / pv : (T)0;
        }
      }
      __syncthreads();
      const int p = s_p;
      const T rp = s_rp;
      if (rp == (T)0 && info == 0) info = j + 1;
      if (p != j)
        for (int c = tid; c < n; c += nth) {
          const T t = a[j + (size_t)c * ld];
          a[j + (size_t)c * ld] = a[p + (size_t)c * ld];
          a[p + (size_t)c * ld] = t;
        }
      __syncthreads();
      if (rp != (T)0)
        for (int i = j + 1 + tid; i < n; i += nth) a[i + (size_t)j * ld] *= rp;
      __syncthreads();
      const int m = n - j - 1;
      for (int e = tid; e < m * m; e += nth) {
        const int i = j + 1 + e % m, k = j + 1 + e / m;
        a[i + (size_t)k * ld] = fma(-a[i + (size_t)j * ld], a[j + (size_t)k * ld], a[i + (size_t)k * ld]);
      }
      __syncthreads();
    }
    if (in_smem && !solve_only)
      for (int e = tid; e < n * n; e += nth) {
        const int r = e % n, c = e / n;
        gA[r + (size_t)c * glda] = sA[r + c * smem_n];
      }
    if (tid == 0 && infov && !solve_only) infov[sys] = info;
    // solve: B <- U^{-1} L^{-1} P B, right-hand sides staged in shared memory
    if (nrhs > 0) {
      T* gB = Bv[sys];
      const int gldb = ldbv[sys];
      T* b = sB;
      const int ldbs = smem_n;
      const bool b_in_smem = n <= smem_n;
      T* bb = b_in_smem ? b : gB;
      const int lbb = b_in_smem ? ldbs : gldb;
      if (b_in_smem)
        for (int e = tid; e < n * nrhs; e += nth) {
          const int r = e % n, c = e / n;
          b[r + c * ldbs] = gB[r + (size_t)c * gldb];
        }
      __syncthreads();
      if (tid < nrhs)
        for (int j = 0; j < n; ++j) {
          const int p = piv[j] - 1;
          if (p > j && p < n) {  // pivots outside j+1 .. n are no interchange
            const T t = bb[j + (size_t)tid * lbb];
            bb[j + (size_t)tid * lbb] = bb[p + (size_t)tid * lbb];
            bb[p + (size_t)tid * lbb] = t;
          }
        }
      __syncthreads();
      for (int j = 0; j < n; ++j) {
        for (int e = tid; e < (n - j - 1) * nrhs; e += nth) {
          const int i = j + 1 + e % (n - j - 1), c = e / (n - j - 1);
          bb[i + (size_t)c * lbb] = fma(-a[i + (size_t)j * ld], bb[j + (size_t)c * lbb], bb[i + (size_t)c * lbb]);
        }
        __syncthreads();
      }
      for (int j = n - 1; j >= 0; --j) {
        if (tid < nrhs) bb[j + (size_t)tid * lbb] = bb[j + (size_t)tid * lbb] / a[j + (size_t)j * ld];
        __syncthreads();
        for (int e = tid; e < j * nrhs; e += nth) {
          const int i = e % j, c = e / j;
          bb[i + (size_t)c * lbb] = fma(-a[i + (size_t)j * ld], bb[j + (size_t)c * lbb], bb[i + (size_t)c * lbb]);
        }
        __syncthreads();
      }
      if (b_in_smem)
        for (int e = tid; e < n * nrhs; e += nth) {
          const int r = e % n, c = e / n;
          gB[r + (size_t)c * gldb] = b[r + c * ldbs];
        }
    }
    __syncthreads();
  }
}

// Batched Cholesky A = L L^t and solve (paper section 2 for symmetric
// positive definite systems) with the same persistent structure: one CTA per
// system, the lower triangle in shared memory when it fits. Column j:
// d = a_jj (already reduced by the earlier columns); d <= 0 (or NaN) stops the
// factorisation with info = j + 1 and leaves that system's right-hand sides
// untouched; otherwise l_jj = sqrt(d), l_ij = a_ij * (1 / l_jj) and
// a_ik -= l_ij l_kj for i >= k > j. Only the lower triangle is read or
// written. The solve is L y = b (forward) then L^t x = y (backward).
template <typename T>
__global__ void batched_chol_kernel(int batch, const int* __restrict__ nv, T* const* __restrict__ Av,
                                    const int* __restrict__ ldav, const int* __restrict__ nrhsv,
                                    T* const* __restrict__ Bv, const int* __restrict__ ldbv,
                                    int* __restrict__ infov, const int* __restrict__ order,
                                    unsigned* __restrict__ counter, int smem_n, int solve_only) {
  extern __shared__ unsigned char smraw[];
  T* sA = reinterpret_cast<T*>(smraw);                        // smem_n x smem_n (ld = smem_n)
  T* sB = sA + (size_t)smem_n * smem_n;                       // smem_n x kBatchMaxRhs
  __shared__ int s_idx, s_bad;
  __shared__ T s_rl;
  const int tid = threadIdx.x, nth = blockDim.x;

  while (true) {
    if (tid == 0) s_idx = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int idx = s_idx;
    __syncthreads();
    if (idx >= batch) break;
    const int sys = order ? order[idx] : idx;
    const int n = nv[sys];
    const int nrhs = min(nrhsv ? nrhsv[sys] : 0, kBatchMaxRhs);
    T* gA = Av[sys];
    const int glda = ldav[sys];
    const bool in_smem = n <= smem_n;
    T* a = in_smem ? sA : gA;
    const int ld = in_smem ? smem_n : glda;
    if (in_smem)
      for (int e = tid; e < n * n; e += nth) {
        const int r = e % n, c = e / n;
        if (r >= c) sA[r + c * smem_n] = gA[r + (size_t)c * glda];
      }
    if (tid == 0) s_bad = 0;
    int info = 0;
    __syncthreads();
    for (int j = 0; j < (solve_only ? 0 : n); ++j) {
      if (tid == 0) {
        const T d = a[j + (size_t)j * ld];
        if (!(d > (T)0)) {
          s_bad = j + 1;
        } else {
          const T l = sqrt(d);
          a[j + (size_t)j * ld] = l;
          s_rl = (T)1 / l;
        }
      }
      __syncthreads();
      if (s_bad) {
        info = s_bad;
        break;
      }
      const T rl = s_rl;
      for (int i = j + 1 + tid; i < n; i += nth) a[i + (size_t)j * ld] *= rl;
      __syncthreads();
      const int m = n - j - 1;
      for (int e = tid; e < m * m; e += nth) {
        const int i = j + 1 + e % m, k = j + 1 + e / m;
        if (i >= k) a[i + (size_t)k * ld] = fma(-a[i + (size_t)j * ld], a[k + (size_t)j * ld], a[i + (size_t)k * ld]);
      }
      __syncthreads();
    }
    if (in_smem && !solve_only)
      for (int e = tid; e < n * n; e += nth) {
        const int r = e % n, c = e / n;
        if (r >= c) gA[r + (size_t)c * glda] = sA[r + c * smem_n];
      }
    if (tid == 0 && infov && !solve_only) infov[sys] = info;
    if (nrhs > 0 && info == 0) {
      T* gB = Bv[sys];
      const int gldb = ldbv[sys];
      T* bb = in_smem ? sB : gB;
      const int lbb = in_smem ? smem_n : gldb;
      if (in_smem)
        for (int e = tid; e < n * nrhs; e += nth) {
          const int r = e % n, c = e / n;
          sB[r + c * smem_n] = gB[r + (size_t)c * gldb];
        }
      __syncthreads();
      // L y = b
      for (int j = 0; j < n; ++j) {
        if (tid < nrhs) bb[j + (size_t)tid * lbb] = bb[j + (size_t)tid * lbb] / a[j + (size_t)j * ld];
        __syncthreads();
        for (int e = tid; e < (n - j - 1) * nrhs; e += nth) {
          const int i = j + 1 + e % (n - j - 1), c = e / (n - j - 1);
          bb[i + (size_t)c * lbb] = fma(-a[i + (size_t)j * ld], bb[j + (size_t)c * lbb], bb[i + (size_t)c * lbb]);
        }
        __syncthreads();
      }
      // L^t x = y: (L^t)_{ij} = l_ji
      for (int j = n - 1; j >= 0; --j) {
        if (tid < nrhs) bb[j + (size_t)tid * lbb] = bb[j + (size_t)tid * lbb] / a[j + (size_t)j * ld];
        __syncthreads();
        for (int e = tid; e < j * nrhs; e += nth) {
          const int i = e % j, c = e / j;
          bb[i + (size_t)c * lbb] = fma(-a[j + (size_t)i * ld], bb[j + (size_t)c * lbb], bb[i + (size_t)c * lbb]);
        }
        __syncthreads();
      }
      if (in_smem)
        for (int e = tid; e < n * nrhs; e += nth) {
          const int r = e % n, c = e / n;
          gB[r + (size_t)c * gldb] = sB[r + c * smem_n];
        }
    }
    __syncthreads();
  }
}

// Largest n whose matrix and right-hand sides fit the shared memory of one CTA.
template <typename T>
int batched_smem_n(int ctas_per_sm) {
  const DeviceProps& dp = device_props();
  size_t cap = dp.smem_optin > 2048 ? dp.smem_optin - 2048 : 0;
  if (ctas_per_sm > 1) cap = cap / ctas_per_sm;
  int n = 0;
  while ((size_t)((n + 1) * (n + 1) + (n + 1) * kBatchMaxRhs) * sizeof(T) <= cap) ++n;
  return n;
}

template <typename T>
cudaError_t launch_lu_batched(int batch, const int* n, T* const* A, const int* lda, int* const* ipiv,
                              const int* nrhs, T* const* B, const int* ldb, int* info,
                              const int* order, int max_n, int threads, int ctas_per_sm,
                              unsigned* counter, bool solve_only, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const DeviceProps& dp = device_props();
  if (threads <= 0) threads = 256;
  if (ctas_per_sm <= 0) ctas_per_sm = 1;
  int smem_n = batched_smem_n<T>(ctas_per_sm);
  if (smem_n > max_n) smem_n = max_n;
  const size_t smem = (size_t)(smem_n * smem_n + smem_n * kBatchMaxRhs) * sizeof(T);
  cudaError_t e = ensure_dyn_smem(batched_lu_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int grid = dp.num_sms * ctas_per_sm;
  if (grid > batch) grid = batch;
  batched_lu_kernel<T><<<grid, threads, smem, s>>>(batch, n, A, lda, ipiv, nrhs, B, ldb, info, order,
                                                   counter, smem_n, solve_only ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chol_batched(int batch, const int* n, T* const* A, const int* lda, const int* nrhs,
                                T* const* B, const int* ldb, int* info, const int* order, int max_n,
                                int threads, int ctas_per_sm, unsigned* counter, bool solve_only,
                                cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const DeviceProps& dp = device_props();
  if (threads <= 0) threads = 256;
  if (ctas_per_sm <= 0) ctas_per_sm = 1;
  int smem_n = batched_smem_n<T>(ctas_per_sm);
  if (smem_n > max_n) smem_n = max_n;
  const size_t smem = (size_t)(smem_n * smem_n + smem_n * kBatchMaxRhs) * sizeof(T);
  cudaError_t e = ensure_dyn_smem(batched_chol_kernel<T>, smem);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int grid = dp.num_sms * ctas_per_sm;
  if (grid > batch) grid = batch;
  batched_chol_kernel<T><<<grid, threads, smem, s>>>(batch, n, A, lda, nrhs, B, ldb, info, order,
                                                     counter, smem_n, solve_only ? 1 : 0);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_chol_batched<double>(int, const int*, double* const*, const int*, const int*,
                                                 double* const*, const int*, int*, const int*, int, int,
                                                 int, unsigned*, bool, cudaStream_t);
template cudaError_t launch_chol_batched<float>(int, const int*, float* const*, const int*, const int*,
                                                float* const*, const int*, int*, const int*, int, int,
                                                int, unsigned*, bool, cudaStream_t);

template cudaError_t launch_lu_batched<double>(int, const int*, double* const*, const int*, int* const*,
                                               const int*, double* const*, const int*, int*, const int*,
                                               int, int, int, unsigned*, bool, cudaStream_t);
template cudaError_t launch_lu_batched<float>(int, const int*, float* const*, const int*, int* const*,
                                              const int*, float* const*, const int*, int*, const int*,
                                              int, int, int, unsigned*, bool, cudaStream_t);

}  // namespace gbla
