// Host-side declarations shared by the translation units of libgbla (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/gbla.h"

namespace gbla {

// ---- process-wide settings ------------------------------------------------
uint64_t wait_timeout_ns();
int substitution_ctas();  // cap on the refinement substitution's persistent grid (0: one per SM)
bool lookahead_enabled();  // factor the next outer block's panels during the trailing update

struct DeviceProps {
  int device = -1;
  int num_sms = 0;
  int coop = 0;
  size_t smem_optin = 0;
};
const DeviceProps& device_props();

// Raise a kernel's dynamic shared-memory limit to at least `bytes` (tracked
// per kernel; the limit must leave room for the kernel's static shared
// memory). Returns cudaErrorInvalidValue when the request cannot fit.
cudaError_t ensure_dyn_smem_ptr(const void* func, size_t bytes);
template <typename F>
cudaError_t ensure_dyn_smem(F* func, size_t bytes) {
  return ensure_dyn_smem_ptr(reinterpret_cast<const void*>(func), bytes);
}

// ---- workspace carving -----------------------------------------------------
struct Carver {
  char* base;
  size_t cap;
  size_t off = 0;
  bool ok = true;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (base == nullptr) {  // sizing pass
      off += bytes;
      return nullptr;
    }
    if (off + bytes > cap) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// ---- last-error record of the C entry points (thread-local) ------------------
void api_clear_error();
// GBLA_OK for cudaSuccess; otherwise records the first failure of the call
// (the expression text and line) and returns GBLA_ERR_CUDA.
int api_cuda_status(cudaError_t e, const char* what, const char* file, int line);

// ---- instrumentation -----------------------------------------------------------
// Kernel groups that can be bracketed with CUDA events (gbla_prof_*).
enum KernelKind {
  KK_PANEL = 0,
  KK_LASWP,
  KK_TRSM,
  KK_GEMM_SIMT,
  KK_GEMM_TC,
  KK_CONVERT,
  KK_TRSV,
  KK_MATVEC,
  KK_MGS,
  KK_UPDATE,
  KK_PERM,
  KK_COPY,
  KK_BATCHED,
  KK_COUNT
};
void count_launch(int k = 1);                 // every kernel launch of the library
void prof_begin(int kind, cudaStream_t s);    // no-op unless the kind is enabled
void prof_end(int kind, cudaStream_t s);

// ---- precision kinds of the mixed trailing update ---------------------------
inline bool prec_is_tensor(int p) { return p >= GBLA_PREC_TF32 && p <= GBLA_PREC_BF16X3; }
inline bool prec_is_split(int p) { return p == GBLA_PREC_FP16X3 || p == GBLA_PREC_BF16X3; }
// tcgen05 operand kind executing the update
inline int prec_mma_kind(int p) {
  return p == GBLA_PREC_FP16X3 ? GBLA_PREC_FP16 : (p == GBLA_PREC_BF16X3 ? GBLA_PREC_BF16 : p);
}
// K-major copies hold kmult * K elements per row ([hi|hi|lo] for L21, [hi|lo|hi] for U12)
inline int prec_kmult(int p) { return prec_is_split(p) ? 3 : 1; }

// ---- kernel launchers (all stream-ordered; return cudaError_t) -------------
constexpr int kPanelWidth = 32;  // inner panel width handled by the panel kernels
constexpr int kPanelSlotW = 72;  // doubles per published candidate slot
// The L2-exchange panel kernels use at most kPanelMaxSms CTAs.
constexpr int kPanelMaxSms = 256;
// Layout of the panel scratch (panel_slots_doubles() doubles, zeroed once per
// factorisation): exchange slots for up to kPanelMaxSms CTAs (two parities),
// then kInnerCounters words for the fused inner update's per-column-tile
// counters.
constexpr size_t kPanelExchangeDoubles = (size_t)2 * (kPanelMaxSms + 1) * kPanelSlotW;
constexpr int kInnerCounters = 64;

// Exchange area of the panel kernels. It must be zeroed once before the
// first panel of a factorisation; panel_index (distinct for every panel of
// one factorisation, < 2^25) tags the words. A is the panel's top-left
// element (row = column = row0, m rows below it including itself, w <= 32
// columns). Besides factoring the panel, the launch applies the panel's row
// interchanges to the nleft columns left of it and the nright columns right
// of it (the rest of its outer block).
size_t panel_slots_doubles();

template <typename Ts>
cudaError_t launch_panel(Ts* A, int lda, int m, int w, int row0, int* ipiv, int* info,
                         double* slots, unsigned panel_index, int nleft, int nright,
                         cudaStream_t s);

// Row interchanges of one outer block (ipiv[0 .. kb): 1-based absolute rows,
// the block starting at row k0, kb <= 256) applied, in order, to columns
// [0, skip_lo) and [skip_hi, ncols) of the nrows x ncols matrix A. No waits.
template <typename T>
cudaError_t launch_laswp_block(T* A, int lda, int ncols, int nrows, int k0, int kb, const int* ipiv,
                               int skip_lo, int skip_hi, cudaStream_t s);

// The interchanges of the columns left of every outer block, applied once
// after the last block (a permutation gather per column). work:
// left_perm_ints(n, nb) ints. Possible when left_deferred_fits<T>(n, nb)
// (a row permutation and a column segment fit in one CTA's shared memory).
size_t left_perm_ints(int n, int nb);
template <typename T>
bool left_deferred_fits(int n, int nb);
template <typename T>
cudaError_t launch_left_interchanges(T* A, int lda, int n, int nb, const int* ipiv, int* work,
                                     cudaStream_t s);

// B (w x N, ldb) <- L^{-1} B with L unit lower (w x w, ldl). Tc: arithmetic type.
// out_kind: 0 none, GBLA_PREC_BF16/FP16/TF32 -> also write a K-major copy of
// the result (column j at outK + j*ldk, 2- or 4-byte elements) with one
// power-of-two scale exponent per column (outE[j]; 0 for TF32).
template <typename Ts, typename Tc>
cudaError_t launch_trsm_lunit(const Ts* L, int ldl, Ts* B, int ldb, int w, int N, int out_kind,
                              void* outK, int ldk, int* outE, cudaStream_t s);

// Inner step of the blocked LU for a 32-column panel whose top-left element
// is P: U12 = L11^{-1} A12 (L11 the unit lower 32 x 32 block at P, A12 the
// 32 x N block right of it) and A22 -= L21 U12 (M x N, below A12), in one
// launch. counters: kInnerCounters zeroed words (left zeroed on return).
template <typename T>
cudaError_t launch_inner_update(int M, int N, T* P, int lda, unsigned* counters, cudaStream_t s);

// C = alpha * A * op(B) + beta * C (column-major). transB: op(B) = B^t with B
// stored N x K. lower: only elements with row >= col are written.
template <typename T>
cudaError_t launch_gemm_simt(int M, int N, int K, T alpha, const T* A, int lda, const T* B,
                             int ldb, bool transB, T beta, T* C, int ldc, bool lower,
                             cudaStream_t s);

// K-major low-precision copy of an FP32 M x K block (rows scaled per row).
// right: the split kinds' right-operand pattern [hi | lo | hi] (else [hi | hi | lo]).
cudaError_t launch_convert_rows(const float* F, int ldf, int M, int K, int kind, void* outK,
                                int ldk, int* outE, bool right, cudaStream_t s);

// F = fp32(A) (m x n); lower: only the elements on or below the diagonal.
cudaError_t launch_copy_d2f(const double* A, int lda, float* F, int ldf, int m, int n,
                            cudaStream_t s, bool lower = false);

// tcgen05 trailing update: C (M x N FP32) -= 2^-eA[i] * (A_k B_k^t)[i,j] * 2^-eB[j].
// A_k: M rows of K elements (row stride ldak elements), B_k: N rows of K (ldbk).
// lower (M == N): only the 128 x 128 tiles on or below the diagonal (the
// diagonal tiles are updated whole, upper part included).
// grid_cap > 0: at most that many persistent CTAs (the rest of the GPU stays
// free for work on another stream).
cudaError_t launch_gemm_tc(int kind, int M, int N, int K, const void* Ak, int ldak,
                           const void* Bk, int ldbk, const int* eA, const int* eB, float* C,
                           int ldc, int* info, bool lower, cudaStream_t s, int grid_cap = 0);

// ---- triangular solves ------------------------------------------------------
// uplo_lower: the stored triangle; trans: solve with its transpose; unit: unit diagonal.
// X (n x nrhs, ldx) FP64 is overwritten in place. flags: >= ceil(n/64)+1 uints.
template <typename Ts>
cudaError_t launch_trsv(bool lower, bool trans, bool unit, int n, int nrhs, const Ts* T, int ldt,
                        double* X, int ldx, unsigned* flags, int* info, cudaStream_t s);
size_t trsv_flags_count(int n, int nrhs);

// Preconditioner apply with inverted 64 x 64 diagonal blocks (one RHS).
// Dinv holds diag_inv_doubles(n) doubles per triangular factor.
size_t diag_inv_doubles(int n);
template <typename Ts>
cudaError_t launch_diag_inv(bool lower, bool unit, int n, const Ts* T, int ldt, double* Dinv,
                            cudaStream_t s);
// X <- T^{-1} rhs (X and rhs distinct; X is overwritten, flags: one uint).
template <typename Ts>
cudaError_t launch_trsv_inv(bool lower, int n, const Ts* T, int ldt, const double* Dinv,
                            const double* rhs, double* X, unsigned* flags, int* info,
                            cudaStream_t s);

// ipiv == nullptr: the identity
cudaError_t launch_ipiv_to_perm(int n, const int* ipiv, int* perm, cudaStream_t s);
// dst[i, c] = src[perm[i], c] (forward) or dst[perm[i], c] = src[i, c] (inverse)
cudaError_t launch_permute_rows(int n, int nrhs, const int* perm, bool inverse, const double* src,
                                int lds, double* dst, int ldd, cudaStream_t s);

// ---- residual / norms / GMRES -----------------------------------------------
// R = B - A X (or R = A X when B == nullptr); partial sums in work (chunks x n x nrhs doubles).
size_t residual_work_doubles(int n, int nrhs);
cudaError_t launch_residual(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                            const double* B, int ldb, double* R, int ldr, double* work,
                            cudaStream_t s);
// anorm[0] = max_i sum_j |a_ij|; work >= residual_work_doubles(n, 1)
cudaError_t launch_row_abs_sum_max(int n, const double* A, int lda, double* work, double* anorm,
                                   cudaStream_t s);
// beta[c] = max|R(:,c)| / (anorm * max|X(:,c)|)
cudaError_t launch_backward_error_finish(int n, int nrhs, const double* R, int ldr,
                                         const double* X, int ldx, const double* anorm,
                                         double* beta, cudaStream_t s);

// GMRES pieces (krylov.cu). st points to a device GmresState {double res, pad}.
size_t mgs_slots_doubles();
cudaError_t launch_mgs_step(int n, int j, double* V, int ldv, const double* w, double* H, int ldh,
                            double* cs, double* sn, double* g, void* st, double* slots,
                            unsigned* counter, int* info, cudaStream_t s);
// out = a x + b y (FP64 vectors; out may alias x or y)
cudaError_t launch_axpby(int n, double a, const double* x, double b, const double* y, double* out,
                         cudaStream_t s);
cudaError_t launch_gmres_update(int n, int k, const double* V, int ldv, const double* H, int ldh,
                                const double* g, double* x, cudaStream_t s);

// ---- standalone Krylov solvers (iterative.cu) --------------------------------
// out0 = (x0, y0) [, out1 = (x1, y1)] for K = 1 [2]; fixed summation order.
size_t dot_part_doubles();
cudaError_t launch_dots(int n, int K, const double* x0, const double* y0, const double* x1,
                        const double* y1, double* part, double* out0, double* out1,
                        cudaStream_t s);
// Scalars of the BiCGSTAB recurrence, kept on the device.
struct BcgState {
  double rho, rho_new, alpha, omega, rv, ts, tt, rr;
  int status;  // 0, 1 = breakdown (rho' or (r~, v) vanished), 2 = t vanished
  int pad;
};
cudaError_t launch_bcg_init(BcgState* st, cudaStream_t s);
cudaError_t launch_bcg_p(int n, const double* r, const double* v, double* p, const BcgState* st,
                         cudaStream_t s);
cudaError_t launch_bcg_s(int n, const double* r, const double* v, double* sv, BcgState* st,
                         cudaStream_t s);
cudaError_t launch_bcg_xr(int n, double* x, const double* ph, const double* sh, const double* sv,
                          const double* t, double* r, BcgState* st, cudaStream_t s);

// C = alpha * U V^t + beta * C (FP64; any k, in passes of 16)
cudaError_t launch_rank_k(int m, int n, int k, double alpha, const double* U, int ldu,
                          const double* V, int ldv, double beta, double* C, int ldc,
                          cudaStream_t s);

// ---- batched LU + solve (batched.cu) -----------------------------------------
// solve_only: A holds the factors (and ipiv the pivots) of an earlier
// factor-only launch; only the right-hand sides are solved.
template <typename T>
cudaError_t launch_lu_batched(int batch, const int* n, T* const* A, const int* lda, int* const* ipiv,
                              const int* nrhs, T* const* B, const int* ldb, int* info,
                              const int* order, int max_n, int threads, int ctas_per_sm,
                              unsigned* counter, bool solve_only, cudaStream_t s);

template <typename T>
cudaError_t launch_chol_batched(int batch, const int* n, T* const* A, const int* lda, const int* nrhs,
                                T* const* B, const int* ldb, int* info, const int* order, int max_n,
                                int threads, int ctas_per_sm, unsigned* counter, bool solve_only,
                                cudaStream_t s);

// ---- Cholesky (chol.cu) ------------------------------------------------------
// nb: outer block width, a multiple of 64 up to 256 (0: 64)
cudaError_t launch_chol(int n, double* A, int lda, int nb, int* info, cudaStream_t s);
// Mixed-precision Cholesky of the FP32 lower triangle of F (see chol.cu); the
// strict upper triangle receives L^t. Ak, Bk: K-major copies (n x ldk of the
// precision's element), eA: n ints.
cudaError_t launch_chol_mixed(int n, float* F, int ldf, int nb, int prec, void* Ak, void* Bk, int ldk,
                              int* eA, int* info, cudaStream_t s);
cudaError_t launch_mirror_lower(int n, float* F, int ldf, cudaStream_t s);

// ---- blocked LU driver (api.cu) ---------------------------------------------
struct LuWork {
  double* slots;        // panel exchange slots, panel_slots_doubles(), zeroed per factorisation
  // left_perm_ints(n, nb) ints: the interchanges left of each outer block are
  // applied once at the end (nullptr: block by block)
  int* left = nullptr;
  // mixed path only
  void* Ak;
  void* Bk;
  int* eA;
  int* eB;
  int ldk;
};
template <typename Ts>
cudaError_t blocked_lu(int n, Ts* A, int lda, int* ipiv, int* info, int nb, int prec,
                       const LuWork& w, cudaStream_t s);

}  // namespace gbla
