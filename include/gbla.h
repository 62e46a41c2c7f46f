/*
 * gbla -- dense LU / Cholesky solvers for one GB300 GPU (sm_103a), C ABI.
 *
 * The operations are those of the paper's direct method (Oancea & Andrei,
 * "Developing a High Performance Software Library with MPI and CUDA for Matrix
 * Computations", section 2): factor A = LU with partial pivoting (or A = L L^t
 * for SPD A), then solve L y = b and U x = y by forward and back substitution;
 * the factorisation is blocked by delayed updating (k rank-1 updates replaced
 * by one rank-k update). The mixed-precision variant factors in low precision
 * and recovers FP64 accuracy by GMRES (section 2: Gram-Schmidt, restarted)
 * used as the inner solver of iterative refinement.
 *
 * Conventions for every entry point
 *   - Matrices are column-major: element (i, j) of A is A[i + j*lda], 0-based,
 *     lda >= max(1, n). Pivots are LAPACK getrf style: 1-based, row j was
 *     interchanged with row ipiv[j] at step j, applied in order j = 0..n-1.
 *   - Every pointer is a DEVICE pointer owned by the caller unless stated
 *     otherwise. The library allocates no device memory: calls that need
 *     scratch take a caller-provided device workspace of at least the size
 *     the matching *_workspace function returns (256-byte aligned).
 *   - Every call is enqueued on `stream` (a cudaStream_t; NULL = the legacy
 *     default stream) and returns without waiting, except where stated.
 *   - Return value: 0 on success; -i when argument i (1-based) is invalid,
 *     nothing enqueued; a positive GBLA_ERR_* code otherwise.
 *   - Numerical outcome is written to a device int `d_info` (0 = success;
 *     k > 0 = the first exact zero pivot / non-positive leading minor at
 *     1-based k; GBLA_INFO_TIMEOUT when an inter-CTA wait gave up). The
 *     timeout code replaces only a zero.
 */
#ifndef GBLA_H
#define GBLA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *gbla_stream_t; /* same type as cudaStream_t */

#define GBLA_OK 0
#define GBLA_ERR_WORKSPACE 1001     /* workspace NULL, misaligned or too small */
#define GBLA_ERR_CUDA 1002          /* a CUDA runtime call (launch, copy, query) failed */
#define GBLA_ERR_DEVICE 1003        /* device lacks a needed capability (cooperative launch) */
#define GBLA_ERR_NOT_CONVERGED 1004 /* refinement stopped before reaching the tolerance */
#define GBLA_ERR_TIMEOUT 1005       /* host-visible: a device wait gave up (see d_info) */
#define GBLA_ERR_INTERNAL 1006

#define GBLA_INFO_TIMEOUT (-1000)

/* Precision of the trailing-matrix update of the mixed factorisation. */
#define GBLA_PREC_FP32 1 /* FP32 operands, FP32 FMA (SIMT) */
#define GBLA_PREC_TF32 2 /* TF32 operands (nearest, ties away), FP32 accumulate, tensor cores */
#define GBLA_PREC_BF16 3 /* BF16 operands with power-of-two row/column scaling, FP32 accumulate */
#define GBLA_PREC_FP16 4 /* FP16 operands with power-of-two row/column scaling, FP32 accumulate */
/* Split-operand variants: every scaled FP32 operand x is written as hi + lo
 * with hi = rn16(x), lo = rn16(x - hi), and the update accumulates
 * hi*hi + hi*lo + lo*hi in one FP32 tensor-memory accumulator (three times the
 * tensor-core work, close to FP32 accuracy for FP16). */
#define GBLA_PREC_FP16X3 5
#define GBLA_PREC_BF16X3 6

/* Library version string (static storage). */
const char *gbla_version(void);

/* Human-readable text for a return code (static storage). */
const char *gbla_status_string(int status);

/* Text of the last CUDA runtime failure seen by a gbla call on this host
 * thread (CUDA error name, failing call, message); "" if none. */
const char *gbla_last_error(void);

/*
 * Instrumentation (off by default; nothing here changes results).
 * gbla_launch_count: kernels this library has launched in this process.
 * gbla_prof_enable(mask): bracket every later launch group of the kinds set
 *   in mask (bit k = kind k) with a pair of CUDA events on its stream.
 *   Kinds: 0 panel, 1 laswp (an outer block's row interchanges on the
 *   columns outside it), 2 trsm, 3 gemm_simt, 4 gemm_tc, 5 convert,
 *   6 trsv, 7 matvec, 8 mgs, 9 gmres_update, 10 permute, 11 copy, 12 batched.
 * gbla_prof_read: number of recorded groups of `kind` and their summed
 *   device time in ms (waits for the events). gbla_prof_reset forgets them.
 * gbla_prof_list: the same groups one by one.
 */
uint64_t gbla_launch_count(void);
const char *gbla_kernel_kind_name(int kind);
void gbla_prof_enable(unsigned mask);
void gbla_prof_reset(void);
int gbla_prof_read(int kind, int *count, double *total_ms);
/* Device times (ms) of the first max_count recorded groups of `kind`, in
 * launch order; returns how many were written (or < 0 for a bad argument). */
int gbla_prof_list(int kind, int max_count, double *ms);

/*
 * Limit, in nanoseconds, for every inter-CTA wait of later calls (panel
 * barrier, substitution chain). A wait that runs out writes GBLA_INFO_TIMEOUT
 * to d_info and the kernel returns. Default 2e9 (2 s). Process-wide; not
 * thread-safe against concurrent calls.
 */
void gbla_set_wait_timeout_ns(uint64_t ns);
uint64_t gbla_get_wait_timeout_ns(void);

/*
 * Cap on the number of CTAs of the refinement's preconditioner substitution
 * (the inverted-diagonal-block forward and back solves inside
 * gbla_gmresir_solve*, gbla_chol_gmresir_solve_nrhs, gbla_gmres_solve and
 * gbla_bicgstab_solve). The substitution runs as a persistent grid of at most
 * one CTA per SM that draws its tasks in order; a cap leaves the other SMs
 * free for work on other streams (several systems solved concurrently). The
 * result does not depend on the cap. 0 (default): one CTA per SM.
 * Process-wide. Returns -1 for ctas < 0.
 */
int gbla_set_substitution_ctas(int ctas);
int gbla_get_substitution_ctas(void);

/*
 * Look-ahead in the blocked LU factorisations (gbla_lu_factor,
 * gbla_lu_factor_mixed, gbla_lu_factor_static; paper section 2, delayed
 * updating rescheduled): when on, each trailing update is split into the
 * next outer block's columns and the rest; the next block's panels are then
 * factored on a high-priority stream of the library's own while the rest of
 * the update runs on the caller's stream (the persistent tensor-core update
 * leaves the panel's 16 SMs free), and the caller's stream waits for them
 * before the next block's interchanges. The factors are bit-for-bit the same.
 * The streams and events are created on first use (one set per concurrent
 * call) and kept until the process exits. 0 (default): off. Process-wide.
 * Returns -1 for a value other than 0 or 1.
 */
int gbla_set_lookahead(int on);
int gbla_get_lookahead(void);

/*
 * Measured arithmetic rate of the device, for rooflines (the paper has no
 * counterpart: it quotes no peak). precision 0: FP64 fused multiply-add,
 * 1: FP32. Runs one untimed and one timed launch of independent FMA chains
 * filling every SM (`iters` steps of 8 chains per thread; 2 flops per FMA),
 * timed with CUDA events on `stream`, and writes the rate in TFLOP/s to
 * *tflops (host pointer). Synchronises with the stream. Returns -1 for a bad
 * precision, -2 for iters < 1, -3 for a null tflops, GBLA_ERR_CUDA on a
 * runtime failure.
 */
int gbla_fma_peak(int precision, int iters, double *tflops, gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * FP64 LU with partial pivoting (paper section 2; steps a1-a4).
 * Blocked right-looking: each block column of width nb is factored as
 * 32-column panels (warp-shuffle argmax pivot search, row swaps, scaling and
 * rank-1 updates on register-resident rows of one thread-block cluster, or of
 * cooperative CTAs for panels taller than a cluster holds), each followed by
 * the solve and update of the rest of the block column; then the block
 * column's row interchanges are applied to every other column, the U row
 * block is solved against the unit lower diagonal block and the trailing
 * matrix receives one rank-nb update. All work is ordered on `stream`.
 *   n      order of A (n >= 0)
 *   A      n x n, overwritten by L (strict lower, unit diagonal implied) and U
 *   lda    leading dimension (>= max(1, n))
 *   ipiv   n ints, output pivots (1-based)
 *   d_info one int, output (see conventions); set to 0 by the call
 *   nb     block size in [32, 256], multiple of 32; 0 = default (256)
 * ------------------------------------------------------------------------ */
size_t gbla_lu_factor_workspace(int n, int nb);
int gbla_lu_factor(int n, double *A, int lda, int *ipiv, int *d_info, int nb,
                   void *d_work, size_t work_bytes, gbla_stream_t stream);

/*
 * gbla_lu_factor without a workspace argument, for callers that cannot
 * allocate device memory (for example code running inside a memory pool or a
 * host application that owns every device allocation, or a path that must
 * never reach the allocator). The paper has no counterpart; it computes the
 * same factorisation, with the same kernels, as gbla_lu_factor.
 *   Its only scratch, the panel kernels' exchange slots, is a fixed array of
 *   about 290 KiB inside the library's device image (room for the 256 CTAs
 *   that the panel kernels use at most, on any device). Every GPU that loads
 *   the library holds that array until the process exits. The call itself
 *   allocates nothing: all of its work runs on `stream`.
 *   The first call on a device looks up the array's device address for that
 *   device (cudaGetSymbolAddress, with the device current) and keeps it; make
 *   that first call before any stream capture. The kept address belongs to
 *   the device's current context: after cudaDeviceReset the process must not
 *   call this entry point again.
 *   All calls share the one array and it keeps the last call's contents
 *   (each call clears it before use): calls whose work overlaps on the GPU --
 *   on different streams, or from different host threads -- race with each
 *   other and must be serialised by the caller.
 * Arguments and d_info as for gbla_lu_factor.
 */
int gbla_lu_factor_static(int n, double *A, int lda, int *ipiv, int *d_info, int nb,
                          gbla_stream_t stream);

/*
 * Solve op(A) X = B from the gbla_lu_factor output (paper section 2, steps
 * a5-a6): trans = 0: apply P, L y = Pb (unit, forward), U x = y (back);
 * trans = 1: A^t x = b via U^t z = b, L^t w = z, x = P^t w.
 * B (n x nrhs, ldb) is overwritten by X. Needs d_info (one int, set to 0;
 * receives GBLA_INFO_TIMEOUT if a chain wait gave up).
 */
size_t gbla_lu_solve_workspace(int n, int nrhs);
int gbla_lu_solve(int trans, int n, int nrhs, const double *LU, int lda, const int *ipiv,
                  double *B, int ldb, int *d_info, void *d_work, size_t work_bytes,
                  gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * FP64 Cholesky A = L L^t of an SPD matrix (paper section 2; steps a1, a3,
 * a4 for the SPD case). Lower triangle referenced and overwritten with L; the
 * strict upper triangle is neither read nor written. Blocked right-looking
 * with outer blocks of nb columns (nb in 64..256, a multiple of 64; 0 = 64),
 * each done in 64-column steps: diagonal block in shared memory, the block
 * column below it by substitution, the rest of the outer block by a rank-64
 * update; then the trailing lower triangle by one rank-nb update.
 * No scratch. d_info: 0, or k > 0 when the leading minor of order k is not
 * positive definite (the rest of the factor is then undefined).
 * ------------------------------------------------------------------------ */
int gbla_chol_factor(int n, double *A, int lda, int *d_info, int nb, gbla_stream_t stream);

/* Solve A X = B from gbla_chol_factor: L y = b (forward), L^t x = y (back).
 * B (n x nrhs, ldb) is overwritten by X. */
size_t gbla_chol_solve_workspace(int n, int nrhs);
int gbla_chol_solve(int n, int nrhs, const double *L, int lda, double *B, int ldb, int *d_info,
                    void *d_work, size_t work_bytes, gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * Mixed-precision LU (steps a1-a4 in low precision). F (n x n FP32, ldf) is
 * set to fp32(A) and factored in place: panels in FP64 arithmetic rounded to
 * FP32, the U row block by FP32 substitution, the trailing update in the
 * precision `prec` (GBLA_PREC_*): tensor-core (tcgen05, TMEM accumulator,
 * TMA-fed) for TF32 / BF16 / FP16 and the split variants, FP32 SIMT for FP32.
 * 16-bit operands carry one power-of-two scale per row of L21 and per column
 * of U12, undone exactly in the epilogue. A (FP64) is only read.
 * ------------------------------------------------------------------------ */
size_t gbla_lu_factor_mixed_workspace(int n, int nb, int prec);
int gbla_lu_factor_mixed(int n, const double *A, int lda, float *F, int ldf, int *ipiv,
                         int *d_info, int prec, int nb, void *d_work, size_t work_bytes,
                         gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * GMRES-based iterative refinement (steps a7-a8; the GMRES of paper section
 * 2 with Gram-Schmidt orthogonalisation and restarts): x0 = M^{-1} b with
 * M = P^t L U from gbla_lu_factor_mixed (FP32 factors, FP64 arithmetic);
 * then repeat r = b - A x (FP64), stop when
 * ||r||_inf / (||A||_inf ||x||_inf) <= tol; otherwise run restarted GMRES(m)
 * (modified Gram-Schmidt, Givens rotations) on M^{-1} A d = z, z = M^{-1} r,
 * from d = 0: up to `restarts` cycles of at most m steps, cycle c > 0
 * starting from the current d with the residual z - M^{-1} A d, until the
 * least-squares residual falls below inner_tol * ||z||_2; then
 * x <- x + d (FP64).
 * SYNCHRONOUS: reads one scalar back per inner step and per outer step
 * (it synchronises `stream`). Host pointers: opts, stats.
 * Returns 0 when converged, GBLA_ERR_NOT_CONVERGED otherwise (x holds the
 * last iterate), GBLA_ERR_TIMEOUT when a kernel wait gave up.
 * ------------------------------------------------------------------------ */
typedef struct {
  double tol;       /* normwise backward-error target, e.g. 1e-14 */
  double inner_tol; /* GMRES relative tolerance, e.g. 1e-8 */
  int max_outer;    /* refinement steps, e.g. 10 */
  int restart_m;    /* GMRES Krylov dimension per cycle, 1..128, e.g. 50 */
  int restarts;     /* GMRES cycles per refinement step (0 or 1: one cycle) */
} gbla_gmresir_opts;

typedef struct {
  int outer;      /* refinement steps taken */
  int inner;      /* GMRES steps in total */
  int converged;  /* 1 when beta <= tol */
  double beta;    /* final normwise backward error */
  double beta0;   /* backward error of x0 */
} gbla_gmresir_stats;

size_t gbla_gmresir_workspace(int n, int restart_m);
int gbla_gmresir_solve(int n, const double *A, int lda, const float *F, int ldf,
                       const int *ipiv, const double *b, double *x,
                       const gbla_gmresir_opts *opts, gbla_gmresir_stats *stats,
                       void *d_work, size_t work_bytes, gbla_stream_t stream);

/* The same refinement for nrhs right-hand sides (B, X: n x nrhs, ldb, ldx),
 * sharing one set-up of the factors (pivot permutation, inverted diagonal
 * blocks) and one workspace (gbla_gmresir_workspace(n, restart_m)); each
 * column is refined on its own, with its own entry of stats[0 .. nrhs).
 * Returns 0 when every column converged, GBLA_ERR_NOT_CONVERGED when one or
 * more did not (see stats[k].converged), GBLA_ERR_TIMEOUT on a wait that gave
 * up. Synchronous, like gbla_gmresir_solve. */
int gbla_gmresir_solve_nrhs(int n, int nrhs, const double *A, int lda, const float *F, int ldf,
                            const int *ipiv, const double *B, int ldb, double *X, int ldx,
                            const gbla_gmresir_opts *opts, gbla_gmresir_stats *stats,
                            void *d_work, size_t work_bytes, gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * Mixed-precision Cholesky + GMRES-IR for symmetric positive definite A
 * (paper section 2: A = L L^t; the same refinement as for the LU).
 * gbla_chol_factor_mixed: F (n x n FP32, ldf) <- fp32 of A's lower triangle
 *   (A is read on and below the diagonal only), factored in place by the
 *   blocked Cholesky of gbla_chol_factor in FP32 arithmetic with the trailing
 *   update in `prec` (GBLA_PREC_*; the tensor-core kinds update only the
 *   tiles on or below the diagonal, from one scaled copy of L21 per outer
 *   block); nb: outer block width, 64..256, a multiple of 64 (0 = 256). On
 *   return the lower triangle of F holds L and its strict upper triangle
 *   holds L^t (for the refinement's back substitution). d_info: 0 or k > 0
 *   when the leading minor of order k is not positive (in FP32 arithmetic).
 * gbla_chol_gmresir_solve_nrhs: gbla_gmresir_solve_nrhs with M = L L^t from
 *   those factors (no pivots). A must hold the whole symmetric matrix (the
 *   FP64 residual reads both triangles). Workspace: gbla_gmresir_workspace.
 * ------------------------------------------------------------------------ */
size_t gbla_chol_factor_mixed_workspace(int n, int nb, int prec);
int gbla_chol_factor_mixed(int n, const double *A, int lda, float *F, int ldf, int *d_info,
                           int prec, int nb, void *d_work, size_t work_bytes,
                           gbla_stream_t stream);
int gbla_chol_gmresir_solve_nrhs(int n, int nrhs, const double *A, int lda, const float *F,
                                 int ldf, const double *B, int ldb, double *X, int ldx,
                                 const gbla_gmresir_opts *opts, gbla_gmresir_stats *stats,
                                 void *d_work, size_t work_bytes, gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * Standalone Krylov solvers (paper section 2: the non-stationary iterative
 * methods -- GMRES with Gram-Schmidt orthogonalisation and restarts, and
 * BiCGSTAB -- next to the direct solvers), FP64 on a dense A (n x n, lda),
 * with an optional preconditioner M = P^t L U: the FP32 factors F (ldf) and
 * pivots ipiv of gbla_lu_factor_mixed (both NULL: none). x holds the initial
 * guess on entry and the iterate on return.
 * gbla_gmres_solve: restarted GMRES(restart_m), modified Gram-Schmidt,
 *   Givens rotations, left preconditioning; stops when the least-squares
 *   residual is <= tol * ||M^{-1} b||_2 (||b||_2 without M) or after max_iter
 *   Krylov steps.
 * gbla_bicgstab_solve: BiCGSTAB (van der Vorst's stabilised BiCG) with M
 *   applied to the search directions (p^ = M^{-1} p, s^ = M^{-1} s); all its
 *   scalars stay on the device; stops when ||r||_2 <= tol * ||b||_2 (the
 *   recursively updated r) or after max_iter iterations; a vanishing rho',
 *   (r~, v) or t with r not yet small is reported as a breakdown.
 * stats: iterations, converged, breakdown, relres = ||b - A x||_2 / ||b||_2
 * of the returned x (recomputed). SYNCHRONOUS: one scalar read per step.
 * Returns 0 when converged, GBLA_ERR_NOT_CONVERGED otherwise, GBLA_ERR_TIMEOUT
 * when a kernel wait gave up. Workspace: gbla_krylov_workspace(n, restart_m)
 * (restart_m is ignored by BiCGSTAB but sizes the shared layout).
 * ------------------------------------------------------------------------ */
typedef struct {
  double tol;     /* relative residual target */
  int max_iter;   /* Krylov steps (GMRES) or iterations (BiCGSTAB) */
  int restart_m;  /* GMRES restart length, 1..128 */
} gbla_krylov_opts;

typedef struct {
  int iterations;
  int converged;
  int breakdown;
  int pad;
  double relres;  /* ||b - A x||_2 / ||b||_2 of the returned x */
} gbla_krylov_stats;

size_t gbla_krylov_workspace(int n, int restart_m);
int gbla_gmres_solve(int n, const double *A, int lda, const double *b, double *x, const float *F,
                     int ldf, const int *ipiv, const gbla_krylov_opts *opts,
                     gbla_krylov_stats *stats, void *d_work, size_t work_bytes,
                     gbla_stream_t stream);
int gbla_bicgstab_solve(int n, const double *A, int lda, const double *b, double *x,
                        const float *F, int ldf, const int *ipiv, const gbla_krylov_opts *opts,
                        gbla_krylov_stats *stats, void *d_work, size_t work_bytes,
                        gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched LU with partial pivoting + solve (step a9: the factorisation and
 * the two substitutions of paper section 2 for every system of a batch), in
 * ONE persistent kernel launch: a grid of SMs x ctas_per_sm CTAs pulls system
 * indices from a counter (in d_order, or index order if d_order is NULL); one
 * CTA factors and solves one whole system, in shared memory when it fits, in
 * place in global memory otherwise. No host synchronisation and no
 * allocation: the call can be captured in a CUDA graph.
 * Device arrays of length batch: d_n (orders), d_A (column-major matrices,
 * overwritten by their L\U), d_lda, d_ipiv (n_i ints each, 1-based),
 * d_nrhs (0..4 right-hand sides each; NULL = factor only), d_B (n_i x nrhs_i,
 * overwritten by X), d_ldb, d_info (first zero pivot per system or 0; may be
 * NULL). max_n: an upper bound on the orders (sizes shared memory).
 * threads (multiple of 32, 0 = 256) and ctas_per_sm (0 = 1) are tuning knobs.
 * ------------------------------------------------------------------------ */
size_t gbla_lu_batched_workspace(int batch);
int gbla_lu_solve_batched(int batch, const int *d_n, double *const *d_A, const int *d_lda,
                          int *const *d_ipiv, const int *d_nrhs, double *const *d_B,
                          const int *d_ldb, int *d_info, const int *d_order, int max_n,
                          int threads, int ctas_per_sm, void *d_work, size_t work_bytes,
                          gbla_stream_t stream);
int gbla_lu_solve_batched_f32(int batch, const int *d_n, float *const *d_A, const int *d_lda,
                              int *const *d_ipiv, const int *d_nrhs, float *const *d_B,
                              const int *d_ldb, int *d_info, const int *d_order, int max_n,
                              int threads, int ctas_per_sm, void *d_work, size_t work_bytes,
                              gbla_stream_t stream);

/*
 * The batched LU split in two, so that the factors serve later right-hand
 * sides (the same persistent launch structure, no host synchronisation, no
 * allocation, graph-capturable; the same workspace, gbla_lu_batched_workspace):
 * gbla_lu_factor_batched[_f32]: factor only -- d_A overwritten by L\U, d_ipiv
 *   and d_info written, as by gbla_lu_solve_batched with d_nrhs = NULL.
 * gbla_lu_solve_factored_batched[_f32]: B <- U^{-1} L^{-1} P B for every
 *   system from the factors (d_LU) and pivots (d_ipiv) of a factor-only call,
 *   which are only read; d_nrhs (0..4 each) must be given. No info.
 */
int gbla_lu_factor_batched(int batch, const int *d_n, double *const *d_A, const int *d_lda,
                           int *const *d_ipiv, int *d_info, const int *d_order, int max_n,
                           int threads, int ctas_per_sm, void *d_work, size_t work_bytes,
                           gbla_stream_t stream);
int gbla_lu_factor_batched_f32(int batch, const int *d_n, float *const *d_A, const int *d_lda,
                               int *const *d_ipiv, int *d_info, const int *d_order, int max_n,
                               int threads, int ctas_per_sm, void *d_work, size_t work_bytes,
                               gbla_stream_t stream);
int gbla_lu_solve_factored_batched(int batch, const int *d_n, double *const *d_LU,
                                   const int *d_lda, int *const *d_ipiv, const int *d_nrhs,
                                   double *const *d_B, const int *d_ldb, const int *d_order,
                                   int max_n, int threads, int ctas_per_sm, void *d_work,
                                   size_t work_bytes, gbla_stream_t stream);
int gbla_lu_solve_factored_batched_f32(int batch, const int *d_n, float *const *d_LU,
                                       const int *d_lda, int *const *d_ipiv, const int *d_nrhs,
                                       float *const *d_B, const int *d_ldb, const int *d_order,
                                       int max_n, int threads, int ctas_per_sm, void *d_work,
                                       size_t work_bytes, gbla_stream_t stream);

/* ------------------------------------------------------------------------
 * Batched Cholesky + solve (step a9 for symmetric positive definite systems:
 * A = L L^t and the two substitutions of paper section 2, for every system of
 * a batch) in ONE persistent kernel launch, with the launch structure of
 * gbla_lu_solve_batched (same counter-driven grid, same shared-memory /
 * in-place split, no host synchronisation, no allocation, graph-capturable).
 * Only the lower triangle of each A is read and overwritten by L; the strict
 * upper triangle is untouched. d_info[i] = j + 1 when the j-th leading minor
 * of system i is not positive (its factorisation stops there and its
 * right-hand sides are left unchanged), else 0. d_nrhs may be NULL (factor
 * only); at most 4 right-hand sides per system. Workspace:
 * gbla_chol_batched_workspace(batch) bytes, 256-byte aligned.
 * Returns -i for an invalid i-th argument, GBLA_ERR_WORKSPACE, GBLA_ERR_CUDA.
 * ------------------------------------------------------------------------ */
size_t gbla_chol_batched_workspace(int batch);
int gbla_chol_solve_batched(int batch, const int *d_n, double *const *d_A, const int *d_lda,
                            const int *d_nrhs, double *const *d_B, const int *d_ldb, int *d_info,
                            const int *d_order, int max_n, int threads, int ctas_per_sm,
                            void *d_work, size_t work_bytes, gbla_stream_t stream);
int gbla_chol_solve_batched_f32(int batch, const int *d_n, float *const *d_A, const int *d_lda,
                                const int *d_nrhs, float *const *d_B, const int *d_ldb, int *d_info,
                                const int *d_order, int max_n, int threads, int ctas_per_sm,
                                void *d_work, size_t work_bytes, gbla_stream_t stream);

/* The batched Cholesky split in two (as the LU above; workspace
 * gbla_chol_batched_workspace): gbla_chol_factor_batched[_f32] factors only
 * (lower triangles overwritten by L, d_info written);
 * gbla_chol_solve_factored_batched[_f32] solves L y = b, L^t x = y for every
 * system from those factors (only read), d_nrhs given, no info. */
int gbla_chol_factor_batched(int batch, const int *d_n, double *const *d_A, const int *d_lda,
                             int *d_info, const int *d_order, int max_n, int threads,
                             int ctas_per_sm, void *d_work, size_t work_bytes,
                             gbla_stream_t stream);
int gbla_chol_factor_batched_f32(int batch, const int *d_n, float *const *d_A, const int *d_lda,
                                 int *d_info, const int *d_order, int max_n, int threads,
                                 int ctas_per_sm, void *d_work, size_t work_bytes,
                                 gbla_stream_t stream);
int gbla_chol_solve_factored_batched(int batch, const int *d_n, double *const *d_L,
                                     const int *d_lda, const int *d_nrhs, double *const *d_B,
                                     const int *d_ldb, const int *d_order, int max_n, int threads,
                                     int ctas_per_sm, void *d_work, size_t work_bytes,
                                     gbla_stream_t stream);
int gbla_chol_solve_factored_batched_f32(int batch, const int *d_n, float *const *d_L,
                                         const int *d_lda, const int *d_nrhs, float *const *d_B,
                                         const int *d_ldb, const int *d_order, int max_n,
                                         int threads, int ctas_per_sm, void *d_work,
                                         size_t work_bytes, gbla_stream_t stream);

/*
 * Rank-k product C = alpha * U V^t + beta * C (FP64; U m x k, V n x k, C m x n;
 * beta = 0 overwrites C without reading it). With alpha = -1, beta = 0,
 * U = gb = A^{-t} g and V = x it forms the gradient of x = A^{-1} b with
 * respect to A, gA = -gb x^t (step a10; the paper has no gradient -- this is
 * the differentiation the solve is extended with).
 */
int gbla_rank_k_update(int m, int n, int k, double alpha, const double *U, int ldu,
                       const double *V, int ldv, double beta, double *C, int ldc,
                       gbla_stream_t stream);

/*
 * Normwise backward error per column (step a7): d_beta[c] =
 * ||B(:,c) - A X(:,c)||_inf / (||A||_inf ||X(:,c)||_inf), FP64, on the device.
 */
size_t gbla_backward_error_workspace(int n, int nrhs);
int gbla_backward_error(int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                        const double *B, int ldb, double *d_beta, void *d_work,
                        size_t work_bytes, gbla_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* GBLA_H */
