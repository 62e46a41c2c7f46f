// C ABI of libgbla: argument checks, workspace carving and the host-side
// schedule of the blocked factorisations (paper section 2: factor, then the two
// triangular solves; blocked by delayed updating) and of the GMRES-based
// refinement. Every numerical step runs in the kernels of this library.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace gbla {

static uint64_t g_wait_ns = 2000000000ull;
uint64_t wait_timeout_ns() { return g_wait_ns; }
static std::atomic<int> g_subst_ctas{0};
int substitution_ctas() { return g_subst_ctas.load(std::memory_order_relaxed); }
static std::atomic<int> g_lookahead{0};
bool lookahead_enabled() { return g_lookahead.load(std::memory_order_relaxed) != 0; }
constexpr int kClusterSms = 16;  // SMs of the panel's thread-block cluster

const DeviceProps& device_props() {
  static DeviceProps props[64];
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    static DeviceProps none;
    return none;
  }
  DeviceProps& p = props[dev];
  if (p.device < 0) {
    int sms = 0, coop = 0, optin = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    p.num_sms = sms;
    p.coop = coop;
    p.smem_optin = (size_t)optin;
    p.device = dev;
  }
  return p;
}

cudaError_t ensure_dyn_smem_ptr(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> granted;
  if (bytes <= 48 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> lock(mu);
  auto it = granted.find(func);
  if (it != granted.end() && bytes <= it->second) return cudaSuccess;
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  const size_t optin = device_props().smem_optin;
  const size_t cap = optin > fa.sharedSizeBytes ? optin - fa.sharedSizeBytes : 0;
  if (bytes > cap) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap);
  if (e == cudaSuccess) granted[func] = cap;
  return e;
}

// ---- instrumentation ---------------------------------------------------------
static std::atomic<uint64_t> g_launches{0};
void count_launch(int k) { g_launches.fetch_add((uint64_t)k, std::memory_order_relaxed); }

struct ProfRec {
  int kind;
  cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static unsigned g_prof_mask = 0;
static std::vector<ProfRec> g_prof_recs;   // recorded pairs, in order
static std::vector<cudaEvent_t> g_prof_pool;
// the open record of the calling thread (calls on several host threads
// interleave), valid while no reset has happened since it was opened
static thread_local size_t g_prof_open = (size_t)-1;
static thread_local uint64_t g_prof_open_gen = 0;
static uint64_t g_prof_gen = 1;

static cudaEvent_t prof_event() {
  if (!g_prof_pool.empty()) {
    cudaEvent_t e = g_prof_pool.back();
    g_prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void prof_begin(int kind, cudaStream_t s) {
  if (!(g_prof_mask & (1u << kind))) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  ProfRec r{kind, prof_event(), prof_event()};
  cudaEventRecord(r.a, s);
  g_prof_recs.push_back(r);
  g_prof_open = g_prof_recs.size() - 1;
  g_prof_open_gen = g_prof_gen;
}

void prof_end(int kind, cudaStream_t s) {
  if (!(g_prof_mask & (1u << kind))) return;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  if (g_prof_open_gen == g_prof_gen && g_prof_open < g_prof_recs.size() &&
      g_prof_recs[g_prof_open].kind == kind)
    cudaEventRecord(g_prof_recs[g_prof_open].b, s);
  g_prof_open = (size_t)-1;
}

#define PROF(kind, stream, call)   \
  do {                             \
    prof_begin((kind), (stream));  \
    e = (call);                    \
    prof_end((kind), (stream));    \
  } while (0)

static thread_local char g_last_error[256] = "";

static void clear_error() { g_last_error[0] = 0; }
void api_clear_error() { clear_error(); }

static void record_error_in(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_error, sizeof(g_last_error), "%s (%s) at %s:%d: %s", cudaGetErrorName(e), what,
           file, line, cudaGetErrorString(e));
}
static void record_error(cudaError_t e, const char* what, int line) {
  record_error_in(e, what, "api.cu", line);
}

// the first failure of a call is kept; the outer wrappers do not overwrite it
int api_cuda_status(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return GBLA_OK;
  if (g_last_error[0] == 0) record_error_in(e, what, file, line);
  return GBLA_ERR_CUDA;
}
#define cuda_status(e) api_cuda_status((e), #e, "api.cu", __LINE__)

#define GBLA_TRYK(kind, stream, expr)      \
  do {                                     \
    prof_begin((kind), (stream));          \
    cudaError_t _e = (expr);               \
    prof_end((kind), (stream));            \
    if (_e != cudaSuccess) {               \
      record_error(_e, #expr, __LINE__);   \
      return GBLA_ERR_CUDA;                \
    }                                      \
  } while (0)

#define GBLA_TRY(expr)                                   \
  do {                                                   \
    cudaError_t _e = (expr);                             \
    if (_e != cudaSuccess) {                             \
      record_error(_e, #expr, __LINE__);                 \
      return GBLA_ERR_CUDA;                              \
    }                                                    \
  } while (0)

static bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255) == 0; }

// Look-ahead resources: a high-priority stream and two events, taken from a
// process-wide pool for the duration of one factorisation (several host
// threads may factor at once, each with its own set).
struct LookAhead {
  int device = -1;
  cudaStream_t hp = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static std::mutex g_la_mu;
static std::vector<LookAhead> g_la_pool;

static cudaError_t lookahead_acquire(LookAhead* out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lock(g_la_mu);
    for (size_t i = 0; i < g_la_pool.size(); ++i)
      if (g_la_pool[i].device == dev) {
        *out = g_la_pool[i];
        g_la_pool.erase(g_la_pool.begin() + (long)i);
        return cudaSuccess;
      }
  }
  LookAhead r;
  r.device = dev;
  int lo = 0, hi = 0;
  if ((e = cudaDeviceGetStreamPriorityRange(&lo, &hi)) != cudaSuccess) return e;
  if ((e = cudaStreamCreateWithPriority(&r.hp, cudaStreamNonBlocking, hi)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming)) != cudaSuccess) return e;
  if ((e = cudaEventCreateWithFlags(&r.join, cudaEventDisableTiming)) != cudaSuccess) return e;
  *out = r;
  return cudaSuccess;
}
static void lookahead_release(const LookAhead& r) {
  std::lock_guard<std::mutex> lock(g_la_mu);
  g_la_pool.push_back(r);
}

// ----------------------------------------------------------------------------
// Blocked right-looking LU over a generic storage type. Outer blocks of width
// nb; inside each, inner panels of width kPanelWidth factored by the panel
// kernel (which also applies the panel's row interchanges to the other
// columns of the outer block), followed by the inner substitution and update
// restricted to the outer block (one fused launch). After the outer block:
// its interchanges on every other column (one launch), the U row block and
// the trailing update.
//
// Look-ahead (when enabled): the trailing update is split into the next
// outer block's columns and the rest. Once the first part is done, the next
// block's panels are factored on a high-priority stream while the rest of the
// update runs on the caller's stream on all SMs but 16 (the panel's cluster);
// the caller's stream then waits for the panels. Every element receives the
// same operations in the same order as without look-ahead.
static size_t lu_work_layout(Carver& c, int n, int nb, int prec, LuWork* w) {
  double* slots = c.take<double>(panel_slots_doubles());
  const size_t li = left_perm_ints(n, nb);
  int* left = li ? c.take<int>(li) : nullptr;
  if (w) {
    w->slots = slots;
    w->left = left;
    w->Ak = w->Bk = nullptr;
    w->eA = w->eB = nullptr;
    w->ldk = 0;
  }
  if (prec_is_tensor(prec)) {
    const int elem = prec == GBLA_PREC_TF32 ? 4 : 2;
    const int ldk = ((prec_kmult(prec) * nb + 63) / 64) * 64;
    void* Ak = c.take<char>((size_t)std::max(n, 1) * ldk * elem);
    void* Bk = c.take<char>((size_t)std::max(n, 1) * ldk * elem);
    int* eA = c.take<int>((size_t)std::max(n, 1));
    int* eB = c.take<int>((size_t)std::max(n, 1));
    if (w) {
      w->Ak = Ak;
      w->Bk = Bk;
      w->eA = eA;
      w->eB = eB;
      w->ldk = ldk;
    }
  }
  return c.off;
}

template <typename Ts>
cudaError_t blocked_lu(int n, Ts* A, int lda, int* ipiv, int* info, int nb, int prec,
                              const LuWork& w, cudaStream_t s) {
  typedef Ts Tc_trsm;  // substitution arithmetic: FP64 for FP64 storage, FP32 for FP32
  unsigned* inner_ctr = reinterpret_cast<unsigned*>(w.slots + kPanelExchangeDoubles);
  // the columns left of each block get its interchanges at the end when possible
  const bool defer_left = w.left != nullptr && left_deferred_fits<Ts>(n, nb);
  const bool tensor = prec_is_tensor(prec);
  cudaError_t e;
  // the panels of outer block [k0, k0 + kb) and the inner updates, on stream st
  auto panels = [&](int k0, int kb, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    for (int j0 = k0; j0 < k0 + kb; j0 += kPanelWidth) {
      const int jb = std::min(kPanelWidth, k0 + kb - j0);
      // the panel launch also applies its interchanges to the rest of the outer block
      PROF(KK_PANEL, st, launch_panel<Ts>(A + j0 + (size_t)j0 * lda, lda, n - j0, jb, j0, ipiv + j0, info,
                                          w.slots, (unsigned)(j0 / kPanelWidth), j0 - k0,
                                          k0 + kb - j0 - jb, st));
      if (e != cudaSuccess) return e;
      const int nrest = k0 + kb - j0 - jb;
      if (nrest > 0 && jb == kPanelWidth) {
        // U12 of the panel and the update of the rest of the outer block, one launch
        PROF(KK_GEMM_SIMT, st, launch_inner_update<Ts>(n - j0 - jb, nrest, A + j0 + (size_t)j0 * lda, lda,
                                                       inner_ctr, st));
        if (e != cudaSuccess) return e;
      } else if (nrest > 0) {
        PROF(KK_TRSM, st, (launch_trsm_lunit<Ts, Tc_trsm>(A + j0 + (size_t)j0 * lda, lda,
                                            A + j0 + (size_t)(j0 + jb) * lda, lda, jb, nrest, 0,
                                            nullptr, 0, nullptr, st)));
        if (e != cudaSuccess) return e;
        PROF(KK_GEMM_SIMT, st, launch_gemm_simt<Ts>(n - j0 - jb, nrest, jb, (Ts)-1, A + (j0 + jb) + (size_t)j0 * lda,
                                  lda, A + j0 + (size_t)(j0 + jb) * lda, lda, false, (Ts)1,
                                  A + (j0 + jb) + (size_t)(j0 + jb) * lda, lda, false, st));
        if (e != cudaSuccess) return e;
      }
    }
    return cudaSuccess;
  };
  // trailing update of block [k0, k0 + kb) restricted to the columns
  // [k0 + kb + c0, k0 + kb + c0 + nc) (all nt rows below the block)
  auto update = [&](int k0, int kb, int c0, int nc, int grid_cap, cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    const int nt = n - k0 - kb;
    if (tensor) {
      if constexpr (sizeof(Ts) == 4) {
        const size_t eb = prec == GBLA_PREC_TF32 ? 4 : 2;
        const void* Bk = static_cast<const char*>(w.Bk) + (size_t)c0 * w.ldk * eb;
        PROF(KK_GEMM_TC, st, launch_gemm_tc(prec_mma_kind(prec), nt, nc, prec_kmult(prec) * kb, w.Ak, w.ldk, Bk,
                                            w.ldk, w.eA, w.eB + c0,
                                            reinterpret_cast<float*>(A + (k0 + kb) + (size_t)(k0 + kb + c0) * lda),
                                            lda, info, false, st, grid_cap));
        return e;
      } else {
        return cudaErrorInvalidValue;
      }
    }
    PROF(KK_GEMM_SIMT, st, launch_gemm_simt<Ts>(nt, nc, kb, (Ts)-1, A + (k0 + kb) + (size_t)k0 * lda, lda,
                                                A + k0 + (size_t)(k0 + kb + c0) * lda, lda, false, (Ts)1,
                                                A + (k0 + kb) + (size_t)(k0 + kb + c0) * lda, lda, false, st));
    return e;
  };
  const DeviceProps& dp = device_props();
  const bool la_on = lookahead_enabled() && n > 2 * nb && dp.num_sms > 32;
  LookAhead la;
  if (la_on) {
    e = lookahead_acquire(&la);
    if (e != cudaSuccess) { record_error(e, "look-ahead resources", __LINE__); return e; }
  }
  cudaError_t status = cudaSuccess;
  bool have_panels = false;  // the current block's panels were done during the previous update
  for (int k0 = 0; k0 < n && status == cudaSuccess; k0 += nb) {
    const int kb = std::min(nb, n - k0);
    if (!have_panels) {
      e = panels(k0, kb, s);
      if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); status = e; break; }
    }
    have_panels = false;
    // the block's interchanges on the columns right of it (the U row block
    // and the trailing update below read the interchanged rows) and, unless
    // deferred, on the columns left of it
    PROF(KK_LASWP, s, launch_laswp_block<Ts>(A, lda, n, n, k0, kb, ipiv + k0, defer_left ? 0 : k0,
                                             k0 + kb, s));
    if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); status = e; break; }
    const int nt = n - k0 - kb;
    if (nt <= 0) continue;
    PROF(KK_TRSM, s, (launch_trsm_lunit<Ts, Tc_trsm>(A + k0 + (size_t)k0 * lda, lda, A + k0 + (size_t)(k0 + kb) * lda,
                                       lda, kb, nt, tensor ? prec : 0, w.Bk, w.ldk, w.eB, s)));
    if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); status = e; break; }
    if (tensor) {
      if constexpr (sizeof(Ts) == 4) {
        PROF(KK_CONVERT, s, launch_convert_rows(reinterpret_cast<const float*>(A + (k0 + kb) + (size_t)k0 * lda), lda,
                                nt, kb, prec, w.Ak, w.ldk, w.eA, false, s));
        if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); status = e; break; }
      }
    }
    const int nb_next = std::min(nb, nt);
    if (la_on && nt > nb_next) {
      // the next block's columns first, then its panels on the high-priority
      // stream while the rest of the update runs here
      e = update(k0, kb, 0, nb_next, 0, s);
      if (e == cudaSuccess) e = cudaEventRecord(la.fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(la.hp, la.fork, 0);
      if (e == cudaSuccess) e = panels(k0 + kb, nb_next, la.hp);
      if (e == cudaSuccess) e = cudaEventRecord(la.join, la.hp);
      if (e == cudaSuccess) e = update(k0, kb, nb_next, nt - nb_next, dp.num_sms - kClusterSms, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, la.join, 0);
      if (e != cudaSuccess) { record_error(e, "blocked_lu look-ahead", __LINE__); status = e; break; }
      have_panels = true;
    } else {
      e = update(k0, kb, 0, nt, 0, s);
      if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); status = e; break; }
    }
  }
  if (la_on) lookahead_release(la);
  if (status != cudaSuccess) return status;
  if (defer_left) {
    PROF(KK_LASWP, s, launch_left_interchanges<Ts>(A, lda, n, nb, ipiv, w.left, s));
    if (e != cudaSuccess) { record_error(e, "blocked_lu step", __LINE__); return e; }
  }
  return cudaSuccess;
}

template cudaError_t blocked_lu<double>(int, double*, int, int*, int*, int, int, const LuWork&,
                                        cudaStream_t);
template cudaError_t blocked_lu<float>(int, float*, int, int*, int*, int, int, const LuWork&,
                                       cudaStream_t);

static int check_nb(int nb) { return nb == 0 ? 256 : ((nb % 32 == 0 && nb >= 32 && nb <= 256) ? nb : -1); }

}  // namespace gbla

using namespace gbla;

extern "C" {

const char* gbla_version(void) { return "gbla 0.1.0 (sm_103a)"; }

const char* gbla_status_string(int status) {
  switch (status) {
    case GBLA_OK: return "success";
    case GBLA_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case GBLA_ERR_CUDA: return "CUDA runtime call failed";
    case GBLA_ERR_DEVICE: return "device lacks a required capability";
    case GBLA_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
    case GBLA_ERR_TIMEOUT: return "a device-side wait gave up";
    case GBLA_ERR_INTERNAL: return "internal error";
    default: return status < 0 ? "invalid argument" : "unknown status";
  }
}

const char* gbla_last_error(void) { return g_last_error; }

uint64_t gbla_launch_count(void) { return g_launches.load(); }

static const char* kKindNames[KK_COUNT] = {"panel", "laswp",  "trsm", "gemm_simt",    "gemm_tc", "convert",
                                           "trsv",  "matvec", "mgs",  "gmres_update", "permute", "copy",
                                           "batched"};

const char* gbla_kernel_kind_name(int kind) {
  return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "";
}

void gbla_prof_enable(unsigned mask) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  g_prof_mask = mask;
}

void gbla_prof_reset(void) {
  std::lock_guard<std::mutex> lock(g_prof_mu);
  for (auto& r : g_prof_recs) {
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  ++g_prof_gen;
  g_prof_open = (size_t)-1;
}

int gbla_prof_read(int kind, int* count, double* total_ms) {
  if (kind < 0 || kind >= KK_COUNT) return -1;
  if (!count) return -2;
  if (!total_ms) return -3;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  int c = 0;
  double t = 0.0;
  for (auto& r : g_prof_recs) {
    if (r.kind != kind) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return GBLA_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return GBLA_ERR_CUDA;
    ++c;
    t += ms;
  }
  *count = c;
  *total_ms = t;
  return GBLA_OK;
}

int gbla_prof_list(int kind, int max_count, double* ms) {
  if (kind < 0 || kind >= KK_COUNT) return -1;
  if (max_count < 0) return -2;
  if (max_count > 0 && !ms) return -3;
  std::lock_guard<std::mutex> lock(g_prof_mu);
  int c = 0;
  for (auto& r : g_prof_recs) {
    if (r.kind != kind) continue;
    if (c >= max_count) break;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return GBLA_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return GBLA_ERR_CUDA;
    ms[c++] = t;
  }
  return c;
}

void gbla_set_wait_timeout_ns(uint64_t ns) { g_wait_ns = ns; }
int gbla_set_substitution_ctas(int ctas) {
  if (ctas < 0) return -1;
  g_subst_ctas.store(ctas, std::memory_order_relaxed);
  return GBLA_OK;
}
int gbla_get_substitution_ctas(void) { return substitution_ctas(); }
int gbla_set_lookahead(int on) {
  if (on != 0 && on != 1) return -1;
  g_lookahead.store(on, std::memory_order_relaxed);
  return GBLA_OK;
}
int gbla_get_lookahead(void) { return g_lookahead.load(std::memory_order_relaxed); }
uint64_t gbla_get_wait_timeout_ns(void) { return g_wait_ns; }

// ---------------------------------------------------------------------------
size_t gbla_lu_factor_workspace(int n, int nb) {
  nb = check_nb(nb);
  if (n < 0 || nb < 0) return 0;
  Carver c(nullptr, 0);
  return lu_work_layout(c, n, nb, 0, nullptr);
}

int gbla_lu_factor(int n, double* A, int lda, int* ipiv, int* d_info, int nb, void* d_work,
                   size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !ipiv) return -4;
  if (!d_info) return -5;
  nb = check_nb(nb);
  if (nb < 0) return -6;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  LuWork w;
  lu_work_layout(c, n, nb, 0, &w);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return GBLA_ERR_CUDA;
  if (!dp.coop) return GBLA_ERR_DEVICE;
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0) return GBLA_OK;
  GBLA_TRY(cudaMemsetAsync(w.slots, 0, sizeof(double) * panel_slots_doubles(), s));
  return cuda_status(blocked_lu<double>(n, A, lda, ipiv, d_info, nb, 0, w, s));
}

// ---------------------------------------------------------------------------
size_t gbla_lu_factor_mixed_workspace(int n, int nb, int prec) {
  nb = check_nb(nb);
  if (n < 0 || nb < 0 || prec < GBLA_PREC_FP32 || prec > GBLA_PREC_BF16X3) return 0;
  Carver c(nullptr, 0);
  return lu_work_layout(c, n, nb, prec, nullptr);
}

int gbla_lu_factor_mixed(int n, const double* A, int lda, float* F, int ldf, int* ipiv, int* d_info,
                         int prec, int nb, void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !F) return -4;
  if (ldf < std::max(1, n)) return -5;
  if (n > 0 && !ipiv) return -6;
  if (!d_info) return -7;
  if (prec < GBLA_PREC_FP32 || prec > GBLA_PREC_BF16X3) return -8;
  nb = check_nb(nb);
  if (nb < 0) return -9;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  LuWork w;
  lu_work_layout(c, n, nb, prec, &w);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return GBLA_ERR_CUDA;
  if (!dp.coop) return GBLA_ERR_DEVICE;
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0) return GBLA_OK;
  GBLA_TRY(cudaMemsetAsync(w.slots, 0, sizeof(double) * panel_slots_doubles(), s));
  GBLA_TRYK(KK_COPY, s, launch_copy_d2f(A, lda, F, ldf, n, n, s));
  return cuda_status(blocked_lu<float>(n, F, ldf, ipiv, d_info, nb, prec, w, s));
}

// ---------------------------------------------------------------------------
size_t gbla_lu_solve_workspace(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  Carver c(nullptr, 0);
  c.take<int>((size_t)std::max(n, 1));
  c.take<double>((size_t)std::max(n, 1) * std::max(nrhs, 1));
  c.take<unsigned>(trsv_flags_count(std::max(n, 1), std::max(nrhs, 1)));
  return c.off;
}

int gbla_lu_solve(int trans, int n, int nrhs, const double* LU, int lda, const int* ipiv, double* B,
                  int ldb, int* d_info, void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  if (trans != 0 && trans != 1) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (n > 0 && !LU) return -4;
  if (lda < std::max(1, n)) return -5;
  if (n > 0 && !ipiv) return -6;
  if (n > 0 && nrhs > 0 && !B) return -7;
  if (ldb < std::max(1, n)) return -8;
  if (!d_info) return -9;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  int* perm = c.take<int>((size_t)std::max(n, 1));
  double* T = c.take<double>((size_t)std::max(n, 1) * std::max(nrhs, 1));
  unsigned* flags = c.take<unsigned>(trsv_flags_count(std::max(n, 1), std::max(nrhs, 1)));
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0 || nrhs == 0) return GBLA_OK;
  GBLA_TRYK(KK_PERM, s, launch_ipiv_to_perm(n, ipiv, perm, s));
  const int ldt = n;
  if (!trans) {
    GBLA_TRYK(KK_PERM, s, launch_permute_rows(n, nrhs, perm, false, B, ldb, T, ldt, s));
    GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(true, false, true, n, nrhs, LU, lda, T, ldt, flags, d_info, s));
    GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(false, false, false, n, nrhs, LU, lda, T, ldt, flags, d_info, s));
    GBLA_TRY(cudaMemcpy2DAsync(B, sizeof(double) * ldb, T, sizeof(double) * ldt, sizeof(double) * n,
                               nrhs, cudaMemcpyDeviceToDevice, s));
  } else {
    GBLA_TRY(cudaMemcpy2DAsync(T, sizeof(double) * ldt, B, sizeof(double) * ldb, sizeof(double) * n,
                               nrhs, cudaMemcpyDeviceToDevice, s));
    GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(false, true, false, n, nrhs, LU, lda, T, ldt, flags, d_info, s));
    GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(true, true, true, n, nrhs, LU, lda, T, ldt, flags, d_info, s));
    GBLA_TRYK(KK_PERM, s, launch_permute_rows(n, nrhs, perm, true, T, ldt, B, ldb, s));
  }
  return GBLA_OK;
}

// ---------------------------------------------------------------------------
int gbla_chol_factor(int n, double* A, int lda, int* d_info, int nb, gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (!d_info) return -4;
  if (nb != 0 && (nb % 64 != 0 || nb < 64 || nb > 256)) return -5;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0) return GBLA_OK;
  return cuda_status(launch_chol(n, A, lda, nb, d_info, s));
}

size_t gbla_chol_solve_workspace(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  Carver c(nullptr, 0);
  c.take<unsigned>(trsv_flags_count(std::max(n, 1), std::max(nrhs, 1)));
  return c.off;
}

int gbla_chol_solve(int n, int nrhs, const double* L, int lda, double* B, int ldb, int* d_info,
                    void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !L) return -3;
  if (lda < std::max(1, n)) return -4;
  if (n > 0 && nrhs > 0 && !B) return -5;
  if (ldb < std::max(1, n)) return -6;
  if (!d_info) return -7;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  unsigned* flags = c.take<unsigned>(trsv_flags_count(std::max(n, 1), std::max(nrhs, 1)));
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0 || nrhs == 0) return GBLA_OK;
  GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(true, false, false, n, nrhs, L, lda, B, ldb, flags, d_info, s));
  GBLA_TRYK(KK_TRSV, s, launch_trsv<double>(true, true, false, n, nrhs, L, lda, B, ldb, flags, d_info, s));
  return GBLA_OK;
}

// ---------------------------------------------------------------------------
size_t gbla_lu_batched_workspace(int batch) {
  if (batch < 0) return 0;
  Carver c(nullptr, 0);
  c.take<unsigned>(1);
  return c.off;
}

}  // extern "C"

template <typename T>
static int lu_batched_entry(int batch, const int* d_n, T* const* d_A, const int* d_lda,
                            int* const* d_ipiv, const int* d_nrhs, T* const* d_B, const int* d_ldb,
                            int* d_info, const int* d_order, int max_n, int threads, int ctas_per_sm,
                            void* d_work, size_t work_bytes, gbla_stream_t stream, bool solve_only) {
  clear_error();
  if (batch < 0) return -1;
  if (batch > 0 && !d_n) return -2;
  if (batch > 0 && !d_A) return -3;
  if (batch > 0 && !d_lda) return -4;
  if (batch > 0 && !d_ipiv) return -5;
  if (d_nrhs && (!d_B || !d_ldb)) return -7;
  if (solve_only && batch > 0 && !d_nrhs) return -6;
  if (max_n < 0) return -11;
  if (threads != 0 && (threads % 32 != 0 || threads < 32 || threads > 1024)) return -12;
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return -13;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  unsigned* counter = c.take<unsigned>(1);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  if (batch == 0) return GBLA_OK;
  GBLA_TRYK(KK_BATCHED, s, launch_lu_batched<T>(batch, d_n, d_A, d_lda, d_ipiv, d_nrhs, d_B, d_ldb, d_info,
                                              d_order, max_n, threads, ctas_per_sm, counter, solve_only, s));
  return GBLA_OK;
}

extern "C" {

int gbla_lu_solve_batched(int batch, const int* d_n, double* const* d_A, const int* d_lda,
                          int* const* d_ipiv, const int* d_nrhs, double* const* d_B, const int* d_ldb,
                          int* d_info, const int* d_order, int max_n, int threads, int ctas_per_sm,
                          void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return lu_batched_entry<double>(batch, d_n, d_A, d_lda, d_ipiv, d_nrhs, d_B, d_ldb, d_info, d_order,
                                  max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_lu_solve_batched_f32(int batch, const int* d_n, float* const* d_A, const int* d_lda,
                              int* const* d_ipiv, const int* d_nrhs, float* const* d_B,
                              const int* d_ldb, int* d_info, const int* d_order, int max_n, int threads,
                              int ctas_per_sm, void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return lu_batched_entry<float>(batch, d_n, d_A, d_lda, d_ipiv, d_nrhs, d_B, d_ldb, d_info, d_order,
                                 max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_lu_factor_batched(int batch, const int* d_n, double* const* d_A, const int* d_lda,
                           int* const* d_ipiv, int* d_info, const int* d_order, int max_n, int threads,
                           int ctas_per_sm, void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return lu_batched_entry<double>(batch, d_n, d_A, d_lda, d_ipiv, nullptr, nullptr, nullptr, d_info,
                                  d_order, max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_lu_factor_batched_f32(int batch, const int* d_n, float* const* d_A, const int* d_lda,
                               int* const* d_ipiv, int* d_info, const int* d_order, int max_n,
                               int threads, int ctas_per_sm, void* d_work, size_t work_bytes,
                               gbla_stream_t stream) {
  return lu_batched_entry<float>(batch, d_n, d_A, d_lda, d_ipiv, nullptr, nullptr, nullptr, d_info,
                                 d_order, max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_lu_solve_factored_batched(int batch, const int* d_n, double* const* d_LU, const int* d_lda,
                                   int* const* d_ipiv, const int* d_nrhs, double* const* d_B,
                                   const int* d_ldb, const int* d_order, int max_n, int threads,
                                   int ctas_per_sm, void* d_work, size_t work_bytes,
                                   gbla_stream_t stream) {
  return lu_batched_entry<double>(batch, d_n, d_LU, d_lda, d_ipiv, d_nrhs, d_B, d_ldb, nullptr, d_order,
                                  max_n, threads, ctas_per_sm, d_work, work_bytes, stream, true);
}

int gbla_lu_solve_factored_batched_f32(int batch, const int* d_n, float* const* d_LU, const int* d_lda,
                                       int* const* d_ipiv, const int* d_nrhs, float* const* d_B,
                                       const int* d_ldb, const int* d_order, int max_n, int threads,
                                       int ctas_per_sm, void* d_work, size_t work_bytes,
                                       gbla_stream_t stream) {
  return lu_batched_entry<float>(batch, d_n, d_LU, d_lda, d_ipiv, d_nrhs, d_B, d_ldb, nullptr, d_order,
                                 max_n, threads, ctas_per_sm, d_work, work_bytes, stream, true);
}

}  // extern "C"

template <typename T>
static int chol_batched_entry(int batch, const int* d_n, T* const* d_A, const int* d_lda,
                              const int* d_nrhs, T* const* d_B, const int* d_ldb, int* d_info,
                              const int* d_order, int max_n, int threads, int ctas_per_sm,
                              void* d_work, size_t work_bytes, gbla_stream_t stream, bool solve_only) {
  clear_error();
  if (batch < 0) return -1;
  if (batch > 0 && !d_n) return -2;
  if (batch > 0 && !d_A) return -3;
  if (batch > 0 && !d_lda) return -4;
  if (d_nrhs && (!d_B || !d_ldb)) return -6;
  if (solve_only && batch > 0 && !d_nrhs) return -5;
  if (max_n < 0) return -10;
  if (threads != 0 && (threads % 32 != 0 || threads < 32 || threads > 1024)) return -11;
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return -12;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  unsigned* counter = c.take<unsigned>(1);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  if (batch == 0) return GBLA_OK;
  GBLA_TRYK(KK_BATCHED, s, launch_chol_batched<T>(batch, d_n, d_A, d_lda, d_nrhs, d_B, d_ldb, d_info,
                                                d_order, max_n, threads, ctas_per_sm, counter,
                                                solve_only, s));
  return GBLA_OK;
}

extern "C" {

size_t gbla_chol_batched_workspace(int batch) { return gbla_lu_batched_workspace(batch); }

int gbla_chol_solve_batched(int batch, const int* d_n, double* const* d_A, const int* d_lda,
                            const int* d_nrhs, double* const* d_B, const int* d_ldb, int* d_info,
                            const int* d_order, int max_n, int threads, int ctas_per_sm,
                            void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return chol_batched_entry<double>(batch, d_n, d_A, d_lda, d_nrhs, d_B, d_ldb, d_info, d_order,
                                    max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_chol_solve_batched_f32(int batch, const int* d_n, float* const* d_A, const int* d_lda,
                                const int* d_nrhs, float* const* d_B, const int* d_ldb, int* d_info,
                                const int* d_order, int max_n, int threads, int ctas_per_sm,
                                void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return chol_batched_entry<float>(batch, d_n, d_A, d_lda, d_nrhs, d_B, d_ldb, d_info, d_order,
                                   max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_chol_factor_batched(int batch, const int* d_n, double* const* d_A, const int* d_lda,
                             int* d_info, const int* d_order, int max_n, int threads, int ctas_per_sm,
                             void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return chol_batched_entry<double>(batch, d_n, d_A, d_lda, nullptr, nullptr, nullptr, d_info, d_order,
                                    max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_chol_factor_batched_f32(int batch, const int* d_n, float* const* d_A, const int* d_lda,
                                 int* d_info, const int* d_order, int max_n, int threads,
                                 int ctas_per_sm, void* d_work, size_t work_bytes,
                                 gbla_stream_t stream) {
  return chol_batched_entry<float>(batch, d_n, d_A, d_lda, nullptr, nullptr, nullptr, d_info, d_order,
                                   max_n, threads, ctas_per_sm, d_work, work_bytes, stream, false);
}

int gbla_chol_solve_factored_batched(int batch, const int* d_n, double* const* d_L, const int* d_lda,
                                     const int* d_nrhs, double* const* d_B, const int* d_ldb,
                                     const int* d_order, int max_n, int threads, int ctas_per_sm,
                                     void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return chol_batched_entry<double>(batch, d_n, d_L, d_lda, d_nrhs, d_B, d_ldb, nullptr, d_order, max_n,
                                    threads, ctas_per_sm, d_work, work_bytes, stream, true);
}

int gbla_chol_solve_factored_batched_f32(int batch, const int* d_n, float* const* d_L, const int* d_lda,
                                         const int* d_nrhs, float* const* d_B, const int* d_ldb,
                                         const int* d_order, int max_n, int threads, int ctas_per_sm,
                                         void* d_work, size_t work_bytes, gbla_stream_t stream) {
  return chol_batched_entry<float>(batch, d_n, d_L, d_lda, d_nrhs, d_B, d_ldb, nullptr, d_order, max_n,
                                   threads, ctas_per_sm, d_work, work_bytes, stream, true);
}

// ---------------------------------------------------------------------------
int gbla_rank_k_update(int m, int n, int k, double alpha, const double* U, int ldu, const double* V,
                       int ldv, double beta, double* C, int ldc, gbla_stream_t stream) {
  clear_error();
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (k < 0) return -3;
  if (m > 0 && k > 0 && !U) return -5;
  if (ldu < std::max(1, m)) return -6;
  if (n > 0 && k > 0 && !V) return -7;
  if (ldv < std::max(1, n)) return -8;
  if (m > 0 && n > 0 && !C) return -10;
  if (ldc < std::max(1, m)) return -11;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  GBLA_TRYK(KK_UPDATE, s, launch_rank_k(m, n, k, alpha, U, ldu, V, ldv, beta, C, ldc, s));
  return GBLA_OK;
}

// ---------------------------------------------------------------------------
size_t gbla_backward_error_workspace(int n, int nrhs) {
  if (n < 0 || nrhs < 0) return 0;
  Carver c(nullptr, 0);
  c.take<double>((size_t)std::max(n, 1) * std::max(nrhs, 1));
  c.take<double>(residual_work_doubles(std::max(n, 1), std::min(std::max(nrhs, 1), 8)));
  c.take<double>(1);
  return c.off;
}

int gbla_backward_error(int n, int nrhs, const double* A, int lda, const double* X, int ldx,
                        const double* B, int ldb, double* d_beta, void* d_work, size_t work_bytes,
                        gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !A) return -3;
  if (lda < std::max(1, n)) return -4;
  if (n > 0 && nrhs > 0 && !X) return -5;
  if (ldx < std::max(1, n)) return -6;
  if (n > 0 && nrhs > 0 && !B) return -7;
  if (ldb < std::max(1, n)) return -8;
  if (nrhs > 0 && !d_beta) return -9;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  double* R = c.take<double>((size_t)std::max(n, 1) * std::max(nrhs, 1));
  double* part = c.take<double>(residual_work_doubles(std::max(n, 1), std::min(std::max(nrhs, 1), 8)));
  double* anorm = c.take<double>(1);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  if (nrhs == 0) return GBLA_OK;
  if (n == 0) return cuda_status(cudaMemsetAsync(d_beta, 0, sizeof(double) * nrhs, s));
  GBLA_TRYK(KK_MATVEC, s, launch_row_abs_sum_max(n, A, lda, part, anorm, s));
  GBLA_TRYK(KK_MATVEC, s, launch_residual(n, nrhs, A, lda, X, ldx, B, ldb, R, n, part, s));
  GBLA_TRYK(KK_MATVEC, s, launch_backward_error_finish(n, nrhs, R, n, X, ldx, anorm, d_beta, s));
  return GBLA_OK;
}

// ---------------------------------------------------------------------------
struct IrWork {
  int* perm;
  double* V;
  int ldv;
  double* w;
  double* r;
  double* H;
  double* cs;
  double* sn;
  double* g;
  double* st;  // GmresState {res, pad}
  double* slots;
  unsigned* counter;
  unsigned* flags;
  double* t1;
  double* t2;
  double* DinvL;
  double* DinvU;
  int* info;
  double* anorm;
  double* beta;
  double* part;
  double* z;   // M^{-1} r of the current refinement step
  double* d;   // the correction being built by the restart cycles
};

static size_t ir_layout(Carver& c, int n, int m, IrWork* w) {
  const int nn = std::max(n, 1);
  const int ldv = ((nn + 31) / 32) * 32;
  IrWork t;
  t.perm = c.take<int>(nn);
  t.ldv = ldv;
  t.V = c.take<double>((size_t)ldv * (m + 1));
  t.w = c.take<double>(nn);
  t.r = c.take<double>(nn);
  t.H = c.take<double>((size_t)(m + 1) * m);
  t.cs = c.take<double>(m);
  t.sn = c.take<double>(m);
  t.g = c.take<double>(m + 1);
  t.st = c.take<double>(2);
  t.slots = c.take<double>(mgs_slots_doubles());
  t.counter = c.take<unsigned>(1);
  t.flags = c.take<unsigned>(trsv_flags_count(nn, 1));
  t.t1 = c.take<double>(nn);
  t.t2 = c.take<double>(nn);
  t.DinvL = c.take<double>(diag_inv_doubles(nn));
  t.DinvU = c.take<double>(diag_inv_doubles(nn));
  t.info = c.take<int>(1);
  t.anorm = c.take<double>(1);
  t.beta = c.take<double>(1);
  t.part = c.take<double>(residual_work_doubles(nn, 1));
  t.z = c.take<double>(nn);
  t.d = c.take<double>(nn);
  if (w) *w = t;
  return c.off;
}

size_t gbla_gmresir_workspace(int n, int restart_m) {
  if (n < 0 || restart_m < 1 || restart_m > 128) return 0;
  Carver c(nullptr, 0);
  return ir_layout(c, n, restart_m, nullptr);
}

// dst <- M^{-1} src with M = P^t L U (FP32 factors, FP64 arithmetic, inverted
// 64 x 64 diagonal blocks of L and U formed once per solve call); t1, t2:
// n-double temporaries; src and dst distinct
static cudaError_t apply_minv(int n, const float* F, int ldf, const int* perm, const double* DinvL,
                              const double* DinvU, const double* src, double* dst, double* t1,
                              double* t2, unsigned* flags, int* info, cudaStream_t s) {
  cudaError_t e;
  PROF(KK_PERM, s, launch_permute_rows(n, 1, perm, false, src, n, t1, n, s));
  if (e != cudaSuccess) return e;
  PROF(KK_TRSV, s, launch_trsv_inv<float>(true, n, F, ldf, DinvL, t1, t2, flags, info, s));
  if (e != cudaSuccess) return e;
  PROF(KK_TRSV, s, launch_trsv_inv<float>(false, n, F, ldf, DinvU, t2, dst, flags, info, s));
  return e;
}

static int read_scalar(double* host, const double* dev, const int* d_info, cudaStream_t s) {
  int info = 0;
  if (cudaMemcpyAsync(host, dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GBLA_ERR_CUDA;
  if (cudaMemcpyAsync(&info, d_info, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GBLA_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GBLA_ERR_CUDA;
  return info == GBLA_INFO_TIMEOUT ? GBLA_ERR_TIMEOUT : GBLA_OK;
}

static int check_ir_opts(const gbla_gmresir_opts* o) {
  return (o && o->restart_m >= 1 && o->restart_m <= 128 && o->max_outer >= 0 && o->restarts >= 0 &&
          o->tol >= 0.0 && o->inner_tol >= 0.0)
             ? 0
             : 1;
}

// One right-hand side, with the per-call set-up (perm, inverted diagonal
// blocks, ||A||) already in w. Refinement step: r = b - A x and its backward
// error; z = M^{-1} r; then up to `restarts` GMRES(m) cycles on
// M^{-1} A d = z (cycle c > 0 restarts from the current d with the residual
// z - M^{-1} A d), stopping once the least-squares residual is below
// inner_tol * ||z||_2; x <- x + d.
static int gmresir_one(int n, const double* A, int lda, const float* F, int ldf, const double* b,
                       double* x, const gbla_gmresir_opts* opts, gbla_gmresir_stats* stats,
                       const IrWork& w, cudaStream_t s) {
  const int m = opts->restart_m;
  const int cycles = std::max(1, opts->restarts);
  memset(stats, 0, sizeof(*stats));
  GBLA_TRY(apply_minv(n, F, ldf, w.perm, w.DinvL, w.DinvU, b, x, w.t1, w.t2, w.flags, w.info, s));
  int rc = GBLA_OK;
  for (int outer = 0;; ++outer) {
    GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, x, n, b, n, w.r, n, w.part, s));
    GBLA_TRYK(KK_MATVEC, s, launch_backward_error_finish(n, 1, w.r, n, x, n, w.anorm, w.beta, s));
    double beta = 0.0;
    rc = read_scalar(&beta, w.beta, w.info, s);
    if (rc != GBLA_OK) return rc;
    if (outer == 0) stats->beta0 = beta;
    stats->beta = beta;
    stats->outer = outer;
    if (beta <= opts->tol) {
      stats->converged = 1;
      return GBLA_OK;
    }
    if (outer >= opts->max_outer) return GBLA_ERR_NOT_CONVERGED;
    // z = M^{-1} r; d = 0
    GBLA_TRY(apply_minv(n, F, ldf, w.perm, w.DinvL, w.DinvU, w.r, w.z, w.t1, w.t2, w.flags, w.info, s));
    GBLA_TRY(cudaMemsetAsync(w.d, 0, sizeof(double) * (size_t)n, s));
    double znorm = 0.0;
    for (int cyc = 0; cyc < cycles; ++cyc) {
      // v_0 = c / ||c|| with c = z (first cycle) or z - M^{-1} A d
      const double* c0 = w.z;
      if (cyc > 0) {
        GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, w.d, n, nullptr, n, w.w, n, w.part, s));
        GBLA_TRY(apply_minv(n, F, ldf, w.perm, w.DinvL, w.DinvU, w.w, w.r, w.t1, w.t2, w.flags, w.info, s));
        GBLA_TRYK(KK_UPDATE, s, launch_axpby(n, 1.0, w.z, -1.0, w.r, w.w, s));
        c0 = w.w;
      }
      GBLA_TRYK(KK_MGS, s, launch_mgs_step(n, -1, w.V, w.ldv, c0, w.H, m + 1, w.cs, w.sn, w.g, w.st, w.slots,
                               w.counter, w.info, s));
      double beta_in = 0.0;
      rc = read_scalar(&beta_in, w.st, w.info, s);
      if (rc != GBLA_OK) return rc;
      if (cyc == 0) znorm = beta_in;
      if (!(beta_in > opts->inner_tol * znorm) || !(beta_in > 0.0)) break;
      int k = 0;
      double res = beta_in;
      for (int j = 0; j < m; ++j) {
        // w = M^{-1} A v_j
        GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, w.V + (size_t)j * w.ldv, n, nullptr, n, w.w, n, w.part, s));
        GBLA_TRY(apply_minv(n, F, ldf, w.perm, w.DinvL, w.DinvU, w.w, w.r, w.t1, w.t2, w.flags, w.info, s));
        GBLA_TRYK(KK_MGS, s, launch_mgs_step(n, j, w.V, w.ldv, w.r, w.H, m + 1, w.cs, w.sn, w.g, w.st, w.slots,
                                 w.counter, w.info, s));
        rc = read_scalar(&res, w.st, w.info, s);
        if (rc != GBLA_OK) return rc;
        k = j + 1;
        if (res <= opts->inner_tol * znorm) break;
      }
      stats->inner += k;
      GBLA_TRYK(KK_UPDATE, s, launch_gmres_update(n, k, w.V, w.ldv, w.H, m + 1, w.g, w.d, s));
      if (res <= opts->inner_tol * znorm) break;
    }
    GBLA_TRYK(KK_UPDATE, s, launch_axpby(n, 1.0, w.d, 1.0, x, x, s));
  }
}

// Per-call set-up of the refinement: the permutation of the pivots, the
// inverted diagonal blocks of L and U, ||A||_inf. Cholesky factors (ipiv
// null): no interchanges, L with its own diagonal, L^t in the upper triangle.
static int gmresir_setup(int n, const double* A, int lda, const float* F, int ldf, const int* ipiv,
                         const IrWork& w, cudaStream_t s) {
  GBLA_TRY(cudaMemsetAsync(w.info, 0, sizeof(int), s));
  GBLA_TRYK(KK_PERM, s, launch_ipiv_to_perm(n, ipiv, w.perm, s));
  GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(true, ipiv != nullptr, n, F, ldf, w.DinvL, s));
  GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(false, false, n, F, ldf, w.DinvU, s));
  GBLA_TRYK(KK_MATVEC, s, launch_row_abs_sum_max(n, A, lda, w.part, w.anorm, s));
  return GBLA_OK;
}

static int gmresir_nrhs(int n, int nrhs, const double* A, int lda, const float* F, int ldf,
                        const int* ipiv, const double* B, int ldb, double* X, int ldx,
                        const gbla_gmresir_opts* opts, gbla_gmresir_stats* stats, void* d_work,
                        size_t work_bytes, gbla_stream_t stream, bool chol) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !A) return -3;
  if (lda < std::max(1, n)) return -4;
  if (n > 0 && !F) return -5;
  if (ldf < std::max(1, n)) return -6;
  if (!chol && n > 0 && !ipiv) return -7;
  if (n > 0 && nrhs > 0 && !B) return -8;
  if (ldb < std::max(1, n)) return -9;
  if (n > 0 && nrhs > 0 && !X) return -10;
  if (ldx < std::max(1, n)) return -11;
  if (check_ir_opts(opts)) return -12;
  if (nrhs > 0 && !stats) return -13;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  IrWork w;
  ir_layout(c, n, opts->restart_m, &w);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  for (int k = 0; k < nrhs; ++k) memset(&stats[k], 0, sizeof(stats[k]));
  if (n == 0) {
    for (int k = 0; k < nrhs; ++k) stats[k].converged = 1;
    return GBLA_OK;
  }
  if (nrhs == 0) return GBLA_OK;
  const DeviceProps& dp = device_props();
  if (!dp.coop) return GBLA_ERR_DEVICE;
  int rc = gmresir_setup(n, A, lda, F, ldf, chol ? nullptr : ipiv, w, s);
  if (rc != GBLA_OK) return rc;
  int all = GBLA_OK;
  for (int k = 0; k < nrhs; ++k) {
    rc = gmresir_one(n, A, lda, F, ldf, B + (size_t)k * ldb, X + (size_t)k * ldx, opts, &stats[k], w, s);
    if (rc == GBLA_ERR_NOT_CONVERGED) all = rc;
    else if (rc != GBLA_OK) return rc;
  }
  return all;
}

int gbla_gmresir_solve_nrhs(int n, int nrhs, const double* A, int lda, const float* F, int ldf,
                            const int* ipiv, const double* B, int ldb, double* X, int ldx,
                            const gbla_gmresir_opts* opts, gbla_gmresir_stats* stats,
                            void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  return gmresir_nrhs(n, nrhs, A, lda, F, ldf, ipiv, B, ldb, X, ldx, opts, stats, d_work, work_bytes,
                      stream, false);
}

int gbla_chol_gmresir_solve_nrhs(int n, int nrhs, const double* A, int lda, const float* F, int ldf,
                                 const double* B, int ldb, double* X, int ldx,
                                 const gbla_gmresir_opts* opts, gbla_gmresir_stats* stats,
                                 void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  const int rc = gmresir_nrhs(n, nrhs, A, lda, F, ldf, nullptr, B, ldb, X, ldx, opts, stats, d_work,
                              work_bytes, stream, true);
  // argument positions of this entry point (no ipiv)
  return rc < 0 && rc <= -8 ? rc + 1 : rc;
}

// ---------------------------------------------------------------------------
// Mixed-precision Cholesky (steps a1, a3, a4 for SPD systems in low
// precision): F <- fp32 of A's lower triangle, factored in place; the strict
// upper triangle of F receives L^t for the refinement's back substitution.
static size_t chol_mixed_layout(Carver& c, int n, int nb, int prec, void** Ak, void** Bk, int** eA,
                                int* ldk) {
  const int elem = prec == GBLA_PREC_TF32 ? 4 : 2;
  const int lk = ((prec_kmult(prec) * nb + 63) / 64) * 64;
  void* a = nullptr;
  void* b = nullptr;
  int* e = nullptr;
  if (prec_is_tensor(prec)) {
    a = c.take<char>((size_t)std::max(n, 1) * lk * elem);
    if (prec_is_split(prec)) b = c.take<char>((size_t)std::max(n, 1) * lk * elem);
    e = c.take<int>((size_t)std::max(n, 1));
  } else {
    c.take<int>(1);
  }
  if (Ak) *Ak = a;
  if (Bk) *Bk = b;
  if (eA) *eA = e;
  if (ldk) *ldk = lk;
  return c.off;
}

size_t gbla_chol_factor_mixed_workspace(int n, int nb, int prec) {
  if (nb == 0) nb = 256;
  if (n < 0 || nb % 64 != 0 || nb < 64 || nb > 256 || prec < GBLA_PREC_FP32 || prec > GBLA_PREC_BF16X3)
    return 0;
  Carver c(nullptr, 0);
  return chol_mixed_layout(c, n, nb, prec, nullptr, nullptr, nullptr, nullptr);
}

int gbla_chol_factor_mixed(int n, const double* A, int lda, float* F, int ldf, int* d_info, int prec,
                           int nb, void* d_work, size_t work_bytes, gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !F) return -4;
  if (ldf < std::max(1, n)) return -5;
  if (!d_info) return -6;
  if (prec < GBLA_PREC_FP32 || prec > GBLA_PREC_BF16X3) return -7;
  if (nb == 0) nb = 256;
  if (nb % 64 != 0 || nb < 64 || nb > 256) return -8;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  void* Ak = nullptr;
  void* Bk = nullptr;
  int* eA = nullptr;
  int ldk = 0;
  chol_mixed_layout(c, n, nb, prec, &Ak, &Bk, &eA, &ldk);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  GBLA_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0) return GBLA_OK;
  GBLA_TRYK(KK_COPY, s, launch_copy_d2f(A, lda, F, ldf, n, n, s, true));
  return cuda_status(launch_chol_mixed(n, F, ldf, nb, prec, Ak, Bk, ldk, eA, d_info, s));
}

int gbla_gmresir_solve(int n, const double* A, int lda, const float* F, int ldf, const int* ipiv,
                       const double* b, double* x, const gbla_gmresir_opts* opts,
                       gbla_gmresir_stats* stats, void* d_work, size_t work_bytes,
                       gbla_stream_t stream) {
  clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !F) return -4;
  if (ldf < std::max(1, n)) return -5;
  if (n > 0 && !ipiv) return -6;
  if (n > 0 && !b) return -7;
  if (n > 0 && !x) return -8;
  if (check_ir_opts(opts)) return -9;
  if (!stats) return -10;
  return gbla_gmresir_solve_nrhs(n, 1, A, lda, F, ldf, ipiv, b, std::max(1, n), x, std::max(1, n),
                                 opts, stats, d_work, work_bytes, stream);
}


// ---------------------------------------------------------------------------
// Standalone GMRES(m) and BiCGSTAB (paper section 2: the library's
// non-stationary iterative solvers), FP64, with an optional preconditioner
// M = P^t L U from gbla_lu_factor_mixed (FP32 factors, FP64 arithmetic).
struct KrylovWork {
  IrWork ir;        // Krylov basis, Hessenberg, rotations, preconditioner pieces
  double* rt;       // BiCGSTAB shadow residual
  double* p;
  double* v;
  double* sv;
  double* t;
  double* ph;
  double* sh;
  double* dpart;    // inner-product partial sums
  double* scal;     // scalars read by the host
  BcgState* bcg;
};

static size_t krylov_layout(Carver& c, int n, int m, KrylovWork* w) {
  const int nn = std::max(n, 1);
  KrylovWork t;
  ir_layout(c, n, m, &t.ir);
  t.rt = c.take<double>(nn);
  t.p = c.take<double>(nn);
  t.v = c.take<double>(nn);
  t.sv = c.take<double>(nn);
  t.t = c.take<double>(nn);
  t.ph = c.take<double>(nn);
  t.sh = c.take<double>(nn);
  t.dpart = c.take<double>(dot_part_doubles());
  t.scal = c.take<double>(4);
  t.bcg = reinterpret_cast<BcgState*>(c.take<char>(sizeof(BcgState)));
  if (w) *w = t;
  return c.off;
}

size_t gbla_krylov_workspace(int n, int restart_m) {
  if (n < 0 || restart_m < 1 || restart_m > 128) return 0;
  Carver c(nullptr, 0);
  return krylov_layout(c, n, restart_m, nullptr);
}

static int krylov_args(int n, const double* A, int lda, const double* b, double* x, const float* F,
                       int ldf, const int* ipiv, const gbla_krylov_opts* opts,
                       gbla_krylov_stats* stats) {
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && !b) return -4;
  if (n > 0 && !x) return -5;
  if ((F != nullptr) != (ipiv != nullptr)) return -6;
  if (F && ldf < std::max(1, n)) return -7;
  if (!opts || !(opts->tol >= 0.0) || opts->max_iter < 0 || opts->restart_m < 1 || opts->restart_m > 128)
    return -9;
  if (!stats) return -10;
  return 0;
}

// ||b - A x||_2 / ||b||_2 with the device matvec and inner products
static int krylov_relres(int n, const double* A, int lda, const double* b, const double* x,
                         const KrylovWork& w, cudaStream_t s, double* relres) {
  GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, x, n, b, n, w.ir.r, n, w.ir.part, s));
  GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 2, w.ir.r, w.ir.r, b, b, w.dpart, w.scal, w.scal + 1, s));
  double h[2];
  GBLA_TRY(cudaMemcpyAsync(h, w.scal, sizeof(h), cudaMemcpyDeviceToHost, s));
  GBLA_TRY(cudaStreamSynchronize(s));
  *relres = h[1] > 0.0 ? sqrt(h[0] / h[1]) : sqrt(h[0]);
  return GBLA_OK;
}

int gbla_gmres_solve(int n, const double* A, int lda, const double* b, double* x, const float* F,
                     int ldf, const int* ipiv, const gbla_krylov_opts* opts,
                     gbla_krylov_stats* stats, void* d_work, size_t work_bytes,
                     gbla_stream_t stream) {
  clear_error();
  const int bad = krylov_args(n, A, lda, b, x, F, ldf, ipiv, opts, stats);
  if (bad) return bad;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  const int m = opts->restart_m;
  Carver c(d_work, work_bytes);
  KrylovWork w;
  krylov_layout(c, n, m, &w);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  memset(stats, 0, sizeof(*stats));
  if (n == 0) {
    stats->converged = 1;
    return GBLA_OK;
  }
  const DeviceProps& dp = device_props();
  if (!dp.coop) return GBLA_ERR_DEVICE;
  const IrWork& ir = w.ir;
  const bool pre = F != nullptr;
  GBLA_TRY(cudaMemsetAsync(ir.info, 0, sizeof(int), s));
  if (pre) {
    GBLA_TRYK(KK_PERM, s, launch_ipiv_to_perm(n, ipiv, ir.perm, s));
    GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(true, true, n, F, ldf, ir.DinvL, s));
    GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(false, false, n, F, ldf, ir.DinvU, s));
    GBLA_TRY(apply_minv(n, F, ldf, ir.perm, ir.DinvL, ir.DinvU, b, ir.z, ir.t1, ir.t2, ir.flags, ir.info, s));
  }
  // the stopping norm: ||M^{-1} b||_2 (left preconditioning) or ||b||_2
  const double* bz = pre ? ir.z : b;
  GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 1, bz, bz, nullptr, nullptr, w.dpart, w.scal, nullptr, s));
  double bn2 = 0.0;
  int rc = read_scalar(&bn2, w.scal, ir.info, s);
  if (rc != GBLA_OK) return rc;
  const double bn = sqrt(bn2);
  int it = 0;
  bool conv = bn == 0.0;
  while (!conv) {
    // r = b - A x; z = M^{-1} r; v_0 = z / ||z||
    GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, x, n, b, n, ir.r, n, ir.part, s));
    const double* z = ir.r;
    if (pre) {
      GBLA_TRY(apply_minv(n, F, ldf, ir.perm, ir.DinvL, ir.DinvU, ir.r, ir.z, ir.t1, ir.t2, ir.flags, ir.info, s));
      z = ir.z;
    }
    GBLA_TRYK(KK_MGS, s, launch_mgs_step(n, -1, ir.V, ir.ldv, z, ir.H, m + 1, ir.cs, ir.sn, ir.g, ir.st,
                             ir.slots, ir.counter, ir.info, s));
    double beta = 0.0;
    rc = read_scalar(&beta, ir.st, ir.info, s);
    if (rc != GBLA_OK) return rc;
    if (beta <= opts->tol * bn) {
      conv = true;
      break;
    }
    if (it >= opts->max_iter) break;
    int k = 0;
    double res = beta;
    for (int j = 0; j < m && it < opts->max_iter; ++j) {
      GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, ir.V + (size_t)j * ir.ldv, n, nullptr, n, ir.w, n,
                                              ir.part, s));
      const double* wv = ir.w;
      if (pre) {
        GBLA_TRY(apply_minv(n, F, ldf, ir.perm, ir.DinvL, ir.DinvU, ir.w, ir.r, ir.t1, ir.t2, ir.flags, ir.info, s));
        wv = ir.r;
      }
      GBLA_TRYK(KK_MGS, s, launch_mgs_step(n, j, ir.V, ir.ldv, wv, ir.H, m + 1, ir.cs, ir.sn, ir.g, ir.st,
                               ir.slots, ir.counter, ir.info, s));
      rc = read_scalar(&res, ir.st, ir.info, s);
      if (rc != GBLA_OK) return rc;
      ++it;
      k = j + 1;
      if (res <= opts->tol * bn) break;
    }
    GBLA_TRYK(KK_UPDATE, s, launch_gmres_update(n, k, ir.V, ir.ldv, ir.H, m + 1, ir.g, x, s));
    if (res <= opts->tol * bn) conv = true;
  }
  stats->iterations = it;
  stats->converged = conv ? 1 : 0;
  rc = krylov_relres(n, A, lda, b, x, w, s, &stats->relres);
  if (rc != GBLA_OK) return rc;
  return conv ? GBLA_OK : GBLA_ERR_NOT_CONVERGED;
}

int gbla_bicgstab_solve(int n, const double* A, int lda, const double* b, double* x, const float* F,
                        int ldf, const int* ipiv, const gbla_krylov_opts* opts,
                        gbla_krylov_stats* stats, void* d_work, size_t work_bytes,
                        gbla_stream_t stream) {
  clear_error();
  const int bad = krylov_args(n, A, lda, b, x, F, ldf, ipiv, opts, stats);
  if (bad) return bad;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (!d_work || !aligned256(d_work)) return GBLA_ERR_WORKSPACE;
  Carver c(d_work, work_bytes);
  KrylovWork w;
  krylov_layout(c, n, opts->restart_m, &w);
  if (!c.ok) return GBLA_ERR_WORKSPACE;
  memset(stats, 0, sizeof(*stats));
  if (n == 0) {
    stats->converged = 1;
    return GBLA_OK;
  }
  const DeviceProps& dp = device_props();
  if (!dp.coop) return GBLA_ERR_DEVICE;
  const IrWork& ir = w.ir;
  const bool pre = F != nullptr;
  GBLA_TRY(cudaMemsetAsync(ir.info, 0, sizeof(int), s));
  if (pre) {
    GBLA_TRYK(KK_PERM, s, launch_ipiv_to_perm(n, ipiv, ir.perm, s));
    GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(true, true, n, F, ldf, ir.DinvL, s));
    GBLA_TRYK(KK_TRSV, s, launch_diag_inv<float>(false, false, n, F, ldf, ir.DinvU, s));
  }
  // r = b - A x, r~ = r, p = v = 0, rho = alpha = omega = 1
  double* r = ir.r;
  GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, x, n, b, n, r, n, ir.part, s));
  GBLA_TRY(cudaMemcpyAsync(w.rt, r, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, s));
  GBLA_TRY(cudaMemsetAsync(w.p, 0, sizeof(double) * (size_t)n, s));
  GBLA_TRY(cudaMemsetAsync(w.v, 0, sizeof(double) * (size_t)n, s));
  GBLA_TRYK(KK_UPDATE, s, launch_bcg_init(w.bcg, s));
  GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 2, r, r, b, b, w.dpart, &w.bcg->rr, w.scal, s));
  BcgState h;
  double bn2 = 0.0;
  GBLA_TRY(cudaMemcpyAsync(&h, w.bcg, sizeof(h), cudaMemcpyDeviceToHost, s));
  GBLA_TRY(cudaMemcpyAsync(&bn2, w.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  GBLA_TRY(cudaStreamSynchronize(s));
  const double bn = sqrt(bn2);
  const double* ph = pre ? w.ph : w.p;
  const double* sh = pre ? w.sh : w.sv;
  bool conv = bn == 0.0 || sqrt(h.rr) <= opts->tol * bn;
  int it = 0, brk = 0;
  while (!conv && it < opts->max_iter) {
    GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 1, w.rt, r, nullptr, nullptr, w.dpart, &w.bcg->rho_new, nullptr, s));
    GBLA_TRYK(KK_UPDATE, s, launch_bcg_p(n, r, w.v, w.p, w.bcg, s));
    if (pre) GBLA_TRY(apply_minv(n, F, ldf, ir.perm, ir.DinvL, ir.DinvU, w.p, w.ph, ir.t1, ir.t2, ir.flags, ir.info, s));
    GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, ph, n, nullptr, n, w.v, n, ir.part, s));
    GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 1, w.rt, w.v, nullptr, nullptr, w.dpart, &w.bcg->rv, nullptr, s));
    GBLA_TRYK(KK_UPDATE, s, launch_bcg_s(n, r, w.v, w.sv, w.bcg, s));
    if (pre) GBLA_TRY(apply_minv(n, F, ldf, ir.perm, ir.DinvL, ir.DinvU, w.sv, w.sh, ir.t1, ir.t2, ir.flags, ir.info, s));
    GBLA_TRYK(KK_MATVEC, s, launch_residual(n, 1, A, lda, sh, n, nullptr, n, w.t, n, ir.part, s));
    GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 2, w.t, w.sv, w.t, w.t, w.dpart, &w.bcg->ts, &w.bcg->tt, s));
    GBLA_TRYK(KK_UPDATE, s, launch_bcg_xr(n, x, ph, sh, w.sv, w.t, r, w.bcg, s));
    GBLA_TRYK(KK_MATVEC, s, launch_dots(n, 1, r, r, nullptr, nullptr, w.dpart, &w.bcg->rr, nullptr, s));
    int info = 0;
    GBLA_TRY(cudaMemcpyAsync(&h, w.bcg, sizeof(h), cudaMemcpyDeviceToHost, s));
    GBLA_TRY(cudaMemcpyAsync(&info, ir.info, sizeof(int), cudaMemcpyDeviceToHost, s));
    GBLA_TRY(cudaStreamSynchronize(s));
    if (info == GBLA_INFO_TIMEOUT) return GBLA_ERR_TIMEOUT;
    ++it;
    conv = sqrt(h.rr) <= opts->tol * bn;
    if (!conv && h.status) {
      brk = 1;  // rho', (r~, v) or t vanished without the residual being small
      break;
    }
  }
  stats->iterations = it;
  stats->converged = conv ? 1 : 0;
  stats->breakdown = brk;
  int rc = krylov_relres(n, A, lda, b, x, w, s, &stats->relres);
  if (rc != GBLA_OK) return rc;
  return conv ? GBLA_OK : GBLA_ERR_NOT_CONVERGED;
}

}  // extern "C"
