// FP64 LU factorisation for callers that cannot allocate device memory.
//
// Some callers have no way to obtain scratch memory on the device: code that
// runs where cudaMalloc is forbidden or unavailable (inside a pre-sized memory
// pool they do not own, in a plugin whose host application owns every
// allocation, or on a path that must not touch the allocator at all). For them
// gbla_lu_factor_static performs the same factorisation as gbla_lu_factor but
// keeps its only scratch -- the exchange slots of the panel kernel -- in a
// fixed array that lives in this library's device image. The caller passes
// the matrix, the pivot vector and the info word, nothing else.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it (kStaticSlotsBytes, about 290 KiB) until the process exits.
// Host code cannot use the array's name as a device address, so the address
// is looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on that device.
#include <mutex>

#include "internal.h"

namespace gbla {

// Room for the panel kernels' exchange area (two parities of slots for up to
// kPanelMaxSms CTAs; the panel launcher never uses more CTAs than that, on
// any device) and the inner update's counters.
constexpr int kStaticMaxSms = 256;
static_assert(kStaticMaxSms == kPanelMaxSms, "the fixed array follows the panel kernels' bound");
constexpr size_t kStaticSlotsDoubles =
    (size_t)2 * (kStaticMaxSms + 1) * kPanelSlotW + kInnerCounters / 2;
constexpr size_t kStaticSlotsBytes = kStaticSlotsDoubles * sizeof(double);
static_assert(kStaticSlotsBytes < 300 * 1024, "the fixed scratch is meant to stay below 300 KiB");

static __device__ __align__(256) double g_static_slots[kStaticSlotsDoubles];

static cudaError_t static_slots_address(int device, double** out) {
  static std::mutex mu;
  static double* addr[64] = {nullptr};
  std::lock_guard<std::mutex> lock(mu);
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  if (!addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_slots);
    if (e != cudaSuccess) return e;
    addr[device] = static_cast<double*>(p);
  }
  *out = addr[device];
  return cudaSuccess;
}

#define NOALLOC_TRY(expr)                                                        \
  do {                                                                           \
    const int _st = api_cuda_status((expr), #expr, "noalloc.cu", __LINE__);      \
    if (_st != GBLA_OK) return _st;                                              \
  } while (0)

}  // namespace gbla

using namespace gbla;

extern "C" int gbla_lu_factor_static(int n, double* A, int lda, int* ipiv, int* d_info, int nb,
                                     gbla_stream_t stream) {
  api_clear_error();
  if (n < 0) return -1;
  if (n > 0 && !A) return -2;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (n > 0 && !ipiv) return -4;
  if (!d_info) return -5;
  if (nb == 0) nb = 256;
  if (nb % 32 != 0 || nb < 32 || nb > 256) return -6;
  int dev = -1;
  NOALLOC_TRY(cudaGetDevice(&dev));
  const DeviceProps& dp = device_props();
  if (dp.device < 0) return GBLA_ERR_CUDA;
  if (!dp.coop) return GBLA_ERR_DEVICE;
  // the fixed array must hold every slot the panel kernels can use
  if (panel_slots_doubles() > kStaticSlotsDoubles) return GBLA_ERR_WORKSPACE;
  double* slots = nullptr;
  NOALLOC_TRY(static_slots_address(dev, &slots));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  NOALLOC_TRY(cudaMemsetAsync(d_info, 0, sizeof(int), s));
  if (n == 0) return GBLA_OK;
  // the array keeps the previous call's contents: stale slot tags must not
  // match this factorisation's, so the slots start from zero every call
  NOALLOC_TRY(cudaMemsetAsync(slots, 0, sizeof(double) * panel_slots_doubles(), s));
  LuWork w;
  w.slots = slots;
  w.Ak = w.Bk = nullptr;
  w.eA = w.eB = nullptr;
  w.ldk = 0;
  return api_cuda_status(blocked_lu<double>(n, A, lda, ipiv, d_info, nb, 0, w, s),
                         "blocked_lu<double>", "noalloc.cu", __LINE__);
}
