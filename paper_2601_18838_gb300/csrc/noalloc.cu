// kpme_spread_noalloc: charge spreading for callers that cannot allocate device memory.
//
// Some callers of this library are not allowed to call cudaMalloc at the moment they
// need a charge mesh: code that runs while a stream is being captured into a CUDA graph
// (where an allocation is either forbidden or not recorded), engines whose device memory
// is entirely owned by their own pool allocator, and latency-critical loops that cannot
// afford the device-wide synchronisation an allocation implies.  They cannot create a
// plan either, because a plan allocates its scratch.  This entry point spreads into a
// float32 accumulation mesh that lives in a fixed static device array instead, then
// writes the float64 mesh into the caller's buffer; it calls no allocating routine.
//
// The static array is shared by every call in the process: calls whose GPU work
// overlaps (different streams, or different host threads on one device) race on it and
// must be serialised by the caller.  Each call clears the part it uses before spreading.
#include "kpme_internal.cuh"

#include <cmath>
#include <mutex>

namespace {

// Float64 charge sum in the first 256 bytes, then the float32 mesh (K <= KPME_NOALLOC_MAX_K).
constexpr int64_t kMeshFloats = (int64_t)KPME_NOALLOC_MAX_K * KPME_NOALLOC_MAX_K * KPME_NOALLOC_MAX_K;
constexpr int64_t kScratchBytes = 256 + kMeshFloats * (int64_t)sizeof(float);
static __device__ __align__(256) double g_noalloc_scratch[kScratchBytes / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

// One-time per-device set-up (with that device current): the device address of the static
// array and the SM count.  Host code must not use g_noalloc_scratch directly: on the host
// that name is only a stand-in for the symbol.
kpme_status_t setup(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return KPME_ERR_CUDA;
    }
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return KPME_ERR_CUDA;
    }
    g_sms[dev] = n;
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  *sms = g_sms[dev];
  return KPME_OK;
}

}  // namespace

extern "C" kpme_status_t kpme_spread_noalloc(const kpme_params_t* params, void* stream, int64_t n, const double* x,
                                             const double* q, double* Q) {
  if (!params || !Q || n < 0 || (n > 0 && (!x || !q))) return KPME_ERR_INVALID_ARG;
  const kpme_params_t& p = *params;
  if (p.interp != KPME_INTERP_BSPLINE) return KPME_ERR_UNSUPPORTED;   // B-spline spreading only
  const bool ok = std::isfinite(p.radius) && p.radius > 0 && (p.order == 4 || p.order == 6 || p.order == 8) &&
                  p.K % 2 == 0 && p.K >= 2 * p.order && std::isfinite(p.center[0]) && std::isfinite(p.center[1]) &&
                  std::isfinite(p.center[2]);
  if (!ok) return KPME_ERR_INVALID_ARG;
  if (p.K > KPME_NOALLOC_MAX_K) return KPME_ERR_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KPME_ERR_CUDA;
  void* base = nullptr;
  int sms = 0;
  kpme_status_t st = setup(dev, &base, &sms);
  if (st != KPME_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t k3 = (int64_t)p.K * p.K * p.K;
  double* sumq = reinterpret_cast<double*>(base);
  float* mesh = reinterpret_cast<float*>(reinterpret_cast<char*>(base) + 256);
  if (cudaMemsetAsync(base, 0, 256 + k3 * sizeof(float), s) != cudaSuccess) return KPME_ERR_CUDA;
  if (kpme::launch_spread_raw(p, sms, s, n, x, q, mesh, sumq) != cudaSuccess) return KPME_ERR_CUDA;
  if (kpme::launch_convert(mesh, false, Q, true, k3, s) != cudaSuccess) return KPME_ERR_CUDA;
  return KPME_OK;
}
