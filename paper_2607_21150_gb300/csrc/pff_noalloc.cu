// Chebyshev smoothing for callers that cannot allocate device memory.
//
// pff_chebyshev_smooth needs three work vectors that the caller allocates.  Some
// callers cannot do that at the point where they smooth: code whose device
// memory belongs to another allocator (a framework's caching pool, or a budget
// reserved once at start-up) and that is not allowed to call cudaMalloc itself,
// and code inside a latency-sensitive solver loop, where cudaMalloc/cudaFree may
// synchronise the whole device.  pff_chebyshev_smooth_noalloc serves them: the
// work vectors live in one fixed array compiled into this library
// (kNoAllocMaxEntries entries per vector, 48 MiB, held by every GPU that loads
// the library until the process exits), and the call itself allocates nothing.
#include <mutex>
#include <string>

#include "../../include/pff.h"
#include "pff_internal.h"

namespace {

constexpr long long kNoAllocMaxEntries = 1LL << 21;  // per work vector: 4 * N_n <= 2 097 152
constexpr int kMaxDevices = 64;

// Three work vectors of up to kNoAllocMaxEntries doubles each.  FP64 calls
// place them at doubles 0, n and 2n; FP32 calls pack their three vectors of
// n floats contiguously at floats 0, n and 2n, i.e. in the first half of the
// array.  Shared by every call on a device.
static __device__ __align__(256) double g_smooth_scratch[3 * kNoAllocMaxEntries];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int pff_chebyshev_smooth_noalloc(pff_level* level, pff_prec prec, int degree, double lmin, double lmax,
                                            const void* diag, const void* b, void* x, void* stream) {
  if (!level) return pff::set_last_error(PFF_ERR_INVALID, "pff_chebyshev_smooth_noalloc: null level");
  const long long n = 4 * (long long)pff_level_num_nodes(level);
  if (n > kNoAllocMaxEntries)
    return pff::set_last_error(
        PFF_ERR_INVALID,
        ("pff_chebyshev_smooth_noalloc: level has " + std::to_string(n) + " DoFs, more than the " +
         std::to_string(kNoAllocMaxEntries) + " its built-in work space holds; use pff_chebyshev_smooth")
            .c_str());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return pff::set_last_error(PFF_ERR_CUDA, (std::string("pff_chebyshev_smooth_noalloc: cudaGetDevice: ") +
                                              cudaGetErrorString(e)).c_str());
  if (dev < 0 || dev >= kMaxDevices)
    return pff::set_last_error(PFF_ERR_INVALID, "pff_chebyshev_smooth_noalloc: device index beyond 63");
  void* work = nullptr;
  {
    // One-time set-up per device (with that device current): the host-side
    // name of the array is only a stand-in, so ask the runtime for its device
    // address.
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_smooth_scratch);
      if (e != cudaSuccess)
        return pff::set_last_error(PFF_ERR_CUDA, (std::string("pff_chebyshev_smooth_noalloc: cudaGetSymbolAddress: ") +
                                                  cudaGetErrorString(e)).c_str());
      g_scratch_ptr[dev] = p;
    }
    work = g_scratch_ptr[dev];
  }
  // Same smoother as pff_chebyshev_smooth; every work entry it reads is written
  // earlier in the same call, so the array's leftover contents never matter.
  return pff_chebyshev_smooth(level, prec, degree, lmin, lmax, diag, b, x, work, stream);
}
