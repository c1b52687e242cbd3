// direct_noalloc.cu -- an entry point that allocates no device memory.
//
// lens_direct_deflect_noalloc runs the same float32 direct sum as
// lens_direct_deflect, but its scratch (every star split into a float hi/lo
// pair plus a float mass) lives in a fixed file-scope device array instead of
// memory obtained per call.  It serves callers that may not allocate device
// memory: a host application that owns the whole device-memory budget and
// hands the library only its input and output buffers, a memory-capped
// service whose pool must not grow while it runs, or a loop that cannot
// afford an allocation stalling or failing in the middle of a step.
//
// Limits and rules (also in include/lens.h):
//   - at most kNoAllocMaxStars stars per call; larger calls are rejected
//     with LENS_EINVAL before anything is launched;
//   - the array is a single static object per device: every GPU that loads
//     the library holds its kNoAllocScratchBytes until the process exits;
//   - the first call on a device looks up the array's device address with
//     cudaGetSymbolAddress (with that device current) and caches it; that
//     first call should come before any stream capture;
//   - every call writes all the scratch entries it reads (nothing has to
//     start at zero), and all calls share the one array, so two calls that
//     overlap on the GPU (different streams, or different host threads)
//     race: the caller must order them.
#include <mutex>

#include "lens_internal.h"

namespace lens {
void direct_f32_into(const double* stars, const double* masses, int64_t n, double ks, double g,
                     const double* rays, int64_t m, double* y, double* jac, float4* hl, float* mf,
                     cudaStream_t s);
}  // namespace lens

namespace {

constexpr int64_t kNoAllocMaxStars = 1 << 18;  // 262144 stars
constexpr size_t kNoAllocScratchBytes = (size_t)kNoAllocMaxStars * (sizeof(float4) + sizeof(float));

// split star positions (float4) followed by float32 masses
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

void* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) lens::fail(LENS_EINVAL, "device ordinal out of range");
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      lens::fail(LENS_ECUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") +
                                 cudaGetErrorString(e));
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" lens_status lens_direct_deflect_noalloc(const double* stars_xy, const double* masses,
                                                   int64_t n, double kappa_s, double gamma,
                                                   const double* rays_xy, int64_t m,
                                                   double* y_out, double* jac_out, void* stream) {
  try {
    if (n < 0 || m < 0) lens::fail(LENS_EINVAL, "sizes must be >= 0");
    if (n > kNoAllocMaxStars)
      lens::fail(LENS_EINVAL, "lens_direct_deflect_noalloc takes at most 262144 stars (its fixed "
                              "device scratch); use lens_direct_deflect for more");
    if (m > 0 && (!rays_xy || !y_out || (n > 0 && (!stars_xy || !masses))))
      lens::fail(LENS_EINVAL, "NULL buffer");
    int dev = 0;
    LENS_CUDA(cudaGetDevice(&dev));
    unsigned char* base = static_cast<unsigned char*>(scratch_address(dev));
    if (m > 0) {
      float4* hl = reinterpret_cast<float4*>(base);
      float* mf = reinterpret_cast<float*>(base + (size_t)kNoAllocMaxStars * sizeof(float4));
      lens::direct_f32_into(stars_xy, masses, n, kappa_s, gamma, rays_xy, m, y_out, jac_out, hl,
                            mf, reinterpret_cast<cudaStream_t>(stream));
    }
  } catch (const lens::Error& e) {
    lens::set_last_error(e.msg);
    return e.status;
  } catch (const std::exception& e) {
    lens::set_last_error(std::string("internal: ") + e.what());
    return LENS_ECUDA;
  }
  lens::set_last_error("");
  return LENS_OK;
}
