// Allocation-free variant of the l2-ball projection.
//
// gbri_proj_l2ball takes its reduction scratch (one FP64 partial sum per block)
// from the stream-ordered allocator.  Some callers cannot allocate device memory
// at the moment they need the projection: a host whose own pool allocator has
// already claimed all device memory (a cudaMalloc there fails or fragments the
// pool), an out-of-memory recovery path, or a latency-critical loop that must not
// risk the implicit device synchronisation of cudaFree.  For them this file keeps
// the scratch in a fixed, file-scope device array instead.
#include <mutex>

#include "prox.cuh"

namespace gbri {
namespace {

// One FP64 partial per reduction block: 1024 * 8 bytes = 8 KB held by every GPU that
// loads the library, until the process exits.
constexpr int kNoAllocPartials = 1024;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  The symbol's
// host-side name is not a device address, so it is resolved once per device with
// that device current (cudaGetSymbolAddress) and cached.
int32_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(GBRI_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static l2-ball scratch)");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return GBRI_OK;
}

}  // namespace
}  // namespace gbri

using namespace gbri;

extern "C" int32_t gbri_proj_l2ball_noalloc(const float* d_z, const float* d_center, float* d_out, int64_t M,
                                            double eps, double* d_norm_out, void* stream) {
  GBRI_CHECK(M >= 0 && eps >= 0, GBRI_EINVAL, "bad size or eps");
  GBRI_CHECK(M == 0 || (d_z && d_center && d_out), GBRI_EINVAL, "null argument");
  const int need = l2ball_blocks(M);
  if (need > kNoAllocPartials)
    return set_error(GBRI_EINVAL, "gbri_proj_l2ball_noalloc: this launch needs " + std::to_string(need) +
                                      " reduction partials but the static scratch holds " +
                                      std::to_string(kNoAllocPartials));
  double* scratch = nullptr;
  GBRI_TRY(scratch_on_current_device(&scratch));
  // every partial the apply kernel reads is written earlier in the same call: nothing to clear
  return proj_l2ball_with_scratch(d_z, d_center, d_out, M, eps, d_norm_out, scratch, need, (cudaStream_t)stream);
}
