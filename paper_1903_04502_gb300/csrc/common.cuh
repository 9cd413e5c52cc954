// Internal helpers shared by the library's translation units: status handling,
// kernel-launch bookkeeping (launch counter, optional CUDA-event timing per kernel
// kind), device reductions with FP64 block sums.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gbri.h"

namespace gbri {

// ---- status ---------------------------------------------------------------
int32_t set_error(int32_t code, const std::string& msg);
int32_t cuda_error(cudaError_t e, const char* what);

#define GBRI_CHECK_CUDA(call)                                 \
  do {                                                        \
    cudaError_t _e = (call);                                  \
    if (_e != cudaSuccess) return ::gbri::cuda_error(_e, #call); \
  } while (0)

#define GBRI_CHECK(cond, code, msg)                   \
  do {                                                \
    if (!(cond)) return ::gbri::set_error((code), (msg)); \
  } while (0)

#define GBRI_TRY(call)               \
  do {                               \
    int32_t _s = (call);             \
    if (_s < 0) return _s;           \
  } while (0)

// ---- launch bookkeeping ----------------------------------------------------
// Every kernel launch of the library goes through launch_begin / launch_end so
// that the launch count is exact and, when profiling is enabled, a pair of CUDA
// events brackets the launch on its own stream.
// `own` = false for library calls that launch kernels which are not ours
// (cuFFT): they are timed but not counted.
void launch_begin(int kind, cudaStream_t s, bool own = true);
int32_t launch_end(int kind, cudaStream_t s);  // checks cudaGetLastError

int num_sms();
// True while per-kernel event timing is on (graph replay is then avoided so that
// every kernel launch gets its own event pair).
bool profiling_enabled();
// Account for kernels launched by a graph replay (captured launches are not launches).
void add_launches(int64_t n);
int64_t launch_counter();

// ---- device helpers ----------------------------------------------------------
// Block-wide sum of a double; result valid in thread 0.  blockDim.x must be a
// multiple of 32 and at most 1024.
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v, double* sh /* >= 32 doubles */) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}

// Kahan-compensated FP32 accumulator for per-thread partial sums of squares.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Sum a fixed-length array of double partials in a fixed order (deterministic);
// all threads of the block get the result.
__device__ __forceinline__ double reduce_partials(const double* p, int n, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += p[i];
  v = block_sum(v, sh);
  if (threadIdx.x == 0) sh[32] = v;
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace gbri
