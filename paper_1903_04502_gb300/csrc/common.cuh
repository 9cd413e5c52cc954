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
// Test hook (gbri_debug_inject_alloc_failure): true for the one device allocation the caller
// asked to fail; the library's allocation helpers then report GBRI_ENOMEM as for a real failure.
bool alloc_fault_injected();
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

// Plain FP64 accumulator (the FP64 path needs no compensation).
struct SumD {
  double s = 0.0;
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};

// ---- arithmetic type of a path ------------------------------------------------
// R = float: FP32 bulk with FP64 global sums (per-thread compensated FP32 partials);
// R = double: the plain FP64 path.  cplx<R> is the interleaved complex type.
template <class R> struct RealT;
template <> struct RealT<float> { using C = float2; using Acc = KahanF; };
template <> struct RealT<double> { using C = double2; using Acc = SumD; };
template <class R> using cplx = typename RealT<R>::C;
template <class R> using acc_t = typename RealT<R>::Acc;

template <class R>
__host__ __device__ __forceinline__ cplx<R> mkc(R re, R im) {
  cplx<R> v;
  v.x = re;
  v.y = im;
  return v;
}
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float max_r(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_r(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float min_r(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double min_r(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float abs_r(float a) { return fabsf(a); }
__device__ __forceinline__ double abs_r(double a) { return fabs(a); }
__device__ __forceinline__ float copysign_r(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ double copysign_r(double a, double b) { return copysign(a, b); }
__device__ __forceinline__ float hypot_r(float a, float b) { return hypotf(a, b); }
__device__ __forceinline__ double hypot_r(double a, double b) { return hypot(a, b); }

// element size in bytes of a precision code (GBRI_F32 / GBRI_F64)
inline size_t real_bytes(int prec) { return prec == GBRI_F64 ? 8 : 4; }

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
