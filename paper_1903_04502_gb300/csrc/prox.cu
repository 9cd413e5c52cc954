// Proximal operators of Sec. 4: soft thresholding (Sec. 4.3) and the projection
// onto an l2 ball centred at c (Sec. 4.2, the translated ball prox; the global
// constraint of Sec. 6.8 on one GPU).  The ball norm is a two-level reduction:
// per-thread compensated FP32 partial sums of |z - c|^2, FP64 block sums, and a
// fixed-order FP64 sum of the block partials (deterministic).
#include "prox.cuh"

namespace gbri {

namespace {

__global__ void k_soft_real(const float* __restrict__ in, float* __restrict__ out, int64_t n, float lam) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = in[i];
    const float a = fabsf(v) - lam;
    out[i] = a > 0.f ? copysignf(a, v) : 0.f;
  }
}

__global__ void k_soft_complex(const float2* __restrict__ in, float2* __restrict__ out, int64_t n, float lam) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = in[i];
    const float mag = hypotf(v.x, v.y);
    const float s = mag > lam ? (mag - lam) / mag : 0.f;
    out[i] = make_float2(v.x * s, v.y * s);
  }
}

}  // namespace

__global__ void k_l2dist_partials(const float2* __restrict__ z, const float2* __restrict__ c, int64_t M,
                                  double* __restrict__ partials) {
  __shared__ double sh[40];
  KahanF acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = z[i], b = c[i];
    const float dr = a.x - b.x, di = a.y - b.y;
    acc.add(fmaf(dr, dr, di * di));
  }
  const double v = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void k_l2ball_apply(const float2* __restrict__ z, const float2* __restrict__ c, float2* __restrict__ out,
                               int64_t M, double eps, const double* __restrict__ partials, int n_partials,
                               double* __restrict__ norm_out) {
  __shared__ double sh[40];
  const double nrm = sqrt(reduce_partials(partials, n_partials, sh));
  if (blockIdx.x == 0 && threadIdx.x == 0 && norm_out) *norm_out = nrm;
  const float sc = (nrm > eps) ? (float)(eps / nrm) : 1.0f;
  if (sc == 1.0f && out == z) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = z[i], b = c[i];
    out[i] = (nrm > eps) ? make_float2(fmaf(sc, a.x - b.x, b.x), fmaf(sc, a.y - b.y, b.y)) : a;
  }
}

int l2ball_blocks(int64_t M) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M, 256 * 8), (int64_t)num_sms() * 4));
}

int32_t proj_l2ball_with_scratch(const float* d_z, const float* d_center, float* d_out, int64_t M, double eps,
                                 double* d_norm_out, double* partials, int n_partials, cudaStream_t s) {
  const int blocks = std::min(l2ball_blocks(M), n_partials);
  launch_begin(GBRI_K_OTHER, s);
  k_l2dist_partials<<<blocks, 256, 0, s>>>((const float2*)d_z, (const float2*)d_center, M, partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  launch_begin(GBRI_K_OTHER, s);
  k_l2ball_apply<<<blocks, 256, 0, s>>>((const float2*)d_z, (const float2*)d_center, (float2*)d_out, M, eps,
                                        partials, blocks, d_norm_out);
  return launch_end(GBRI_K_OTHER, s);
}

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_prox_l1(const float* d_in, float* d_out, int64_t n, double lambda, int32_t is_complex,
                     int32_t precision, void* stream) {
  GBRI_CHECK(precision == GBRI_F32, GBRI_EINVAL, "only GBRI_F32 is supported");
  GBRI_CHECK(n >= 0 && lambda >= 0, GBRI_EINVAL, "bad size or lambda");
  if (n == 0) return GBRI_OK;
  GBRI_CHECK(d_in && d_out, GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8));
  launch_begin(GBRI_K_OTHER, s);
  if (is_complex)
    k_soft_complex<<<blocks, 256, 0, s>>>((const float2*)d_in, (float2*)d_out, n, (float)lambda);
  else
    k_soft_real<<<blocks, 256, 0, s>>>(d_in, d_out, n, (float)lambda);
  return launch_end(GBRI_K_OTHER, s);
}

int32_t gbri_proj_l2ball(const float* d_z, const float* d_center, float* d_out, int64_t M, double eps,
                         double* d_norm_out, int32_t precision, void* stream) {
  GBRI_CHECK(precision == GBRI_F32, GBRI_EINVAL, "only GBRI_F32 is supported");
  GBRI_CHECK(M >= 0 && eps >= 0, GBRI_EINVAL, "bad size or eps");
  GBRI_CHECK(M == 0 || (d_z && d_center && d_out), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int n_partials = l2ball_blocks(M);
  double* partials = nullptr;
  GBRI_CHECK_CUDA(cudaMallocAsync((void**)&partials, sizeof(double) * n_partials, s));
  const int32_t st = proj_l2ball_with_scratch(d_z, d_center, d_out, M, eps, d_norm_out, partials, n_partials, s);
  cudaFreeAsync(partials, s);
  return st;
}

}  // extern "C"
