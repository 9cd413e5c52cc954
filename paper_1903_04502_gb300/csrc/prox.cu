// Proximal operators of Sec. 4: soft thresholding (Sec. 4.3) and the projection
// onto an l2 ball centred at c (Sec. 4.2, the translated ball prox; the global
// constraint of Sec. 6.8 on one GPU).  The ball norm is a two-level reduction:
// per-thread compensated FP32 partial sums of |z - c|^2, FP64 block sums, and a
// fixed-order FP64 sum of the block partials (deterministic).
#include "prox.cuh"

namespace gbri {

namespace {

// soft thresholding with threshold lam (w null) or lam * w[i]
template <class R>
__global__ void k_soft_real(const R* __restrict__ in, const R* __restrict__ w, R* __restrict__ out, int64_t n,
                            R lam) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const R v = in[i];
    const R a = abs_r(v) - (w ? lam * w[i] : lam);
    out[i] = a > 0 ? copysign_r(a, v) : (R)0;
  }
}

template <class R>
__global__ void k_soft_complex(const cplx<R>* __restrict__ in, const R* __restrict__ w, cplx<R>* __restrict__ out,
                               int64_t n, R lam) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> v = in[i];
    const R t = w ? lam * w[i] : lam;
    const R mag = hypot_r(v.x, v.y);
    const R s = mag > t ? (mag - t) / mag : (R)0;
    out[i] = mkc<R>(v.x * s, v.y * s);
  }
}

template <class R>
__global__ void k_l2dist_partials(const cplx<R>* __restrict__ z, const cplx<R>* __restrict__ c, int64_t M,
                                  double* __restrict__ partials) {
  __shared__ double sh[40];
  acc_t<R> acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> a = z[i], b = c[i];
    const R dr = a.x - b.x, di = a.y - b.y;
    acc.add(fma_r(dr, dr, di * di));
  }
  const double v = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// z and out may be the same vector (in-place projection): neither is declared __restrict__;
// each thread reads element i of z and c before it writes element i of out.
template <class R>
__global__ void k_l2ball_apply(const cplx<R>* z, const cplx<R>* __restrict__ c, cplx<R>* out,
                               int64_t M, double eps, const double* __restrict__ partials, int n_partials,
                               double* __restrict__ norm_out) {
  __shared__ double sh[40];
  const double nrm = sqrt(reduce_partials(partials, n_partials, sh));
  if (blockIdx.x == 0 && threadIdx.x == 0 && norm_out) *norm_out = nrm;
  const R sc = (nrm > eps) ? (R)(eps / nrm) : (R)1;
  if (sc == (R)1 && out == z) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> a = z[i], b = c[i];
    out[i] = (nrm > eps) ? mkc<R>(fma_r(sc, a.x - b.x, b.x), fma_r(sc, a.y - b.y, b.y)) : a;
  }
}

template <class R>
int32_t prox_l1(const void* d_in, const void* d_w, void* d_out, int64_t n, double lambda, int32_t is_complex,
                cudaStream_t s) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8));
  launch_begin(GBRI_K_OTHER, s);
  if (is_complex)
    k_soft_complex<R><<<blocks, 256, 0, s>>>(static_cast<const cplx<R>*>(d_in), static_cast<const R*>(d_w),
                                             static_cast<cplx<R>*>(d_out), n, (R)lambda);
  else
    k_soft_real<R><<<blocks, 256, 0, s>>>(static_cast<const R*>(d_in), static_cast<const R*>(d_w),
                                          static_cast<R*>(d_out), n, (R)lambda);
  return launch_end(GBRI_K_OTHER, s);
}

template <class R>
int32_t proj_l2ball_alloc(const void* d_z, const void* d_center, void* d_out, int64_t M, double eps,
                          double* d_norm_out, cudaStream_t s) {
  const int n_partials = l2ball_blocks(M);
  double* partials = nullptr;
  GBRI_CHECK_CUDA(cudaMallocAsync((void**)&partials, sizeof(double) * n_partials, s));
  const int32_t st = proj_l2ball_with_scratch<R>(static_cast<const R*>(d_z), static_cast<const R*>(d_center),
                                                 static_cast<R*>(d_out), M, eps, d_norm_out, partials, n_partials, s);
  cudaFreeAsync(partials, s);
  return st;
}

}  // namespace

int l2ball_blocks(int64_t M) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(M, 256 * 8), (int64_t)num_sms() * 4));
}

template <class R>
int32_t proj_l2ball_with_scratch(const R* d_z, const R* d_center, R* d_out, int64_t M, double eps,
                                 double* d_norm_out, double* partials, int n_partials, cudaStream_t s) {
  using C = cplx<R>;
  const int blocks = std::min(l2ball_blocks(M), n_partials);
  launch_begin(GBRI_K_OTHER, s);
  k_l2dist_partials<R><<<blocks, 256, 0, s>>>((const C*)d_z, (const C*)d_center, M, partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  launch_begin(GBRI_K_OTHER, s);
  k_l2ball_apply<R><<<blocks, 256, 0, s>>>((const C*)d_z, (const C*)d_center, (C*)d_out, M, eps, partials, blocks,
                                           d_norm_out);
  return launch_end(GBRI_K_OTHER, s);
}

template int32_t proj_l2ball_with_scratch<float>(const float*, const float*, float*, int64_t, double, double*,
                                                 double*, int, cudaStream_t);
template int32_t proj_l2ball_with_scratch<double>(const double*, const double*, double*, int64_t, double, double*,
                                                  double*, int, cudaStream_t);

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_prox_l1(const void* d_in, void* d_out, int64_t n, double lambda, int32_t is_complex, int32_t precision,
                     void* stream) {
  GBRI_CHECK(precision == GBRI_F32 || precision == GBRI_F64, GBRI_EINVAL, "precision must be GBRI_F32 or GBRI_F64");
  GBRI_CHECK(n >= 0 && lambda >= 0, GBRI_EINVAL, "bad size or lambda");
  if (n == 0) return GBRI_OK;
  GBRI_CHECK(d_in && d_out, GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return precision == GBRI_F64 ? prox_l1<double>(d_in, nullptr, d_out, n, lambda, is_complex, s)
                               : prox_l1<float>(d_in, nullptr, d_out, n, lambda, is_complex, s);
}

int32_t gbri_prox_l1_weighted(const void* d_in, const void* d_w, void* d_out, int64_t n, double lambda,
                              int32_t is_complex, int32_t precision, void* stream) {
  GBRI_CHECK(precision == GBRI_F32 || precision == GBRI_F64, GBRI_EINVAL, "precision must be GBRI_F32 or GBRI_F64");
  GBRI_CHECK(n >= 0 && lambda >= 0, GBRI_EINVAL, "bad size or lambda");
  if (n == 0) return GBRI_OK;
  GBRI_CHECK(d_in && d_out && d_w, GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return precision == GBRI_F64 ? prox_l1<double>(d_in, d_w, d_out, n, lambda, is_complex, s)
                               : prox_l1<float>(d_in, d_w, d_out, n, lambda, is_complex, s);
}

int32_t gbri_proj_l2ball(const void* d_z, const void* d_center, void* d_out, int64_t M, double eps,
                         double* d_norm_out, int32_t precision, void* stream) {
  GBRI_CHECK(precision == GBRI_F32 || precision == GBRI_F64, GBRI_EINVAL, "precision must be GBRI_F32 or GBRI_F64");
  GBRI_CHECK(M >= 0 && eps >= 0, GBRI_EINVAL, "bad size or eps");
  GBRI_CHECK(M == 0 || (d_z && d_center && d_out), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return precision == GBRI_F64 ? proj_l2ball_alloc<double>(d_z, d_center, d_out, M, eps, d_norm_out, s)
                               : proj_l2ball_alloc<float>(d_z, d_center, d_out, M, eps, d_norm_out, s);
}

}  // extern "C"
