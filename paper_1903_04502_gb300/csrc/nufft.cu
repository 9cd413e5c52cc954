// Measurement operator calls: Phi (Sec. 2, Eq. 2) = degrid(F(pad_correct(x))),
// Phi^dagger = crop_correct(F^H(grid(y))), visibility reordering and the power
// method for ||Phi||^2 (Sec. 6.3.1).
#include <cmath>
#include <cstdint>
#include <vector>

#include "nufft.cuh"

namespace gbri {

namespace {

// Z S: padded[(q - n/2) mod K][(p - n/2) mod K] = corr[p] corr[q] x[q][p] / *d_norm (real;
// the other cells stay zero from plan creation).  A thread takes V consecutive pixels of
// one row: V = 4 on the FP32 path when n % 8 == 0 (no group straddles the wrap at column
// n/2; all vector accesses 16-byte aligned), else V = 1.
template <class R, int V>
__global__ void k_pad(const R* __restrict__ x, const R* __restrict__ corr, R* __restrict__ padded, int n,
                      int K, const double* __restrict__ d_norm) {
  static_assert(V == 1 || (V == 4 && sizeof(R) == 4), "vector path is FP32 only");
  const R s = d_norm ? (R)(1.0 / *d_norm) : (R)1;
  const int groups = n * n / V;
  for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < groups; gi += gridDim.x * blockDim.x) {
    const int i = gi * V;
    const int q = i / n, p = i - q * n;
    int r = q - n / 2; if (r < 0) r += K;
    int c = p - n / 2; if (c < 0) c += K;
    const R cq = corr[q];
    if constexpr (V == 4) {
      const float4 x4 = *reinterpret_cast<const float4*>(x + i);
      const float4 c4 = *reinterpret_cast<const float4*>(corr + p);
      *reinterpret_cast<float4*>(padded + (size_t)r * K + c) =
          make_float4(x4.x * c4.x * cq * s, x4.y * c4.y * cq * s, x4.z * c4.z * cq * s, x4.w * c4.w * cq * s);
    } else {
      padded[(size_t)r * K + c] = x[i] * corr[p] * cq * s;
    }
  }
}

// S^T Z^T and the real part: x[q][p] = corr[p] corr[q] Re(grid[(q - n/2) mod K][(p - n/2) mod K])
// The Hermitian part of the grid on the half plane kx = 0 .. K/2 (the layout of a
// real-to-complex transform): spec[ky][kx] = (grid[ky][kx] + conj(grid[-ky][-kx])) / 2,
// indices mod K.  Its complex-to-real inverse is the real part of the grid's inverse
// transform: the transform of conj(G(-k)) is the conjugate of that of G(k).  One thread per
// half-plane element, rows after rows.
template <class R>
__global__ void k_herm_fold(const cplx<R>* __restrict__ grid, cplx<R>* __restrict__ spec, int K) {
  const int H = K / 2 + 1;
  const int64_t total = (int64_t)K * H;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int ky = (int)(e / H), kx = (int)(e - (int64_t)ky * H);
    const int my = ky == 0 ? 0 : K - ky, mx = kx == 0 ? 0 : K - kx;
    const cplx<R> a = grid[(size_t)ky * K + kx], b = grid[(size_t)my * K + mx];
    cplx<R> h;
    h.x = (R)0.5 * (a.x + b.x);
    h.y = (R)0.5 * (a.y - b.y);
    spec[e] = h;
  }
}

// S^T Z^T of img = Re(F^H grid) (real [K][K], from the complex-to-real inverse) with the
// correction: x[q][p] = corr[p] corr[q] img[(q - n/2) mod K][(p - n/2) mod K].
template <class R>
__global__ void k_crop(const R* __restrict__ img, const R* __restrict__ corr, R* __restrict__ x, int n, int K) {
  const int total = n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int q = i / n, p = i - q * n;
    int r = q - n / 2; if (r < 0) r += K;
    int c = p - n / 2; if (c < 0) c += K;
    x[i] = corr[p] * corr[q] * img[(size_t)r * K + c];
  }
}

template <class T>
__global__ void k_gather(const T* __restrict__ in, const int32_t* __restrict__ perm, T* __restrict__ out, int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
template <class T>
__global__ void k_scatter_vis(const T* __restrict__ in, const int32_t* __restrict__ perm, T* __restrict__ out,
                              int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}

// FP64 sum of squares of an image into partials[blockIdx.x] (FP32 path: per-thread
// compensated FP32 partials; FP64 path: FP64 throughout).
template <class R>
__global__ void k_image_sumsq(const R* __restrict__ x, int64_t n, double* __restrict__ partials) {
  __shared__ double sh[40];
  acc_t<R> acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc.add(x[i] * x[i]);
  const double v = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// norm = sqrt(sum partials) into out[0]
__global__ void k_finish_norm(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double sh[40];
  const double v = reduce_partials(partials, n, sh);
  if (threadIdx.x == 0) out[0] = sqrt(v);
}

// start vector of the power method: 0.5 + U[0,1), U = top 53 bits of SplitMix64(seed + k golden), k = i + 1
template <class R>
__global__ void k_power_start(R* __restrict__ b, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    b[i] = (R)(0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0));
  }
}

int grid_blocks_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 8));
}

}  // namespace

template <class R>
int32_t launch_pad(gbri_plan* p, const R* x, const double* d_norm, cudaStream_t s) {
  const int64_t N = (int64_t)p->n_side * p->n_side;
  // the vector path also needs x 16-byte aligned (a caller's image may be an offset view)
  const bool v4 = sizeof(R) == 4 && p->n_side % 8 == 0 && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
  launch_begin(GBRI_K_PAD, s);
  if (v4)
    k_pad<R, (sizeof(R) == 4 ? 4 : 1)><<<grid_blocks_for(N / 4), 256, 0, s>>>(
        x, p->as<const R>(p->corr), p->as<R>(p->padded), p->n_side, p->K, d_norm);
  else
    k_pad<R, 1><<<grid_blocks_for(N), 256, 0, s>>>(x, p->as<const R>(p->corr), p->as<R>(p->padded), p->n_side,
                                                   p->K, d_norm);
  return launch_end(GBRI_K_PAD, s);
}

template <class R>
int32_t launch_crop(gbri_plan* p, R* x, cudaStream_t s) {
  launch_begin(GBRI_K_CROP, s);
  k_crop<R><<<grid_blocks_for((int64_t)p->n_side * p->n_side), 256, 0, s>>>(
      p->as<const R>(p->grid), p->as<const R>(p->corr), x, p->n_side, p->K);
  return launch_end(GBRI_K_CROP, s);
}

template int32_t launch_pad<float>(gbri_plan*, const float*, const double*, cudaStream_t);
template int32_t launch_pad<double>(gbri_plan*, const double*, const double*, cudaStream_t);
template int32_t launch_crop<float>(gbri_plan*, float*, cudaStream_t);
template int32_t launch_crop<double>(gbri_plan*, double*, cudaStream_t);

// F Z S x: real-to-complex, padded -> spec (the half kx = 0 .. K/2; degridding reads
// kx > K/2 as conj(spec[-ky][K - kx]))
int32_t fft_forward(gbri_plan* p, cudaStream_t s) {
  if (cufftSetStream(p->fft_r2c, s) != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftSetStream");
  launch_begin(GBRI_K_FFT_FWD, s, false);
  const cufftResult r =
      p->prec == GBRI_F64
          ? cufftExecD2Z(p->fft_r2c, p->as<cufftDoubleReal>(p->padded), p->as<cufftDoubleComplex>(p->spec))
          : cufftExecR2C(p->fft_r2c, p->as<cufftReal>(p->padded), p->as<cufftComplex>(p->spec));
  const int32_t st = launch_end(GBRI_K_FFT_FWD, s);
  if (r != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cuFFT forward");
  return st;
}

int32_t fft_inverse_real(gbri_plan* p, cudaStream_t s) {
  if (cufftSetStream(p->fft_c2r, s) != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftSetStream");
  const int64_t total = (int64_t)p->K * (p->K / 2 + 1);
  const int blocks = (int)std::min<int64_t>(ceil_div(total, 256), (int64_t)num_sms() * 16);
  launch_begin(GBRI_K_FFT_INV, s);
  cufftResult r;
  if (p->prec == GBRI_F64) {
    k_herm_fold<double><<<blocks, 256, 0, s>>>(p->as<const cplx<double>>(p->grid), p->as<cplx<double>>(p->spec),
                                                p->K);
    r = cufftExecZ2D(p->fft_c2r, p->as<cufftDoubleComplex>(p->spec), p->as<cufftDoubleReal>(p->grid));
  } else {
    k_herm_fold<float><<<blocks, 256, 0, s>>>(p->as<const cplx<float>>(p->grid), p->as<cplx<float>>(p->spec), p->K);
    r = cufftExecC2R(p->fft_c2r, p->as<cufftComplex>(p->spec), p->as<cufftReal>(p->grid));
  }
  const int32_t st = launch_end(GBRI_K_FFT_INV, s);
  if (r != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cuFFT complex-to-real inverse");
  return st;
}

namespace {

// Phi^dagger Phi b for the power method: b (image) -> out (image), plan-order scratch.
template <class R>
int32_t normal_op(gbri_plan* p, const R* b, const double* d_norm, R* out, cudaStream_t s) {
  GBRI_TRY(launch_pad<R>(p, b, d_norm, s));
  GBRI_TRY(fft_forward(p, s));
  GBRI_TRY(launch_degrid(p, EpiStorePlan<R>{p->as<cplx<R>>(p->vis_tmp)}, s));
  GBRI_TRY(launch_grid(p, SrcPlan<R>{p->as<const cplx<R>>(p->vis_tmp)}, s));
  GBRI_TRY(fft_inverse_real(p, s));
  return launch_crop<R>(p, out, s);
}

template <class R>
int32_t image_norm(gbri_plan* p, const R* x, double* d_out, cudaStream_t s) {
  const int64_t n = (int64_t)p->n_side * p->n_side;
  const int blocks = std::min(grid_blocks_for(n), p->n_partials);
  launch_begin(GBRI_K_OTHER, s);
  k_image_sumsq<R><<<blocks, 256, 0, s>>>(x, n, p->partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  launch_begin(GBRI_K_OTHER, s);
  k_finish_norm<<<1, 256, 0, s>>>(p->partials, blocks, d_out);
  return launch_end(GBRI_K_OTHER, s);
}

template <class R>
int32_t vis_reorder(const gbri_plan* p, const void* d_in, void* d_out, int32_t to_plan, cudaStream_t s) {
  using C = cplx<R>;
  launch_begin(GBRI_K_OTHER, s);
  if (to_plan)
    k_gather<C><<<grid_blocks_for(p->M), 256, 0, s>>>(static_cast<const C*>(d_in), p->perm, static_cast<C*>(d_out),
                                                      p->M);
  else
    k_scatter_vis<C><<<grid_blocks_for(p->M), 256, 0, s>>>(static_cast<const C*>(d_in), p->perm,
                                                           static_cast<C*>(d_out), p->M);
  return launch_end(GBRI_K_OTHER, s);
}

template <class R>
int32_t phi(gbri_plan* p, const void* d_x, void* d_y, uint32_t flags, cudaStream_t s) {
  GBRI_TRY(launch_pad<R>(p, static_cast<const R*>(d_x), nullptr, s));
  GBRI_TRY(fft_forward(p, s));
  if (p->M == 0) return GBRI_OK;
  cplx<R>* y = static_cast<cplx<R>*>(d_y);
  if (flags & GBRI_PLAN_ORDER) return launch_degrid(p, EpiStorePlan<R>{y}, s);
  return launch_degrid(p, EpiStoreRaw<R>{y, p->perm}, s);
}

template <class R>
int32_t phi_adjoint(gbri_plan* p, const void* d_y, void* d_x, uint32_t flags, cudaStream_t s) {
  const cplx<R>* y = static_cast<const cplx<R>*>(d_y);
  if (flags & GBRI_PLAN_ORDER)
    GBRI_TRY(launch_grid(p, SrcPlan<R>{y}, s));
  else
    GBRI_TRY(launch_grid(p, SrcRaw<R>{y, p->perm}, s));
  GBRI_TRY(fft_inverse_real(p, s));
  return launch_crop<R>(p, static_cast<R*>(d_x), s);
}

template <class R>
int32_t op_norm(gbri_plan* p, int32_t max_iter, double tol, uint64_t seed, double* op_norm_sq, int32_t* iters,
                cudaStream_t s) {
  const int64_t n = (int64_t)p->n_side * p->n_side;
  R *b = nullptr, *c = nullptr;
  double* d_norm = p->scalars + 8;  // scalars[8]: norm of the current vector
  GBRI_CHECK_CUDA(cudaMallocAsync((void**)&b, sizeof(R) * n, s));
  cudaError_t e = cudaMallocAsync((void**)&c, sizeof(R) * n, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(b, s);
    return cuda_error(e, "cudaMallocAsync");
  }
  int32_t st = GBRI_OK;
  launch_begin(GBRI_K_OTHER, s);
  k_power_start<R><<<grid_blocks_for(n), 256, 0, s>>>(b, n, seed);
  st = launch_end(GBRI_K_OTHER, s);
  if (st == GBRI_OK) st = image_norm<R>(p, b, d_norm, s);
  double prev = 0.0, val = 0.0;
  int it = 0;
  for (it = 1; it <= max_iter && st == GBRI_OK; ++it) {
    // c = Phi^dagger Phi (b / ||b||), then ||c||
    st = normal_op<R>(p, b, d_norm, c, s);
    if (st != GBRI_OK) break;
    st = image_norm<R>(p, c, d_norm, s);
    if (st != GBRI_OK) break;
    e = cudaMemcpyAsync(&val, d_norm, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "power iteration");
      break;
    }
    std::swap(b, c);
    if (it > 1 && std::fabs(val - prev) <= tol * val) break;
    prev = val;
  }
  cudaFreeAsync(b, s);
  cudaFreeAsync(c, s);
  if (st != GBRI_OK) return st;
  *op_norm_sq = val;
  if (iters) *iters = std::min(it, max_iter);
  return GBRI_OK;
}

}  // namespace

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_vis_reorder(const gbri_plan* p, const void* d_in, void* d_out, int32_t to_plan, void* stream) {
  GBRI_CHECK(p, GBRI_EINVAL, "null plan");
  if (p->M == 0) return GBRI_OK;
  GBRI_CHECK(d_in && d_out && d_in != d_out, GBRI_EINVAL, "bad buffers");
  cudaStream_t s = (cudaStream_t)stream;
  return p->prec == GBRI_F64 ? vis_reorder<double>(p, d_in, d_out, to_plan, s)
                             : vis_reorder<float>(p, d_in, d_out, to_plan, s);
}

int32_t gbri_phi(gbri_plan* p, const void* d_x, void* d_y, uint32_t flags, void* stream) {
  GBRI_CHECK(p && d_x && (d_y || p->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return p->prec == GBRI_F64 ? phi<double>(p, d_x, d_y, flags, s) : phi<float>(p, d_x, d_y, flags, s);
}

int32_t gbri_phi_adjoint(gbri_plan* p, const void* d_y, void* d_x, uint32_t flags, void* stream) {
  GBRI_CHECK(p && d_x && (d_y || p->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  return p->prec == GBRI_F64 ? phi_adjoint<double>(p, d_y, d_x, flags, s) : phi_adjoint<float>(p, d_y, d_x, flags, s);
}

int32_t gbri_op_norm(gbri_plan* p, int32_t max_iter, double tol, uint64_t seed, double* op_norm_sq,
                     int32_t* iters, void* stream) {
  GBRI_CHECK(p && op_norm_sq && max_iter > 0, GBRI_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  return p->prec == GBRI_F64 ? op_norm<double>(p, max_iter, tol, seed, op_norm_sq, iters, s)
                             : op_norm<float>(p, max_iter, tol, seed, op_norm_sq, iters, s);
}

}  // extern "C"
