// Non-coplanar measurement operator by w-stacking (reading R14; the wide-field method the
// paper's software offers, Sec. 7.1).  The visibilities are binned by w into n_planes equal
// bins; plane k holds a coplanar plan (Sec. 2, Eq. 2) over its visibilities, and the image is
// multiplied by the plane's screen C_k = exp(-2 pi i w_k (n - 1)) before it:
//   (Phi x)_{i in plane k} = (Phi_k (C_k x))_i,   Phi^dagger y = Re sum_k conj(C_k) Phi_k^dagger y_k.
// The screen makes the plane's input image complex; the coplanar plans take real images, so
// with x_c = Re(C_k) x and x_s = Im(C_k) x (both real) Phi_k(C_k x) = Phi_k x_c + i Phi_k x_s
// (Phi_k is complex-linear), and with A = the adjoint before its real part,
// Re(conj(C_k) A y) = Re(C_k) Re(A y) + Im(C_k) Re(A (-i y)), i.e. two real adjoints.  Every
// plane therefore costs two coplanar applications; the screens are computed once in FP64 and
// stored in the plan's precision.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "nufft.cuh"

struct gbri_wstack {
  int n_side = 0, n_planes = 0, prec = 0;
  double delta = 0.0, w_lo = 0.0, dw = 0.0;
  int64_t M = 0;
  std::vector<gbri_plan*> plans;      // per plane (null when the plane is empty)
  std::vector<int64_t> counts;        // visibilities per plane
  std::vector<double> centres;        // w_k
  std::vector<int32_t*> idx;          // per plane: caller indices of its visibilities [counts[k]]
  std::vector<void*> scr_re, scr_im;  // per plane: Re C_k, Im C_k [n][n] (plan precision)
  void* xt = nullptr;                 // R [n][n] screened image / adjoint term
  void* z2 = nullptr;                 // R [n][n] second adjoint term
  void* ya = nullptr;                 // C [max count]
  void* yb = nullptr;                 // C [max count]
};

namespace gbri {
namespace {

template <class R>
__global__ void k_ws_mul(const R* __restrict__ a, const R* __restrict__ x, R* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * x[i];
}

// y[idx[j]] = yc[j] + i ys[j]
template <class R>
__global__ void k_ws_combine(const cplx<R>* __restrict__ yc, const cplx<R>* __restrict__ ys,
                             const int32_t* __restrict__ idx, cplx<R>* __restrict__ y, int64_t m) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> a = yc[j], b = ys[j];
    y[idx[j]] = mkc<R>(a.x - b.y, a.y + b.x);
  }
}

// ya[j] = y[idx[j]], yb[j] = -i y[idx[j]]
template <class R>
__global__ void k_ws_gather(const cplx<R>* __restrict__ y, const int32_t* __restrict__ idx, cplx<R>* __restrict__ ya,
                            cplx<R>* __restrict__ yb, int64_t m) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
    const cplx<R> v = y[idx[j]];
    ya[j] = v;
    yb[j] = mkc<R>(v.y, -v.x);
  }
}

// x += Re(C) z1 + Im(C) z2
template <class R>
__global__ void k_ws_accum(const R* __restrict__ cr, const R* __restrict__ ci, const R* __restrict__ z1,
                           const R* __restrict__ z2, R* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += cr[i] * z1[i] + ci[i] * z2[i];
}

int ws_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8)); }

void free_ws(gbri_wstack* w) {
  if (!w) return;
  for (gbri_plan* p : w->plans)
    if (p) gbri_plan_destroy(p);
  for (int32_t* i : w->idx) cudaFree(i);
  for (void* q : w->scr_re) cudaFree(q);
  for (void* q : w->scr_im) cudaFree(q);
  cudaFree(w->xt);
  cudaFree(w->z2);
  cudaFree(w->ya);
  cudaFree(w->yb);
  delete w;
}

int32_t ws_malloc(void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (alloc_fault_injected() || cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    return set_error(GBRI_ENOMEM, "cudaMalloc (w-stacking)");
  }
  return GBRI_OK;
}

template <class R>
int32_t ws_phi(gbri_wstack* w, const R* x, cplx<R>* y, cudaStream_t s) {
  const int64_t N = (int64_t)w->n_side * w->n_side;
  cplx<R>* ya = static_cast<cplx<R>*>(w->ya);
  cplx<R>* yb = static_cast<cplx<R>*>(w->yb);
  R* xt = static_cast<R*>(w->xt);
  for (int k = 0; k < w->n_planes; ++k) {
    const int64_t m = w->counts[k];
    if (m == 0) continue;
    launch_begin(GBRI_K_OTHER, s);
    k_ws_mul<R><<<ws_blocks(N), 256, 0, s>>>(static_cast<const R*>(w->scr_re[k]), x, xt, N);
    GBRI_TRY(launch_end(GBRI_K_OTHER, s));
    GBRI_TRY(gbri_phi(w->plans[k], xt, ya, 0, s));
    launch_begin(GBRI_K_OTHER, s);
    k_ws_mul<R><<<ws_blocks(N), 256, 0, s>>>(static_cast<const R*>(w->scr_im[k]), x, xt, N);
    GBRI_TRY(launch_end(GBRI_K_OTHER, s));
    GBRI_TRY(gbri_phi(w->plans[k], xt, yb, 0, s));
    launch_begin(GBRI_K_OTHER, s);
    k_ws_combine<R><<<ws_blocks(m), 256, 0, s>>>(ya, yb, w->idx[k], y, m);
    GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  }
  return GBRI_OK;
}

template <class R>
int32_t ws_phi_adjoint(gbri_wstack* w, const cplx<R>* y, R* x, cudaStream_t s) {
  const int64_t N = (int64_t)w->n_side * w->n_side;
  cplx<R>* ya = static_cast<cplx<R>*>(w->ya);
  cplx<R>* yb = static_cast<cplx<R>*>(w->yb);
  R* z1 = static_cast<R*>(w->xt);
  R* z2 = static_cast<R*>(w->z2);
  GBRI_CHECK_CUDA(cudaMemsetAsync(x, 0, sizeof(R) * (size_t)N, s));
  for (int k = 0; k < w->n_planes; ++k) {
    const int64_t m = w->counts[k];
    if (m == 0) continue;
    launch_begin(GBRI_K_OTHER, s);
    k_ws_gather<R><<<ws_blocks(m), 256, 0, s>>>(y, w->idx[k], ya, yb, m);
    GBRI_TRY(launch_end(GBRI_K_OTHER, s));
    GBRI_TRY(gbri_phi_adjoint(w->plans[k], ya, z1, 0, s));
    GBRI_TRY(gbri_phi_adjoint(w->plans[k], yb, z2, 0, s));
    launch_begin(GBRI_K_OTHER, s);
    k_ws_accum<R><<<ws_blocks(N), 256, 0, s>>>(static_cast<const R*>(w->scr_re[k]),
                                               static_cast<const R*>(w->scr_im[k]), z1, z2, x, N);
    GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  }
  return GBRI_OK;
}

int32_t build_ws(gbri_wstack* w, const gbri_plan_desc* d, const float* d_uvw, cudaStream_t s) {
  const int64_t M = w->M;
  const int n = w->n_side;
  std::vector<float> h((size_t)M * 4);
  if (M > 0) {
    GBRI_CHECK_CUDA(cudaMemcpyAsync(h.data(), d_uvw, sizeof(float) * 4 * (size_t)M, cudaMemcpyDeviceToHost, s));
    GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  // bins in FP64: [w_lo, w_hi] cut into n_planes equal parts, the last one closed
  double lo = 0.0, hi = 0.0;
  for (int64_t i = 0; i < M; ++i) {
    const double wi = h[(size_t)i * 4 + 2];
    GBRI_CHECK(std::isfinite(wi), GBRI_ENONFINITE, "non-finite w");
    if (i == 0 || wi < lo) lo = wi;
    if (i == 0 || wi > hi) hi = wi;
  }
  const int P = w->n_planes;
  w->w_lo = lo;
  w->dw = hi > lo ? (hi - lo) / P : 0.0;
  std::vector<int> plane((size_t)M, 0);
  w->counts.assign(P, 0);
  for (int64_t i = 0; i < M; ++i) {
    int k = 0;
    if (w->dw > 0.0) k = std::min(P - 1, (int)std::floor(((double)h[(size_t)i * 4 + 2] - lo) / w->dw));
    plane[i] = k;
    ++w->counts[k];
  }
  w->centres.resize(P);
  for (int k = 0; k < P; ++k) w->centres[k] = w->dw > 0.0 ? lo + (k + 0.5) * w->dw : lo;
  // n - 1 on the image grid (l = p' delta along columns, m = q' delta along rows)
  std::vector<double> nm1((size_t)n * n);
  for (int q = 0; q < n; ++q)
    for (int p = 0; p < n; ++p) {
      const double l = (p - n / 2) * w->delta, m = (q - n / 2) * w->delta;
      const double r2 = l * l + m * m;
      GBRI_CHECK(r2 < 1.0, GBRI_EINVAL, "field of view beyond the horizon: reduce pixel_size");
      nm1[(size_t)q * n + p] = std::sqrt(1.0 - r2) - 1.0;
    }
  const size_t rb = real_bytes(w->prec);
  w->plans.assign(P, nullptr);
  w->idx.assign(P, nullptr);
  w->scr_re.assign(P, nullptr);
  w->scr_im.assign(P, nullptr);
  int64_t maxm = 1;
  std::vector<float> sub;
  std::vector<int32_t> ix;
  for (int k = 0; k < P; ++k) {
    const int64_t m = w->counts[k];
    maxm = std::max(maxm, m);
    // screen C_k = exp(-2 pi i w_k (n - 1)): Re = cos(phi), Im = -sin(phi), phi = 2 pi w_k (n - 1)
    std::vector<double> cr((size_t)n * n), ci((size_t)n * n);
    for (size_t i = 0; i < cr.size(); ++i) {
      const double ph = 2.0 * M_PI * w->centres[k] * nm1[i];
      cr[i] = std::cos(ph);
      ci[i] = -std::sin(ph);
    }
    GBRI_TRY(ws_malloc(&w->scr_re[k], rb * cr.size()));
    GBRI_TRY(ws_malloc(&w->scr_im[k], rb * ci.size()));
    if (w->prec == GBRI_F64) {
      GBRI_CHECK_CUDA(cudaMemcpyAsync(w->scr_re[k], cr.data(), rb * cr.size(), cudaMemcpyHostToDevice, s));
      GBRI_CHECK_CUDA(cudaMemcpyAsync(w->scr_im[k], ci.data(), rb * ci.size(), cudaMemcpyHostToDevice, s));
      GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
    } else {
      std::vector<float> fr(cr.begin(), cr.end()), fi(ci.begin(), ci.end());
      GBRI_CHECK_CUDA(cudaMemcpyAsync(w->scr_re[k], fr.data(), rb * fr.size(), cudaMemcpyHostToDevice, s));
      GBRI_CHECK_CUDA(cudaMemcpyAsync(w->scr_im[k], fi.data(), rb * fi.size(), cudaMemcpyHostToDevice, s));
      GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    if (m == 0) continue;
    // the plane's rows (caller order within the plane) and their caller indices
    sub.resize((size_t)m * 4);
    ix.resize((size_t)m);
    int64_t j = 0;
    for (int64_t i = 0; i < M; ++i)
      if (plane[i] == k) {
        std::copy(&h[(size_t)i * 4], &h[(size_t)i * 4] + 4, &sub[(size_t)j * 4]);
        ix[j++] = (int32_t)i;
      }
    void* dsub = nullptr;
    GBRI_TRY(ws_malloc((void**)&w->idx[k], sizeof(int32_t) * (size_t)m));
    GBRI_TRY(ws_malloc(&dsub, sizeof(float) * 4 * (size_t)m));
    cudaError_t e = cudaMemcpyAsync(dsub, sub.data(), sizeof(float) * 4 * (size_t)m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(w->idx[k], ix.data(), sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaFree(dsub);
      return cuda_error(e, "cudaMemcpyAsync (w-stacking planes)");
    }
    gbri_plan_desc pd = *d;
    pd.M = m;
    const int32_t st = gbri_plan_create(&w->plans[k], &pd, static_cast<const float*>(dsub), s);
    cudaFree(dsub);
    if (st != GBRI_OK) return st;
  }
  GBRI_TRY(ws_malloc(&w->xt, rb * (size_t)n * n));
  GBRI_TRY(ws_malloc(&w->z2, rb * (size_t)n * n));
  GBRI_TRY(ws_malloc(&w->ya, 2 * rb * (size_t)maxm));
  GBRI_TRY(ws_malloc(&w->yb, 2 * rb * (size_t)maxm));
  return GBRI_OK;
}

}  // namespace
}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_wstack_create(gbri_wstack** out, const gbri_plan_desc* desc, const float* d_uvw_weight,
                           int32_t n_planes, double pixel_size, void* stream) {
  GBRI_CHECK(out && desc, GBRI_EINVAL, "null argument");
  *out = nullptr;
  GBRI_CHECK(n_planes >= 1 && n_planes <= 4096, GBRI_EINVAL, "n_planes must be in [1, 4096]");
  GBRI_CHECK(pixel_size > 0.0 && std::isfinite(pixel_size), GBRI_EINVAL, "pixel_size must be positive");
  GBRI_CHECK(desc->M >= 0 && desc->M < (int64_t)1 << 31, GBRI_EINVAL, "M must be in [0, 2^31)");
  GBRI_CHECK(desc->M == 0 || d_uvw_weight, GBRI_EINVAL, "null uvw");
  GBRI_CHECK(desc->n_side >= 16 && desc->n_side % 2 == 0, GBRI_EINVAL, "n_side must be even and >= 16");
  GBRI_CHECK(desc->precision == GBRI_F32 || desc->precision == GBRI_F64, GBRI_EINVAL,
             "precision must be GBRI_F32 or GBRI_F64");
  gbri_wstack* w = new (std::nothrow) gbri_wstack();
  GBRI_CHECK(w, GBRI_ENOMEM, "host allocation");
  w->n_side = desc->n_side;
  w->n_planes = n_planes;
  w->prec = desc->precision;
  w->delta = pixel_size;
  w->M = desc->M;
  const int32_t st = build_ws(w, desc, d_uvw_weight, (cudaStream_t)stream);
  if (st != GBRI_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    free_ws(w);
    return st;
  }
  *out = w;
  return GBRI_OK;
}

int32_t gbri_wstack_destroy(gbri_wstack* w) {
  if (w) cudaDeviceSynchronize();
  free_ws(w);
  return GBRI_OK;
}

int32_t gbri_wstack_info(const gbri_wstack* w, int32_t* n_planes, int64_t* counts, double* centres) {
  GBRI_CHECK(w, GBRI_EINVAL, "null argument");
  if (n_planes) *n_planes = w->n_planes;
  for (int k = 0; k < w->n_planes; ++k) {
    if (counts) counts[k] = w->counts[k];
    if (centres) centres[k] = w->centres[k];
  }
  return GBRI_OK;
}

int32_t gbri_wstack_phi(gbri_wstack* w, const void* d_x, void* d_y, void* stream) {
  GBRI_CHECK(w && d_x && (d_y || w->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (w->prec == GBRI_F64) return ws_phi<double>(w, static_cast<const double*>(d_x), static_cast<double2*>(d_y), s);
  return ws_phi<float>(w, static_cast<const float*>(d_x), static_cast<float2*>(d_y), s);
}

int32_t gbri_wstack_phi_adjoint(gbri_wstack* w, const void* d_y, void* d_x, void* stream) {
  GBRI_CHECK(w && d_x && (d_y || w->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (w->prec == GBRI_F64)
    return ws_phi_adjoint<double>(w, static_cast<const double2*>(d_y), static_cast<double*>(d_x), s);
  return ws_phi_adjoint<float>(w, static_cast<const float2*>(d_y), static_cast<float*>(d_x), s);
}

}  // extern "C"
