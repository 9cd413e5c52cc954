// SARA dictionary kernels: periodic 2-D Daubechies analysis (Psi^dagger) and
// synthesis (Psi), rows then columns per level, Mallat layout, batched over the
// non-Dirac bases (blockIdx.y); the Dirac basis is an elementwise copy.
//
// One level of the 1-D periodic analysis of a length-m signal:
//   a[k] = sum_i h[i] x[(2k + i) mod m],   d[k] = sum_i g[i] x[(2k + i) mod m],
// g[i] = (-1)^i h[L-1-i]; the synthesis is its transpose.
#include <cmath>
#include <complex>
#include <new>

#include "wavelet.cuh"

namespace gbri {

// ---- filters (host) ---------------------------------------------------------
std::vector<double> daubechies_lowpass(int N) {
  using C = std::complex<long double>;
  // P(y) = sum_{k<N} binom(N-1+k, k) y^k; its roots by Durand-Kerner iteration.
  std::vector<long double> p(N);
  for (int k = 0; k < N; ++k) {
    long double c = 1.0L;
    for (int j = 1; j <= k; ++j) c = c * (N - 1 + j) / j;
    p[k] = c;
  }
  const int d = N - 1;
  std::vector<C> roots(d);
  auto evalP = [&](C y) {
    C v = 0;
    for (int k = d; k >= 0; --k) v = v * y + p[k];
    return v;
  };
  if (d > 0) {
    const C seed(0.4L, 0.9L);
    C z = 1;
    for (int k = 0; k < d; ++k) {
      roots[k] = z;
      z *= seed;
    }
    for (int it = 0; it < 2000; ++it) {
      long double change = 0;
      for (int k = 0; k < d; ++k) {
        C den = p[d];
        for (int j = 0; j < d; ++j)
          if (j != k) den *= (roots[k] - roots[j]);
        const C delta = evalP(roots[k]) / den;
        roots[k] -= delta;
        change = std::max(change, std::abs(delta));
      }
      if (change < 1e-30L) break;
    }
    // Newton polish
    for (int k = 0; k < d; ++k)
      for (int it = 0; it < 5; ++it) {
        C v = 0, dv = 0;
        for (int j = d; j >= 0; --j) {
          dv = dv * roots[k] + v;
          v = v * roots[k] + p[j];
        }
        if (std::abs(dv) > 0) roots[k] -= v / dv;
      }
  }
  // H(w) = (1 + w)^N prod_k (1 - r_k w), r_k the root of z^2 - (2 - 4 y_k) z + 1 inside |z| < 1.
  std::vector<C> poly(1, C(1));
  for (int k = 0; k < N; ++k) {  // (1 + w)^N
    std::vector<C> q(poly.size() + 1, C(0));
    for (size_t i = 0; i < poly.size(); ++i) {
      q[i] += poly[i];
      q[i + 1] += poly[i];
    }
    poly.swap(q);
  }
  for (int k = 0; k < d; ++k) {
    const C b = C(2) - C(4) * roots[k];
    const C disc = std::sqrt(b * b - C(4));
    const C z1 = (b + disc) / C(2), z2 = (b - disc) / C(2);
    const C r = (std::abs(z1) < std::abs(z2)) ? z1 : z2;
    std::vector<C> q(poly.size() + 1, C(0));
    for (size_t i = 0; i < poly.size(); ++i) {
      q[i] += poly[i];
      q[i + 1] -= r * poly[i];
    }
    poly.swap(q);
  }
  long double sum = 0;
  for (auto& c : poly) sum += c.real();
  std::vector<double> h(poly.size());
  for (size_t i = 0; i < poly.size(); ++i) h[i] = (double)(poly[i].real() * std::sqrt(2.0L) / sum);
  return h;
}

namespace {

__device__ __forceinline__ int pmod(int v, int m) {
  v %= m;
  return v < 0 ? v + m : v;
}

// Row pass of the analysis at block size m (pitch n): out[r][k] = a, out[r][m/2 + k] = d.
__global__ void k_dwt_rows(const float* __restrict__ in, size_t in_stride, float* __restrict__ out, int m, int n,
                           const Filters F) {
  const int j = blockIdx.y;
  const int L = F.len[j];
  const int half = m >> 1;
  const float* src = in + in_stride * j;
  float* dst = out + (size_t)n * n * j;
  const int total = m * half;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int r = t / half, k = t - r * half;
    const float* row = src + (size_t)r * n;
    float a = 0.f, d = 0.f;
    for (int i = 0; i < L; ++i) {
      int idx = 2 * k + i;
      idx = (idx < m) ? idx : pmod(idx, m);
      const float v = row[idx];
      a = fmaf(F.h[j][i], v, a);
      d = fmaf(F.g[j][i], v, d);
    }
    dst[(size_t)r * n + k] = a;
    dst[(size_t)r * n + half + k] = d;
  }
}

__device__ __forceinline__ void emit(float* __restrict__ out, size_t q, float v, const DualEpi& e) {
  if (e.mode == 0) {
    out[q] = v;
  } else {
    const float u = fmaf(e.ca, out[q], e.cb * v);
    out[q] = fminf(fmaxf(u, -e.lim), e.lim) * e.ce;
  }
}

// Column pass: rows k (a) and m/2 + k (d) of column c.  The LL quadrant goes to
// the carry buffer unless this is the last level; every other coefficient is final.
__global__ void k_dwt_cols(const float* __restrict__ tmp, float* __restrict__ ll, float* __restrict__ out, int m,
                           int n, bool last, float scale, const Filters F, const DualEpi e) {
  const int j = blockIdx.y;
  const int L = F.len[j];
  const int half = m >> 1;
  const float* src = tmp + (size_t)n * n * j;
  float* carry = ll + (size_t)n * n * j;
  float* dst = out + (size_t)n * n * F.aidx[j];
  const int total = half * m;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int k = t / m, c = t - k * m;
    float a = 0.f, d = 0.f;
    for (int i = 0; i < L; ++i) {
      int idx = 2 * k + i;
      idx = (idx < m) ? idx : pmod(idx, m);
      const float v = src[(size_t)idx * n + c];
      a = fmaf(F.h[j][i], v, a);
      d = fmaf(F.g[j][i], v, d);
    }
    if (c < half && !last) carry[(size_t)k * n + c] = a;
    else emit(dst, (size_t)k * n + c, scale * a, e);
    emit(dst, (size_t)(half + k) * n + c, scale * d, e);
  }
}

// Synthesis, column pass at block size m: tmp[r][c] = sum over taps i with (r - i) even of
// h[i] A[k_i][c] + g[i] A[m/2 + k_i][c], k_i = ((r - i)/2) mod (m/2).  A's LL quadrant comes from
// the reconstruction buffer (from_rec) or from the coefficients (coarsest level).
__global__ void k_idwt_cols(const float* __restrict__ alpha, const float* __restrict__ rec, bool from_rec,
                            float* __restrict__ tmp, int m, int n, const Filters F) {
  const int j = blockIdx.y;
  const int L = F.len[j];
  const int half = m >> 1;
  const float* coef = alpha + (size_t)n * n * F.aidx[j];
  const float* llsrc = from_rec ? rec + (size_t)n * n * j : coef;
  float* dst = tmp + (size_t)n * n * j;
  const int total = m * m;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int r = t / m, c = t - r * m;
    const float* lo = (c < half) ? llsrc : coef;
    float v = 0.f;
    for (int i = r & 1; i < L; i += 2) {
      const int k = pmod((r - i) >> 1, half);
      v = fmaf(F.h[j][i], lo[(size_t)k * n + c], v);
      v = fmaf(F.g[j][i], coef[(size_t)(half + k) * n + c], v);
    }
    dst[(size_t)r * n + c] = v;
  }
}

// Synthesis, row pass: rec[r][c] = sum over taps with (c - i) even of h[i] tmp[r][k_i] + g[i] tmp[r][m/2 + k_i].
__global__ void k_idwt_rows(const float* __restrict__ tmp, float* __restrict__ rec, int m, int n, const Filters F) {
  const int j = blockIdx.y;
  const int L = F.len[j];
  const int half = m >> 1;
  const float* src = tmp + (size_t)n * n * j;
  float* dst = rec + (size_t)n * n * j;
  const int total = m * m;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int r = t / m, c = t - r * m;
    const float* row = src + (size_t)r * n;
    float v = 0.f;
    for (int i = c & 1; i < L; i += 2) {
      const int k = pmod((c - i) >> 1, half);
      v = fmaf(F.h[j][i], row[k], v);
      v = fmaf(F.g[j][i], row[half + k], v);
    }
    dst[(size_t)r * n + c] = v;
  }
}

// Dirac basis of the analysis: out[q] = epi(scale * x[q]).
__global__ void k_dirac(const float* __restrict__ x, float* __restrict__ out, int64_t N, float scale, const DualEpi e) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
    emit(out, (size_t)q, scale * x[q], e);
}

// x[q] = scale * (sum_j rec[j][q] + alpha[dirac][q])
__global__ void k_psi_sum(const float* __restrict__ rec, int nb, const float* __restrict__ dirac, float* __restrict__ x,
                          int64_t N, float scale) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
    float v = dirac ? dirac[q] : 0.f;
    for (int j = 0; j < nb; ++j) v += rec[(size_t)N * j + q];
    x[q] = scale * v;
  }
}

int blocks_for(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)num_sms() * 8));
}

}  // namespace

int32_t psi_adjoint_apply(gbri_wavelet* w, const float* x, float* out, DualEpi epi, cudaStream_t s) {
  const int n = w->n;
  const int64_t N = (int64_t)n * n;
  if (w->dirac_idx >= 0) {
    launch_begin(GBRI_K_PSI_ADJ, s);
    k_dirac<<<blocks_for(N), 256, 0, s>>>(x, out + (size_t)N * w->dirac_idx, N, w->scale, epi);
    GBRI_TRY(launch_end(GBRI_K_PSI_ADJ, s));
  }
  if (w->nb == 0) return GBRI_OK;
  for (int lev = 0; lev < w->levels; ++lev) {
    const int m = n >> lev;
    const float* in = (lev == 0) ? x : w->ll;
    const size_t in_stride = (lev == 0) ? 0 : (size_t)N;
    dim3 gr(blocks_for((int64_t)m * m / 2 / std::max(1, w->nb) + 1), w->nb);
    launch_begin(GBRI_K_PSI_ADJ, s);
    k_dwt_rows<<<gr, 256, 0, s>>>(in, in_stride, w->tmp, m, n, w->F);
    GBRI_TRY(launch_end(GBRI_K_PSI_ADJ, s));
    launch_begin(GBRI_K_PSI_ADJ, s);
    k_dwt_cols<<<gr, 256, 0, s>>>(w->tmp, w->ll, out, m, n, lev == w->levels - 1, w->scale, w->F, epi);
    GBRI_TRY(launch_end(GBRI_K_PSI_ADJ, s));
  }
  return GBRI_OK;
}

int32_t psi_apply(gbri_wavelet* w, const float* alpha, float* x, cudaStream_t s) {
  const int n = w->n;
  const int64_t N = (int64_t)n * n;
  for (int lev = w->levels - 1; lev >= 0 && w->nb > 0; --lev) {
    const int m = n >> lev;
    dim3 gr(blocks_for((int64_t)m * m / std::max(1, w->nb) + 1), w->nb);
    launch_begin(GBRI_K_PSI, s);
    k_idwt_cols<<<gr, 256, 0, s>>>(alpha, w->ll, lev != w->levels - 1, w->tmp, m, n, w->F);
    GBRI_TRY(launch_end(GBRI_K_PSI, s));
    launch_begin(GBRI_K_PSI, s);
    k_idwt_rows<<<gr, 256, 0, s>>>(w->tmp, w->ll, m, n, w->F);
    GBRI_TRY(launch_end(GBRI_K_PSI, s));
  }
  launch_begin(GBRI_K_PSI, s);
  k_psi_sum<<<blocks_for(N), 256, 0, s>>>(w->ll, w->nb, w->dirac_idx >= 0 ? alpha + (size_t)N * w->dirac_idx : nullptr,
                                          x, N, w->scale);
  return launch_end(GBRI_K_PSI, s);
}

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_wavelet_create(gbri_wavelet** out, int32_t n_side, int32_t levels, const int32_t* db_orders,
                            int32_t n_w, int32_t precision) {
  GBRI_CHECK(out && db_orders, GBRI_EINVAL, "null argument");
  *out = nullptr;
  GBRI_CHECK(precision == GBRI_F32, GBRI_EINVAL, "only GBRI_F32 is supported");
  GBRI_CHECK(n_w >= 1 && n_w <= kMaxBases, GBRI_EINVAL, "n_w must be in [1, 16]");
  GBRI_CHECK(levels >= 1 && levels <= 12, GBRI_EINVAL, "levels must be in [1, 12]");
  GBRI_CHECK(n_side >= 4 && n_side % (1 << levels) == 0 && (n_side >> levels) >= 2, GBRI_EINVAL,
             "n_side must be divisible by 2^levels with n_side >> levels >= 2");
  gbri_wavelet* w = new (std::nothrow) gbri_wavelet();
  GBRI_CHECK(w, GBRI_ENOMEM, "host allocation");
  w->n = n_side;
  w->levels = levels;
  w->nw = n_w;
  w->scale = (float)(1.0 / std::sqrt((double)n_w));
  for (int b = 0; b < n_w; ++b) {
    const int N = db_orders[b];
    if (N < 0 || N > kMaxTaps / 2 || (N == 0 && w->dirac_idx >= 0)) {
      delete w;
      return set_error(GBRI_EINVAL, "db order must be 0 (once) or 1..16");
    }
    w->orders.push_back(N);
    if (N == 0) {
      w->dirac_idx = b;
      continue;
    }
    const std::vector<double> h = daubechies_lowpass(N);
    const int L = (int)h.size();
    const int j = w->nb++;
    for (int i = 0; i < kMaxTaps; ++i) {
      w->F.h[j][i] = i < L ? (float)h[i] : 0.f;
      w->F.g[j][i] = i < L ? (float)((i % 2 ? -1.0 : 1.0) * h[L - 1 - i]) : 0.f;
    }
    w->F.len[j] = L;
    w->F.aidx[j] = b;
  }
  const size_t bytes = sizeof(float) * (size_t)std::max(1, w->nb) * n_side * n_side;
  if (cudaMalloc((void**)&w->tmp, bytes) != cudaSuccess || cudaMalloc((void**)&w->ll, bytes) != cudaSuccess) {
    cudaFree(w->tmp);
    cudaFree(w->ll);
    delete w;
    return set_error(GBRI_ENOMEM, "cudaMalloc wavelet buffers");
  }
  *out = w;
  return GBRI_OK;
}

int32_t gbri_wavelet_destroy(gbri_wavelet* w) {
  if (!w) return GBRI_OK;
  cudaDeviceSynchronize();
  cudaFree(w->tmp);
  cudaFree(w->ll);
  delete w;
  return GBRI_OK;
}

int32_t gbri_psi(gbri_wavelet* w, const float* d_alpha, float* d_x, void* stream) {
  GBRI_CHECK(w && d_alpha && d_x, GBRI_EINVAL, "null argument");
  return psi_apply(w, d_alpha, d_x, (cudaStream_t)stream);
}

int32_t gbri_psi_adjoint(gbri_wavelet* w, const float* d_x, float* d_alpha, void* stream) {
  GBRI_CHECK(w && d_alpha && d_x, GBRI_EINVAL, "null argument");
  DualEpi e{0, 0.f, 0.f, 0.f, 0.f};
  return psi_adjoint_apply(w, d_x, d_alpha, e, (cudaStream_t)stream);
}

}  // extern "C"
