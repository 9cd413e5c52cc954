// Measurement operator calls: Phi (Sec. 2, Eq. 2) = degrid(F(pad_correct(x))),
// Phi^dagger = crop_correct(F^H(grid(y))), visibility reordering and the power
// method for ||Phi||^2 (Sec. 6.3.1).
#include <cmath>
#include <mutex>
#include <vector>

#include "nufft.cuh"

namespace gbri {

// Degridding (G then W, Sec. 2).  A block takes one chunk (one contiguous range of
// at most kThreads * kRun visibilities of one 16 x 16 tile), copies the tile's
// (T + J - 1)^2 grid window into shared memory when the tile changes, and gives one
// thread per visibility with kRun visibilities in flight per thread (coalesced
// metadata and epilogue streams):
//   v = w * sum_{t'} wy[t'] sum_t wx[t] win[cy + t'][cx + t]
// with the two J-tap weight rows from the shared-memory table.  The visibilities of
// a sub-run share a cell, so neighbouring lanes often read the same window words.
// `Epi` consumes (plan position, v).  Persistent blocks stride over the chunks.
template <int J, class Epi>
__global__ void __launch_bounds__(kThreads, (J == 4 ? 4 : 3)) k_degrid(VisGeom geo, const float2* __restrict__ grid,
                                                                       Epi epi) {
  extern __shared__ float4 smem_dg[];
  constexpr int P = kTile + J - 1;
  float* sw = reinterpret_cast<float*>(smem_dg);
  const int S = 1 << geo.log2S;
  float2* win = reinterpret_cast<float2*>(sw + table_floats(S, J));
  copy_table_to_smem(sw, geo.wtab, table_floats(S, J));
  const int K = geo.K;
  int cur_tile = -1;
  for (int c = blockIdx.x; c < geo.n_chunks; c += gridDim.x) {
    const int4 ch = geo.chunks[c];
    const int2 s0 = geo.subruns[ch.y], s1 = geo.subruns[ch.y + ch.z - 1];
    const int lo = s0.x, cnt = s1.x + s1.y - s0.x;
    if (ch.x != cur_tile) {
      __syncthreads();
      const int ty = ch.x / geo.nT, tx = ch.x - ty * geo.nT;
      const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
      for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int r = i / P, cc = i - r * P;
        win[r * kWinPitch + cc] = __ldg(grid + (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K));
      }
      cur_tile = ch.x;
      __syncthreads();
    }
    uint2 m[kRun];
    typename Epi::Pre pre[kRun];
#pragma unroll
    for (int k = 0; k < kRun; ++k) {
      const int i = threadIdx.x + k * kThreads;
      if (i < cnt) {
        m[k] = geo.meta[lo + i];
        pre[k] = epi.load(lo + i);
      }
    }
#pragma unroll
    for (int k = 0; k < kRun; ++k) {
      const int i = threadIdx.x + k * kThreads;
      if (i >= cnt) break;
      const int lx = m[k].x & 0xffff, ly = m[k].x >> 16;
      float wx[J], wy[J];
      load_taps<J>(sw, lx & (S - 1), S, wx);
      load_taps<J>(sw, ly & (S - 1), S, wy);
      const float2* base = win + (ly >> geo.log2S) * kWinPitch + (lx >> geo.log2S);
      float ar = 0.f, ai = 0.f;
#pragma unroll
      for (int tp = 0; tp < J; ++tp) {
        float rr = 0.f, ri = 0.f;
#pragma unroll
        for (int t = 0; t < J; ++t) {
          const float2 gv = base[tp * kWinPitch + t];
          rr = fmaf(wx[t], gv.x, rr);
          ri = fmaf(wx[t], gv.y, ri);
        }
        ar = fmaf(wy[tp], rr, ar);
        ai = fmaf(wy[tp], ri, ai);
      }
      const float w = __uint_as_float(m[k].y);
      epi.store(lo + i, pre[k], make_float2(w * ar, w * ai));
    }
  }
  epi.finish();
}

// Gridding (W^T then G^T, Sec. 2).  A block takes one chunk (up to kThreads sub-run
// slots of one tile; each round of the rank-major order starts at a warp boundary,
// so the 32 lanes of a warp hold sub-runs of 32 distinct cells).  Thread t loads
// its sub-run (<= kRun visibilities of one cell) at once, sums w * v * wy[t'] wx[t]
// into a J x J register patch and adds it to its warp's private (T + J - 1)^2
// accumulator in shared memory with plain read-modify-writes: the lanes of one
// instruction touch distinct cells, and successive instructions of a warp are
// ordered, so no atomics are needed.  The block then sums the warp accumulators and
// writes the tile window to the global grid: plain stores for the cells no other
// tile touches when the tile is a single chunk, vector atomics otherwise.
// `Src` gives the visibility value at a plan position.
template <int J, class Src>
__global__ void __launch_bounds__(kThreads, (J == 4 ? 3 : 2)) k_grid(VisGeom geo, float2* __restrict__ grid, Src src) {
  extern __shared__ float4 smem_gr[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  const int S = 1 << geo.log2S;
  float* sw = reinterpret_cast<float*>(smem_gr);
  float2* accs = reinterpret_cast<float2*>(sw + table_floats(S, J));
  copy_table_to_smem(sw, geo.wtab, table_floats(S, J));
  float2* acc = accs + (threadIdx.x >> 5) * (P * kAccPitch2);
  const int K = geo.K;
  for (int c = blockIdx.x; c < geo.n_chunks; c += gridDim.x) {
    const int4 ch = geo.chunks[c];
    for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) accs[i] = make_float2(0.f, 0.f);
    __syncthreads();
    {
      const int2 sr = ((int)threadIdx.x < ch.z) ? geo.subruns[ch.y + threadIdx.x] : make_int2(0, 0);
      const bool active = sr.y > 0;
      uint2 m[kRun];
      float2 v[kRun];
#pragma unroll
      for (int k = 0; k < kRun; ++k)
        if (k < sr.y) {
          m[k] = geo.meta[sr.x + k];
          v[k] = src(sr.x + k);
        }
      float2 pt[J][J];
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) pt[tp][t] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        if (k >= sr.y) break;
        float wx[J], wy[J];
        load_taps<J>(sw, (m[k].x & 0xffff) & (S - 1), S, wx);
        load_taps<J>(sw, (m[k].x >> 16) & (S - 1), S, wy);
        const float w = __uint_as_float(m[k].y);
        const float vr = w * v[k].x, vi = w * v[k].y;
#pragma unroll
        for (int tp = 0; tp < J; ++tp) {
          const float br = wy[tp] * vr, bi = wy[tp] * vi;
#pragma unroll
          for (int t = 0; t < J; ++t) {
            pt[tp][t].x = fmaf(wx[t], br, pt[tp][t].x);
            pt[tp][t].y = fmaf(wx[t], bi, pt[tp][t].y);
          }
        }
      }
      const int a0 = active ? ((int)(m[0].x >> 16) >> geo.log2S) * kAccPitch2 + ((int)(m[0].x & 0xffff) >> geo.log2S)
                            : 0;
      // all 32 lanes walk the taps in lockstep: within one tap the active lanes touch
      // distinct cells, and the warp barrier orders one tap's stores before the next
      // tap's loads (a neighbour cell's patch overlaps this one)
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (active) {
            float2* q = acc + a0 + tp * kAccPitch2 + t;
            const float2 o = *q;
            *q = make_float2(o.x + pt[tp][t].x, o.y + pt[tp][t].y);
          }
          __syncwarp();
        }
    }
    __syncthreads();
    const int ty = ch.x / geo.nT, tx = ch.x - ty * geo.nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    // accumulator rows / cols [lo_x, hi_x) belong to no other tile's window
    constexpr int lo_x = J - 1, hi_x = kTile;
    const bool single = ch.w != 0;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
      const int r = i / P, cc = i - r * P;
      float2 a = make_float2(0.f, 0.f);
#pragma unroll
      for (int wq = 0; wq < W; ++wq) {
        const float2 b = accs[wq * (P * kAccPitch2) + r * kAccPitch2 + cc];
        a.x += b.x;
        a.y += b.y;
      }
      float2* dst = grid + (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
      if (single && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) *dst = a;
      else if (a.x != 0.f || a.y != 0.f) atomicAdd(dst, a);
    }
    __syncthreads();
  }
}

template <int J, class Epi>
inline void degrid_instance(gbri_plan* p, const float2* grid, Epi epi, cudaStream_t s) {
  k_degrid<J, Epi><<<p->degrid_blocks, kThreads, degrid_smem(p), s>>>(vis_geom(p), grid, epi);
}

template <class Epi>
int32_t launch_degrid(gbri_plan* p, const float2* grid, Epi epi, cudaStream_t s) {
  launch_begin(GBRI_K_DEGRID, s);
  if (p->J == 4) degrid_instance<4>(p, grid, epi, s);
  else degrid_instance<6>(p, grid, epi, s);
  return launch_end(GBRI_K_DEGRID, s);
}

template <int J, class Src>
inline void grid_instance(gbri_plan* p, float2* grid, Src src, cudaStream_t s) {
  k_grid<J, Src><<<p->grid_blocks, kThreads, grid_smem(p), s>>>(vis_geom(p), grid, src);
}

// Zeroes p->grid, then grids every visibility into it.
template <class Src>
int32_t launch_grid(gbri_plan* p, Src src, cudaStream_t s) {
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->grid, 0, sizeof(float2) * (size_t)p->K * p->K, s));
  if (p->n_chunks == 0) return GBRI_OK;
  launch_begin(GBRI_K_GRID, s);
  if (p->J == 4) grid_instance<4>(p, p->grid, src, s);
  else grid_instance<6>(p, p->grid, src, s);
  return launch_end(GBRI_K_GRID, s);
}


// Dynamic shared memory above 48 KB needs a per-kernel attribute; it is set once
// for every instantiation before any launch (so never inside a stream capture).
int32_t prepare_visibility_kernels() {
  static int32_t status = -100;
  static std::once_flag once;
  std::call_once(once, [] {
    const int lim = 200 * 1024;
    cudaError_t e = cudaSuccess;
#define GBRI_ATTR(kern) if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
    GBRI_ATTR((k_degrid<4, EpiStorePlan>)); GBRI_ATTR((k_degrid<6, EpiStorePlan>));
    GBRI_ATTR((k_degrid<4, EpiStoreRaw>)); GBRI_ATTR((k_degrid<6, EpiStoreRaw>));
    GBRI_ATTR((k_degrid<4, EpiPD1>)); GBRI_ATTR((k_degrid<6, EpiPD1>));
    GBRI_ATTR((k_degrid<4, EpiADMM1>)); GBRI_ATTR((k_degrid<6, EpiADMM1>));
    GBRI_ATTR((k_grid<4, SrcPlan>)); GBRI_ATTR((k_grid<6, SrcPlan>));
    GBRI_ATTR((k_grid<4, SrcRaw>)); GBRI_ATTR((k_grid<6, SrcRaw>));
    GBRI_ATTR((k_grid<4, SrcADMM2>)); GBRI_ATTR((k_grid<6, SrcADMM2>));
#undef GBRI_ATTR
    status = (e == cudaSuccess) ? GBRI_OK : cuda_error(e, "cudaFuncSetAttribute");
  });
  return status;
}

// Every visibility kernel is instantiated here and only here.
template int32_t launch_degrid<EpiStorePlan>(gbri_plan*, const float2*, EpiStorePlan, cudaStream_t);
template int32_t launch_degrid<EpiStoreRaw>(gbri_plan*, const float2*, EpiStoreRaw, cudaStream_t);
template int32_t launch_degrid<EpiPD1>(gbri_plan*, const float2*, EpiPD1, cudaStream_t);
template int32_t launch_degrid<EpiADMM1>(gbri_plan*, const float2*, EpiADMM1, cudaStream_t);
template int32_t launch_grid<SrcPlan>(gbri_plan*, SrcPlan, cudaStream_t);
template int32_t launch_grid<SrcRaw>(gbri_plan*, SrcRaw, cudaStream_t);
template int32_t launch_grid<SrcADMM2>(gbri_plan*, SrcADMM2, cudaStream_t);

namespace {

// Z S: padded[(q - n/2) mod K][(p - n/2) mod K] = corr[p] corr[q] x[q][p] * inv_scale
__global__ void k_pad(const float* __restrict__ x, const float* __restrict__ corr, float2* __restrict__ padded,
                      int n, int K, const double* __restrict__ d_norm) {
  const float s = d_norm ? (float)(1.0 / *d_norm) : 1.0f;
  const int total = n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int q = i / n, p = i - q * n;
    int r = q - n / 2; if (r < 0) r += K;
    int c = p - n / 2; if (c < 0) c += K;
    padded[(size_t)r * K + c] = make_float2(x[i] * corr[p] * corr[q] * s, 0.f);
  }
}

// S^T Z^T and the real part: x[q][p] = corr[p] corr[q] Re(grid[(q - n/2) mod K][(p - n/2) mod K])
__global__ void k_crop(const float2* __restrict__ grid, const float* __restrict__ corr, float* __restrict__ x,
                       int n, int K) {
  const int total = n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int q = i / n, p = i - q * n;
    int r = q - n / 2; if (r < 0) r += K;
    int c = p - n / 2; if (c < 0) c += K;
    x[i] = corr[p] * corr[q] * grid[(size_t)r * K + c].x;
  }
}

__global__ void k_gather(const float2* __restrict__ in, const int32_t* __restrict__ perm, float2* __restrict__ out,
                         int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
__global__ void k_scatter_vis(const float2* __restrict__ in, const int32_t* __restrict__ perm,
                              float2* __restrict__ out, int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}

// FP64 sum of squares of an image into partials[blockIdx.x] (per-thread FP32 Kahan partials).
__global__ void k_image_sumsq(const float* __restrict__ x, int64_t n, double* __restrict__ partials) {
  __shared__ double sh[40];
  KahanF acc;
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
__global__ void k_power_start(float* __restrict__ b, int64_t n, uint64_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    b[i] = (float)(0.5 + (double)(z >> 11) * (1.0 / 9007199254740992.0));
  }
}

int grid_blocks_for(int64_t n, int threads = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, threads), (int64_t)num_sms() * 8));
}

}  // namespace

int32_t launch_pad(gbri_plan* p, const float* x, const double* d_norm, cudaStream_t s) {
  launch_begin(GBRI_K_PAD, s);
  k_pad<<<grid_blocks_for((int64_t)p->n_side * p->n_side), 256, 0, s>>>(x, p->corr, p->padded, p->n_side, p->K,
                                                                         d_norm);
  return launch_end(GBRI_K_PAD, s);
}

int32_t launch_crop(gbri_plan* p, float* x, cudaStream_t s) {
  launch_begin(GBRI_K_CROP, s);
  k_crop<<<grid_blocks_for((int64_t)p->n_side * p->n_side), 256, 0, s>>>(p->grid, p->corr, x, p->n_side, p->K);
  return launch_end(GBRI_K_CROP, s);
}

int32_t fft_forward(gbri_plan* p, cudaStream_t s) {
  if (cufftSetStream(p->fft, s) != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftSetStream");
  launch_begin(GBRI_K_FFT_FWD, s, false);
  const cufftResult r = cufftExecC2C(p->fft, reinterpret_cast<cufftComplex*>(p->padded),
                                     reinterpret_cast<cufftComplex*>(p->grid), CUFFT_FORWARD);
  const int32_t st = launch_end(GBRI_K_FFT_FWD, s);
  if (r != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftExecC2C forward");
  return st;
}

int32_t fft_inverse(gbri_plan* p, cudaStream_t s) {
  if (cufftSetStream(p->fft, s) != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftSetStream");
  launch_begin(GBRI_K_FFT_INV, s, false);
  const cufftResult r = cufftExecC2C(p->fft, reinterpret_cast<cufftComplex*>(p->grid),
                                     reinterpret_cast<cufftComplex*>(p->grid), CUFFT_INVERSE);
  const int32_t st = launch_end(GBRI_K_FFT_INV, s);
  if (r != CUFFT_SUCCESS) return set_error(GBRI_ECUFFT, "cufftExecC2C inverse");
  return st;
}

int32_t normal_op(gbri_plan* p, const float* b, const double* d_norm, float* out, cudaStream_t s) {
  GBRI_TRY(launch_pad(p, b, d_norm, s));
  GBRI_TRY(fft_forward(p, s));
  GBRI_TRY(launch_degrid(p, p->grid, EpiStorePlan{p->vis_tmp}, s));
  GBRI_TRY(launch_grid(p, SrcPlan{p->vis_tmp}, s));
  GBRI_TRY(fft_inverse(p, s));
  return launch_crop(p, out, s);
}

int32_t image_norm(gbri_plan* p, const float* x, double* d_out, cudaStream_t s) {
  const int64_t n = (int64_t)p->n_side * p->n_side;
  const int blocks = std::min(grid_blocks_for(n), p->n_partials);
  launch_begin(GBRI_K_OTHER, s);
  k_image_sumsq<<<blocks, 256, 0, s>>>(x, n, p->partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, s));
  launch_begin(GBRI_K_OTHER, s);
  k_finish_norm<<<1, 256, 0, s>>>(p->partials, blocks, d_out);
  return launch_end(GBRI_K_OTHER, s);
}

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_vis_reorder(const gbri_plan* pc, const float* d_in, float* d_out, int32_t to_plan, void* stream) {
  GBRI_CHECK(pc, GBRI_EINVAL, "null plan");
  if (pc->M == 0) return GBRI_OK;
  GBRI_CHECK(d_in && d_out && d_in != d_out, GBRI_EINVAL, "bad buffers");
  cudaStream_t s = (cudaStream_t)stream;
  gbri_plan* p = const_cast<gbri_plan*>(pc);
  launch_begin(GBRI_K_OTHER, s);
  if (to_plan)
    k_gather<<<grid_blocks_for(p->M), 256, 0, s>>>((const float2*)d_in, p->perm, (float2*)d_out, p->M);
  else
    k_scatter_vis<<<grid_blocks_for(p->M), 256, 0, s>>>((const float2*)d_in, p->perm, (float2*)d_out, p->M);
  return launch_end(GBRI_K_OTHER, s);
}

int32_t gbri_phi(gbri_plan* p, const float* d_x, float* d_y, uint32_t flags, void* stream) {
  GBRI_CHECK(p && d_x && (d_y || p->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  GBRI_TRY(launch_pad(p, d_x, nullptr, s));
  GBRI_TRY(fft_forward(p, s));
  if (p->M == 0) return GBRI_OK;
  if (flags & GBRI_PLAN_ORDER) return launch_degrid(p, p->grid, EpiStorePlan{(float2*)d_y}, s);
  return launch_degrid(p, p->grid, EpiStoreRaw{(float2*)d_y, p->perm}, s);
}

int32_t gbri_phi_adjoint(gbri_plan* p, const float* d_y, float* d_x, uint32_t flags, void* stream) {
  GBRI_CHECK(p && d_x && (d_y || p->M == 0), GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (flags & GBRI_PLAN_ORDER)
    GBRI_TRY(launch_grid(p, SrcPlan{(const float2*)d_y}, s));
  else
    GBRI_TRY(launch_grid(p, SrcRaw{(const float2*)d_y, p->perm}, s));
  GBRI_TRY(fft_inverse(p, s));
  return launch_crop(p, d_x, s);
}

int32_t gbri_op_norm(gbri_plan* p, int32_t max_iter, double tol, uint64_t seed, double* op_norm_sq,
                     int32_t* iters, void* stream) {
  GBRI_CHECK(p && op_norm_sq && max_iter > 0, GBRI_EINVAL, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = (int64_t)p->n_side * p->n_side;
  float *b = nullptr, *c = nullptr;
  double* d_norm = p->scalars + 8;  // scalars[8]: norm of the current vector
  GBRI_CHECK_CUDA(cudaMallocAsync((void**)&b, sizeof(float) * n, s));
  cudaError_t e = cudaMallocAsync((void**)&c, sizeof(float) * n, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(b, s);
    return cuda_error(e, "cudaMallocAsync");
  }
  int32_t st = GBRI_OK;
  launch_begin(GBRI_K_OTHER, s);
  k_power_start<<<grid_blocks_for(n), 256, 0, s>>>(b, n, seed);
  st = launch_end(GBRI_K_OTHER, s);
  if (st == GBRI_OK) st = image_norm(p, b, d_norm, s);
  double prev = 0.0, val = 0.0;
  int it = 0;
  for (it = 1; it <= max_iter && st == GBRI_OK; ++it) {
    // c = Phi^dagger Phi (b / ||b||), then ||c||
    st = normal_op(p, b, d_norm, c, s);
    if (st != GBRI_OK) break;
    st = image_norm(p, c, d_norm, s);
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

}  // extern "C"
