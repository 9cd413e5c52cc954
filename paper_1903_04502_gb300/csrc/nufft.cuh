// Measurement operator Phi = W G F Z S (Sec. 2, Eq. 2) on one GPU: the plan
// object and the kernel templates shared by the operator calls and the solvers.
//
// Data layout in HBM (per plan):
//   meta   [M] uint2   plan (sorted) order: .x = (ly << 16) | lx, the tile-local
//                      fixed-point coordinates (cell-in-tile * S + fraction),
//                      .y = weight bits (float).  8 bytes per visibility.
//   perm   [M] int32   plan position -> caller's visibility index.
//   chunks [C] int4    {tile, first plan position, count, 0}; a chunk holds at
//                      most kChunk visibilities of one T x T tile.
//   wtab   [S][J] f32  tap weights by fractional offset f = k~ mod S: entry t is
//                      table[|f + (J/2 - 1 - t) S|] (Sec. 8.1 zeroth-order table,
//                      re-indexed so one visibility reads one row per axis).
//   corr   [n] f32     1 / ghat(p'/K) (the S factor along one axis).
//   padded [K][K] c64  FFT input; zero outside the n x n image block (kept zero).
//   grid   [K][K] c64  FFT output / gridding accumulator.
#pragma once

#include <cufft.h>

#include <vector>

#include "common.cuh"

namespace gbri {

constexpr int kTile = 16;      // grid tile side in cells (T * S <= 65536 keeps 16-bit local coords)
constexpr int kChunk = 1024;   // visibilities per work chunk
constexpr int kThreads = 256;  // threads per block of the visibility kernels

}  // namespace gbri

struct gbri_plan {
  int n_side = 0, K = 0, J = 0, S = 0, log2S = 0, nT = 0, prec = 0;
  double beta = 0;
  int64_t M = 0;
  uint2* meta = nullptr;
  int32_t* perm = nullptr;
  int4* chunks = nullptr;
  int64_t n_chunks = 0;
  float* wtab = nullptr;
  float* corr = nullptr;
  float2* padded = nullptr;
  float2* grid = nullptr;
  float2* vis_tmp = nullptr;   // [M] plan-order scratch
  double* partials = nullptr;  // reduction partials
  double* scalars = nullptr;   // small device scalars
  int n_partials = 0;
  cufftHandle fft = 0;
  bool fft_ok = false;
  int64_t device_bytes = 0;
  int degrid_blocks = 0, grid_blocks = 0;
};

namespace gbri {

__device__ __forceinline__ int wrapK(int v, int K) { return v < 0 ? v + K : (v >= K ? v - K : v); }

// Load the J tap weights of one axis for fractional offset f from the shared table.
template <int J>
__device__ __forceinline__ void load_taps(const float* sw, int f, float (&w)[J]) {
  if constexpr (J == 4) {
    float4 v = reinterpret_cast<const float4*>(sw)[f];
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
  } else if constexpr (J == 6) {
    const float2* p = reinterpret_cast<const float2*>(sw + f * 6);
    float2 a = p[0], b = p[1], c = p[2];
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y; w[4] = c.x; w[5] = c.y;
  } else {
#pragma unroll
    for (int t = 0; t < J; ++t) w[t] = sw[f * J + t];
  }
}

__device__ __forceinline__ void copy_table_to_smem(float* sw, const float* __restrict__ g, int nfloats) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float4* s4 = reinterpret_cast<float4*>(sw);
  for (int i = threadIdx.x; i < nfloats / 4; i += blockDim.x) s4[i] = __ldg(g4 + i);
}

struct VisGeom {
  const uint2* __restrict__ meta;
  const int4* __restrict__ chunks;
  const float* __restrict__ wtab;
  int n_chunks, K, log2S, nT;
};

// Degridding (G then W, Sec. 2): for every visibility of every chunk,
//   v = w * sum_{t'} wy[t'] sum_t wx[t] grid[row(t')][col(t)]
// with the grid read through the read-only path and the kernel table in shared
// memory; `Epi` consumes (plan position, v).  Persistent blocks stride over chunks.
template <int J, class Epi>
__global__ void __launch_bounds__(kThreads) k_degrid(VisGeom geo, const float2* __restrict__ grid, Epi epi) {
  extern __shared__ float4 smem_dg[];
  float* sw = reinterpret_cast<float*>(smem_dg);
  const int S = 1 << geo.log2S;
  copy_table_to_smem(sw, geo.wtab, S * J);
  __syncthreads();
  const int K = geo.K;
  for (int c = blockIdx.x; c < geo.n_chunks; c += gridDim.x) {
    const int4 ch = geo.chunks[c];
    const int ty = ch.x / geo.nT, tx = ch.x - ty * geo.nT;
    const int ox = tx * kTile - (J / 2 - 1), oy = ty * kTile - (J / 2 - 1);
    for (int i = threadIdx.x; i < ch.z; i += blockDim.x) {
      const int pos = ch.y + i;
      const uint2 m = geo.meta[pos];
      const int lx = m.x & 0xffff, ly = m.x >> 16;
      const int cx = ox + (lx >> geo.log2S), cy = oy + (ly >> geo.log2S);
      float wx[J], wy[J];
      load_taps<J>(sw, lx & (S - 1), wx);
      load_taps<J>(sw, ly & (S - 1), wy);
      int col[J];
#pragma unroll
      for (int t = 0; t < J; ++t) col[t] = wrapK(cx + t, K);
      float ar = 0.f, ai = 0.f;
#pragma unroll
      for (int tp = 0; tp < J; ++tp) {
        const float2* gr = grid + (size_t)wrapK(cy + tp, K) * K;
        float rr = 0.f, ri = 0.f;
#pragma unroll
        for (int t = 0; t < J; ++t) {
          const float2 g = __ldg(gr + col[t]);
          rr = fmaf(wx[t], g.x, rr);
          ri = fmaf(wx[t], g.y, ri);
        }
        ar = fmaf(wy[tp], rr, ar);
        ai = fmaf(wy[tp], ri, ai);
      }
      const float w = __uint_as_float(m.y);
      epi(pos, make_float2(w * ar, w * ai));
    }
  }
  epi.finish();
}

// Gridding (W^T then G^T, Sec. 2): every visibility of a chunk adds
// w * wy[t'] * wx[t] * v to its J x J cells in a shared (T+J-1)^2 accumulator
// tile; the tile is then flushed to the global grid with one vector atomic per
// non-zero cell.  `Src` gives the visibility value at a plan position.
template <int J, class Src>
__global__ void __launch_bounds__(kThreads) k_grid(VisGeom geo, float2* __restrict__ grid, Src src) {
  extern __shared__ float4 smem_gr[];
  constexpr int P = kTile + J - 1;
  const int S = 1 << geo.log2S;
  float* sw = reinterpret_cast<float*>(smem_gr);
  float2* acc = reinterpret_cast<float2*>(sw + S * J);
  copy_table_to_smem(sw, geo.wtab, S * J);
  const int K = geo.K;
  for (int c = blockIdx.x; c < geo.n_chunks; c += gridDim.x) {
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) acc[i] = make_float2(0.f, 0.f);
    __syncthreads();
    const int4 ch = geo.chunks[c];
    const int ty = ch.x / geo.nT, tx = ch.x - ty * geo.nT;
    for (int i = threadIdx.x; i < ch.z; i += blockDim.x) {
      const int pos = ch.y + i;
      const uint2 m = geo.meta[pos];
      const int lx = m.x & 0xffff, ly = m.x >> 16;
      const int lcx = lx >> geo.log2S, lcy = ly >> geo.log2S;
      float wx[J], wy[J];
      load_taps<J>(sw, lx & (S - 1), wx);
      load_taps<J>(sw, ly & (S - 1), wy);
      float2 v = src(pos);
      const float w = __uint_as_float(m.y);
      v.x *= w;
      v.y *= w;
#pragma unroll
      for (int tp = 0; tp < J; ++tp) {
        float* rowp = reinterpret_cast<float*>(acc + (lcy + tp) * P + lcx);
        const float br = wy[tp] * v.x, bi = wy[tp] * v.y;
#pragma unroll
        for (int t = 0; t < J; ++t) {
          atomicAdd(rowp + 2 * t, wx[t] * br);
          atomicAdd(rowp + 2 * t + 1, wx[t] * bi);
        }
      }
    }
    __syncthreads();
    const int ox = tx * kTile - (J / 2 - 1), oy = ty * kTile - (J / 2 - 1);
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
      const float2 a = acc[i];
      if (a.x != 0.f || a.y != 0.f) {
        const int r = i / P, cc = i - r * P;
        atomicAdd(grid + (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K), a);
      }
    }
    __syncthreads();
  }
}

inline size_t degrid_smem(const gbri_plan* p) { return (size_t)p->S * p->J * sizeof(float); }
inline size_t grid_smem(const gbri_plan* p) {
  const int P = kTile + p->J - 1;
  return (size_t)p->S * p->J * sizeof(float) + (size_t)P * P * sizeof(float2);
}

inline VisGeom vis_geom(const gbri_plan* p) {
  VisGeom g;
  g.meta = p->meta;
  g.chunks = p->chunks;
  g.wtab = p->wtab;
  g.n_chunks = (int)p->n_chunks;
  g.K = p->K;
  g.log2S = p->log2S;
  g.nT = p->nT;
  return g;
}

// ---- epilogues / sources ------------------------------------------------------
struct EpiStorePlan {  // y[pos] = v
  float2* y;
  __device__ __forceinline__ void operator()(int pos, float2 v) { y[pos] = v; }
  __device__ __forceinline__ void finish() {}
};
struct EpiStoreRaw {  // y[perm[pos]] = v
  float2* y;
  const int32_t* perm;
  __device__ __forceinline__ void operator()(int pos, float2 v) { y[perm[pos]] = v; }
  __device__ __forceinline__ void finish() {}
};
struct SrcPlan {
  const float2* y;
  __device__ __forceinline__ float2 operator()(int pos) const { return y[pos]; }
};
struct SrcRaw {
  const float2* y;
  const int32_t* perm;
  __device__ __forceinline__ float2 operator()(int pos) const { return y[perm[pos]]; }
};

// ---- launch helpers -------------------------------------------------------------
template <int J, class Epi>
inline void degrid_instance(gbri_plan* p, const float2* grid, Epi epi, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = degrid_smem(p);
  if (!attr) {
    cudaFuncSetAttribute(k_degrid<J, Epi>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_degrid<J, Epi><<<p->degrid_blocks, kThreads, smem, s>>>(vis_geom(p), grid, epi);
}

template <class Epi>
inline int32_t launch_degrid(gbri_plan* p, const float2* grid, Epi epi, cudaStream_t s) {
  launch_begin(GBRI_K_DEGRID, s);
  if (p->J == 4) degrid_instance<4>(p, grid, epi, s);
  else degrid_instance<6>(p, grid, epi, s);
  return launch_end(GBRI_K_DEGRID, s);
}

template <int J, class Src>
inline void grid_instance(gbri_plan* p, float2* grid, Src src, cudaStream_t s) {
  static bool attr = false;
  const size_t smem = grid_smem(p);
  if (!attr) {
    cudaFuncSetAttribute(k_grid<J, Src>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_grid<J, Src><<<p->grid_blocks, kThreads, smem, s>>>(vis_geom(p), grid, src);
}

// Zeroes p->grid, then grids every visibility into it.
template <class Src>
inline int32_t launch_grid(gbri_plan* p, Src src, cudaStream_t s) {
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->grid, 0, sizeof(float2) * (size_t)p->K * p->K, s));
  if (p->n_chunks == 0) return GBRI_OK;
  launch_begin(GBRI_K_GRID, s);
  if (p->J == 4) grid_instance<4>(p, p->grid, src, s);
  else grid_instance<6>(p, p->grid, src, s);
  return launch_end(GBRI_K_GRID, s);
}

// Z S x into p->padded; optional extra scaling by *d_scale (device, may be null).
int32_t launch_pad(gbri_plan* p, const float* x, const double* d_inv_scale, cudaStream_t s);
// F: padded -> grid (forward, unnormalised); F^H: grid in place (inverse, unnormalised).
int32_t fft_forward(gbri_plan* p, cudaStream_t s);
int32_t fft_inverse(gbri_plan* p, cudaStream_t s);
// S^T Z^T Re(grid) into x.
int32_t launch_crop(gbri_plan* p, float* x, cudaStream_t s);
// Phi^dagger Phi b for the power method: b (image) -> out (image), plan-order scratch.
int32_t normal_op(gbri_plan* p, const float* b, const double* d_inv_scale, float* out, cudaStream_t s);

}  // namespace gbri
