// FP32 degridding and gridding kernels of Sec. 2 / Eq. 2 with polynomial taps (kTapPoly):
// the tap weights come from the kernel's per-segment polynomial fit evaluated in registers,
// and the complex multiply-adds of the interpolation run on packed (re, im) pairs (f32x2
// FMA: one instruction per complex-by-real multiply-add).  Work items (degridding chunks, gridding
// tiles) are handed out dynamically: each warp takes the next item from a device counter,
// so the persistent blocks finish together although the items differ in size (they are
// listed heaviest first).  Included only by the FP32 visibility translation unit.
#pragma once

#include "nufft.cuh"

namespace gbri {

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// Tap weights of both axes from the packed coordinates mx = (ly << 16) | lx: w[t] =
// (wx[t], wy[t]), the same weights as load_taps (entry t of an axis is g at
// distance |f + (J/2 - 1 - t) S| / S, f the coordinate's fraction).  Scalar FMAs with the
// coefficients as constant operands: evaluating both axes in packed pairs made the
// compiler hold the coefficient pairs in registers, which the kernels need (spills).
template <int J>
__device__ __forceinline__ void taps_xy(const PolyTaps& c, uint32_t mx, int S, float two_over_S, float2 (&w)[J]) {
  const int fx = (int)(mx & (uint32_t)(S - 1)), fy = (int)((mx >> 16) & (uint32_t)(S - 1));
  const float zx = fmaf((float)fx, two_over_S, -1.f), zy = fmaf((float)fy, two_over_S, -1.f);
  const float ux = zx * zx, uy = zy * zy;
#pragma unroll
  for (int k = 0; k < J / 2; ++k) {
    float ex = c.e[k][kPolyHalf - 1], ox = c.o[k][kPolyHalf - 1], ey = ex, oy = ox;
#pragma unroll
    for (int i = kPolyHalf - 2; i >= 0; --i) {
      ex = fmaf(ex, ux, c.e[k][i]);
      ox = fmaf(ox, ux, c.o[k][i]);
      ey = fmaf(ey, uy, c.e[k][i]);
      oy = fmaf(oy, uy, c.o[k][i]);
    }
    w[J / 2 - 1 - k] = make_float2(fmaf(zx, ox, ex), fmaf(zy, oy, ey));
    w[J / 2 + k] = make_float2(fmaf(-zx, ox, ex), fmaf(-zy, oy, ey));
  }
  if (fx == 0) w[J - 1].x = 0.f;
  if (fy == 0) w[J - 1].y = 0.f;
}

// Next work item of a warp from the device counter ctr[0] (lane 0 takes it, all lanes get it).
__device__ __forceinline__ int take_item(unsigned int* ctr) {
  unsigned int v = 0;
  if ((threadIdx.x & 31) == 0) v = atomicAdd(ctr, 1u);
  return (int)__shfl_sync(0xffffffffu, v, 0);
}

// The first / next work item of a warp: from the device counter, or, for deterministic
// plans, in a fixed order (warp w of the launch takes items w, w + warps, ...), so that every
// block's partial sums cover the same items in every run.
__device__ __forceinline__ int first_item(unsigned int* ctr, bool fixed) {
  return fixed ? (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) : take_item(ctr);
}
__device__ __forceinline__ int next_item(unsigned int* ctr, bool fixed, int cur) {
  return fixed ? cur + (int)(gridDim.x * (blockDim.x >> 5)) : take_item(ctr);
}

// Called by every thread of a block once its warps have taken their last item: the last
// block of the launch to get here resets the counter pair {next item, finished blocks} for
// the next launch (stream order makes the reset visible to it).
__device__ __forceinline__ void release_items(unsigned int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1u) == gridDim.x - 1) {
      atomicExch(ctr, 0u);
      atomicExch(ctr + 1, 0u);
    }
  }
}

// Copy the (T + J - 1)^2 half-spectrum window of a tile into a warp's shared window.  A
// tile whose window lies in columns [0, K/2] reads them directly; one lying wholly in
// (K/2, K) reads the mirrored cells conj(spec[(K - ky) mod K][K - kx]); both walk the rows
// with one lane per column.  Others (the window crosses column 0 or K/2) go cell by cell.
template <int J>
__device__ __forceinline__ void load_window_f32(float2* win, const float2* __restrict__ spec, int tile, int nT, int K,
                                                int lane, unsigned int* dbg = nullptr) {
  constexpr int P = kTile + J - 1;
  const int H = (K >> 1) + 1;
  const int ty = tile / nT, tx = tile - ty * nT;
  const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
  if (ox >= 0 && ox + P - 1 <= (K >> 1)) {
    if (lane < P) {
      const float2* src = spec + ox + lane;
#pragma unroll 5
      for (int r = 0; r < P; ++r) {
        const size_t q = (size_t)wrapK(oy + r, K) * H + ox + lane;
        if (GBRI_DCHECK(dbg, q < (size_t)K * H, kDbgSpec, q)) win[r * kWinPitch + lane] = __ldg(spec + q);
      }
    }
  } else if (ox > (K >> 1) && ox + P - 1 < K) {
    if (lane < P) {
      const float2* src = spec + (K - ox - lane);
#pragma unroll 5
      for (int r = 0; r < P; ++r) {
        const int ky = wrapK(oy + r, K);
        const size_t q = (size_t)(ky == 0 ? 0 : K - ky) * H + (K - ox - lane);
        if (!GBRI_DCHECK(dbg, q < (size_t)K * H, kDbgSpec, q)) continue;
        float2 v = __ldg(spec + q);
        v.y = -v.y;
        win[r * kWinPitch + lane] = v;
      }
    }
  } else {
    for (int i = lane; i < P * P; i += 32) {
      const int r = i / P, cc = i - r * P;
      const int ky = wrapK(oy + r, K), kx = wrapK(ox + cc, K);
      const bool mirror = kx > (K >> 1);
      const int sy = mirror ? (ky == 0 ? 0 : K - ky) : ky, sx = mirror ? K - kx : kx;
      const size_t q = (size_t)sy * H + sx;
      if (!GBRI_DCHECK(dbg, q < (size_t)K * H, kDbgSpec, q)) continue;
      float2 v = __ldg(spec + q);
      if (mirror) v.y = -v.y;
      win[r * kWinPitch + cc] = v;
    }
  }
}

// Degridding (G then W, Sec. 2), FP32 with polynomial taps.  As k_degrid: a warp takes a
// chunk (consecutive visibilities of one tile), reloads its private window when the tile
// changes, and walks the chunk one visibility per lane, kRun in flight:
//   v = w sum_{t'} wy[t'] sum_t wx[t] win[cy + t'][cx + t]
// in packed (re, im) arithmetic.  Chunks come from the counter ctr (dynamic).
template <int J, class Epi>
__global__ void __launch_bounds__(kThreads, 3)
    k_degrid_fast(VisGeom geo, const float2* __restrict__ spec, Epi epi, unsigned int* ctr) {
  static_assert(sizeof(typename Epi::real) == 4, "FP32 path only");
  using E = typename Epi::SElem;
  extern __shared__ float4 smem_df[];
  constexpr int P = kTile + J - 1;
  const int lane = threadIdx.x & 31;
  float2* win = reinterpret_cast<float2*>(smem_df) + (threadIdx.x >> 5) * (P * kWinPitch);
  const int S = 1 << geo.log2S;
  const float two_over_S = 2.f / (float)S;
  const int K = geo.K;
  const E* streams[2] = {Epi::kStreams > 0 ? epi.stream(0) : nullptr, Epi::kStreams > 1 ? epi.stream(1) : nullptr};
  epi.init();  // block barrier
  int cur_tile = -1;
  int c = first_item(ctr, geo.slots != nullptr);
  while (c < geo.n_chunks) {
    const int c_next = next_item(ctr, geo.slots != nullptr, c);
    const int4 ch = geo.chunks[c];
    const int lo = ch.y, cnt = ch.z;
    epi.begin_chunk(lo);  // warp-uniform
    for (int b0 = 0; b0 < cnt; b0 += 32 * kRun) {
      uint2 m[kRun];
      typename Epi::Pre pre[kRun];
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        const int i = b0 + lane + 32 * k;
        if (i < cnt && GBRI_DCHECK(geo.dbg, lo + i < geo.M, kDbgVis, lo + i)) {
          m[k] = geo.meta[lo + i];
          pre[k] = epi.pre_from(streams, lo + i);
        }
      }
      if (ch.x != cur_tile) {  // warp-uniform
        __syncwarp();
        load_window_f32<J>(win, spec, ch.x, geo.nT, K, lane, geo.dbg);
        cur_tile = ch.x;
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        const int i = b0 + lane + 32 * k;
        if (i >= cnt) break;
        float2 w[J];
        taps_xy<J>(geo.poly, m[k].x, S, two_over_S, w);
        const int cy = (int)(m[k].x >> 16) >> geo.log2S, cx = (int)(m[k].x & 0xffff) >> geo.log2S;
        const bool in_win = GBRI_DCHECK(geo.dbg, cy < kTile && cx < kTile, kDbgWindow, lo + i);
        const float2* base = win + (in_win ? cy * kWinPitch + cx : 0);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int tp = 0; tp < J; ++tp) {
          float2 row = mul2(f2(w[0].x), base[tp * kWinPitch]);
#pragma unroll
          for (int t = 1; t < J; ++t) row = fma2(f2(w[t].x), base[tp * kWinPitch + t], row);
          acc = fma2(f2(w[tp].y), row, acc);
        }
        epi.store(lo + i, pre[k], mul2(f2(__uint_as_float(m[k].y)), acc));
      }
    }
    c = c_next;
  }
  release_items(ctr);
  epi.finish();
}

// Gridding (W^T then G^T, Sec. 2), FP32 with polynomial taps.  As k_grid: a warp takes a
// gridding work item (a tile, or a piece of a heavy tile), one lane per run (consecutive
// visibilities of one cell, 32 distinct cells per warp round), sums w v wy[t'] wx[t] into a
// J x J register patch (packed (re, im) FMAs), adds it to the warp's shared accumulator
// (lanes of one instruction touch distinct cells; a warp barrier per tap orders
// overlapping patches), and flushes the accumulator after the item: plain stores inside
// the tile, vector atomics on the border and for the pieces of a cut tile.  The next
// round's run entries are loaded while the current round is summed.  Items come from the
// counter ctr (dynamic, heaviest first).  Two blocks per SM: the patch, the loads in flight
// and the tap evaluation fit in registers without spills at that occupancy (three blocks
// spilled and were slower; a deeper software pipeline of the visibility loads added
// instructions and was slower too).
template <int J, class Src>
__global__ void __launch_bounds__(kThreads, 2)
    k_grid_fast(VisGeom geo, float2* __restrict__ grid, Src src, unsigned int* ctr) {
  static_assert(sizeof(typename Src::real) == 4, "FP32 path only");
  extern __shared__ float4 smem_gf[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  float2* accs = reinterpret_cast<float2*>(smem_gf);
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) accs[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float2* acc = accs + (threadIdx.x >> 5) * (P * kAccPitch2);
  const int S = 1 << geo.log2S;
  const float two_over_S = 2.f / (float)S;
  const int K = geo.K;
  constexpr int lo_x = J - 1, hi_x = kTile;
  int it = first_item(ctr, geo.slots != nullptr);
  while (it < geo.n_gtiles) {
    const int it_next = next_item(ctr, geo.slots != nullptr, it);
    const int4 gt = geo.gtiles[it];
    const typename Src::Ctx sctx = src.ctx(geo.subruns[gt.y].x);  // a tile's first run is never padding
    int2 sr = geo.subruns[gt.y + lane];  // gt.z is a multiple of 32
    for (int b0 = 0; b0 < gt.z; b0 += 32) {
      const int2 sr_next = (b0 + 32 < gt.z) ? geo.subruns[gt.y + b0 + 32 + lane] : make_int2(0, 0);
      float2 pt[J][J];
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) pt[tp][t] = make_float2(0.f, 0.f);
      int a0 = 0;
      bool in_acc = true;
      for (int k0 = 0; k0 < sr.y; k0 += kRun) {
        uint2 m[kRun];
        float2 v[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k)
          if (k0 + k < sr.y && GBRI_DCHECK(geo.dbg, sr.x + k0 + k < geo.M, kDbgVis, sr.x + k0 + k)) {
            m[k] = geo.meta[sr.x + k0 + k];
            v[k] = src(sr.x + k0 + k, sctx);
          }
        if (k0 == 0) {
          const int cy = (int)(m[0].x >> 16) >> geo.log2S, cx = (int)(m[0].x & 0xffff) >> geo.log2S;
          in_acc = GBRI_DCHECK(geo.dbg, cy < kTile && cx < kTile, kDbgAccum, sr.x);
          a0 = in_acc ? cy * kAccPitch2 + cx : 0;
        }
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
          if (k0 + k >= sr.y) break;
          float2 w[J];
          taps_xy<J>(geo.poly, m[k].x, S, two_over_S, w);
          const float2 wv = mul2(f2(__uint_as_float(m[k].y)), v[k]);
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            const float2 b = mul2(f2(w[tp].y), wv);
#pragma unroll
            for (int t = 0; t < J; ++t) pt[tp][t] = fma2(f2(w[t].x), b, pt[tp][t]);
          }
        }
      }
      const bool active = sr.y > 0 && in_acc;
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (active) {
            float2* q = acc + a0 + tp * kAccPitch2 + t;
            *q = add2(*q, pt[tp][t]);
          }
          __syncwarp();
        }
      sr = sr_next;
    }
    const int ty = gt.x / geo.nT, tx = gt.x - ty * geo.nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    for (int i = lane; i < P * P; i += 32) {
      const int r = i / P, cc = i - r * P;
      float2* q = acc + r * kAccPitch2 + cc;
      const float2 a = *q;
      *q = make_float2(0.f, 0.f);
      if (geo.slots) {  // deterministic: the whole window to the item's slot
        if (GBRI_DCHECK(geo.dbg, it < geo.n_gtiles, kDbgSlot, it))
          static_cast<float2*>(geo.slots)[(size_t)it * (P * P) + i] = a;
        continue;
      }
      const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
      if (!GBRI_DCHECK(geo.dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
      float2* dst = grid + gq;
      if (gt.w == 0 && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) *dst = a;
      else if (a.x != 0.f || a.y != 0.f) atomicAdd(dst, a);
    }
    __syncwarp();  // the zeroed accumulator is visible to every lane before the next item
    it = it_next;
  }
  release_items(ctr);
}

// Degridding fused with the gridding of the updated dual (primal-dual iteration with a
// global ball, FISTA's residual; J = 4), FP32 with polynomial taps: as k_degrid_grid, one
// warp per gridding work item and one lane per run; the lane holds its cell's J x J window
// block in registers, and per visibility one tap evaluation serves both directions.  Two
// visibilities per lane in flight (the window block and the patch take 64 registers; four
// in flight spilled and ran 15 % slower).  Items come from the counter ctr (dynamic,
// heaviest first), so that blocks which start late -- the iteration's wavelet branch holds
// SMs when the kernel is launched -- take fewer items instead of stretching the kernel: with
// items in a fixed order the iteration took either 0.390 or 0.406 ms depending on how the two
// branches met, with the counter 0.386-0.388 ms, and the kernel alone 178 us against 207.
// Deterministic plans keep the fixed order (each block's partial of the ball norm then covers
// the same items in every run).
constexpr int kFusedRun = 2;
template <int J, class Epi>
__global__ void __launch_bounds__(kThreads, 2)
    k_degrid_grid_fast(VisGeom geo, const float2* __restrict__ spec, float2* __restrict__ grid, Epi epi,
                       unsigned int* ctr) {
  static_assert(sizeof(typename Epi::real) == 4, "FP32 path only");
  using E = typename Epi::SElem;
  extern __shared__ float4 smem_dgf[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  const int lane = threadIdx.x & 31;
  float2* wins = reinterpret_cast<float2*>(smem_dgf);
  float2* win = wins + (threadIdx.x >> 5) * (P * kWinPitch);
  float2* acc = wins + W * (P * kWinPitch) + (threadIdx.x >> 5) * (P * kAccPitch2);
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) wins[W * P * kWinPitch + i] = make_float2(0.f, 0.f);
  const int S = 1 << geo.log2S;
  const float two_over_S = 2.f / (float)S;
  const int K = geo.K;
  const E* streams[2] = {Epi::kStreams > 0 ? epi.stream(0) : nullptr, Epi::kStreams > 1 ? epi.stream(1) : nullptr};
  epi.init();  // block barrier: zeroed accumulators in place
  constexpr int lo_x = J - 1, hi_x = kTile;
  const bool fixed = geo.slots != nullptr;  // deterministic plans: the same block partials every run
  int it = first_item(ctr, fixed);
  while (it < geo.n_gtiles) {
    const int it_next = next_item(ctr, fixed, it);
    const int4 gt = geo.gtiles[it];
    int2 sr = geo.subruns[gt.y + lane];  // gt.z is a multiple of 32
    load_window_f32<J>(win, spec, gt.x, geo.nT, K, lane, geo.dbg);
    __syncwarp();
    for (int b0 = 0; b0 < gt.z; b0 += 32) {
      const int2 sr_next = (b0 + 32 < gt.z) ? geo.subruns[gt.y + b0 + 32 + lane] : make_int2(0, 0);
      float2 pt[J][J];
      float2 blk[J][J];
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) pt[tp][t] = make_float2(0.f, 0.f);
      int a0 = 0;
      bool in_win = true;
      for (int k0 = 0; k0 < sr.y; k0 += kFusedRun) {
        uint2 m[kFusedRun];
        typename Epi::Pre pre[kFusedRun];
#pragma unroll
        for (int k = 0; k < kFusedRun; ++k)
          if (k0 + k < sr.y && GBRI_DCHECK(geo.dbg, sr.x + k0 + k < geo.M, kDbgVis, sr.x + k0 + k)) {
            m[k] = geo.meta[sr.x + k0 + k];
            pre[k] = epi.pre_from(streams, sr.x + k0 + k);
          }
        if (k0 == 0) {  // the run's cell: its J x J block of the window
          const int cy = (int)(m[0].x >> 16) >> geo.log2S, cx = (int)(m[0].x & 0xffff) >> geo.log2S;
          in_win = GBRI_DCHECK(geo.dbg, cy < kTile && cx < kTile, kDbgWindow, sr.x);
          a0 = in_win ? cy * kWinPitch + cx : 0;
#pragma unroll
          for (int tp = 0; tp < J; ++tp)
#pragma unroll
            for (int t = 0; t < J; ++t) blk[tp][t] = win[a0 + tp * kWinPitch + t];
        }
#pragma unroll
        for (int k = 0; k < kFusedRun; ++k) {
          if (k0 + k >= sr.y) break;
          float2 w[J];
          taps_xy<J>(geo.poly, m[k].x, S, two_over_S, w);
          float2 dg = make_float2(0.f, 0.f);
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            float2 row = mul2(f2(w[0].x), blk[tp][0]);
#pragma unroll
            for (int t = 1; t < J; ++t) row = fma2(f2(w[t].x), blk[tp][t], row);
            dg = fma2(f2(w[tp].y), row, dg);
          }
          const float2 ww = f2(__uint_as_float(m[k].y));
          const float2 un = epi.update(sr.x + k0 + k, pre[k], mul2(ww, dg));
          const float2 wv = mul2(ww, un);
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            const float2 b = mul2(f2(w[tp].y), wv);
#pragma unroll
            for (int t = 0; t < J; ++t) pt[tp][t] = fma2(f2(w[t].x), b, pt[tp][t]);
          }
        }
      }
      const bool active = sr.y > 0 && in_win;
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (active) {
            float2* q = acc + a0 + tp * kAccPitch2 + t;
            *q = add2(*q, pt[tp][t]);
          }
          __syncwarp();
        }
      sr = sr_next;
    }
    const int ty = gt.x / geo.nT, tx = gt.x - ty * geo.nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    for (int i = lane; i < P * P; i += 32) {
      const int r = i / P, cc = i - r * P;
      float2* q = acc + r * kAccPitch2 + cc;
      const float2 a = *q;
      *q = make_float2(0.f, 0.f);
      if (geo.slots) {  // deterministic: the whole window to the item's slot
        if (GBRI_DCHECK(geo.dbg, it < geo.n_gtiles, kDbgSlot, it))
          static_cast<float2*>(geo.slots)[(size_t)it * (P * P) + i] = a;
        continue;
      }
      const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
      if (!GBRI_DCHECK(geo.dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
      float2* dst = grid + gq;
      if (gt.w == 0 && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) *dst = a;
      else if (a.x != 0.f || a.y != 0.f) atomicAdd(dst, a);
    }
    __syncwarp();  // window and zeroed accumulator visible to every lane before the next item
    it = it_next;
  }
  release_items(ctr);
  epi.finish();
}

}  // namespace gbri
