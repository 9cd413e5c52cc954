// Degridding (G, W) and gridding (G^T, W^T) kernels of Sec. 2 / Eq. 2 over the
// plan's tile-sorted visibilities, templated on the real type R (float: FP32 path,
// double: FP64 path).  Included by exactly one translation unit per precision
// (vis_f32.cu, vis_f64.cu), which instantiates every launch helper it needs.
#pragma once

#include <mutex>

#include "nufft.cuh"

namespace gbri {

// Degridding (G then W, Sec. 2).  Every warp works alone: it takes whole chunks (one
// contiguous range of at most kChunk visibilities of one 16 x 16 tile; warps stride
// over the chunk list) and copies the chunk's tile window ((T + J - 1)^2 grid values)
// into its private shared-memory window when the tile changes.  The grid is the FFT of a
// real image, held as its half spectrum spec[ky][kx], kx = 0 .. K/2 (row pitch K/2 + 1):
// a cell with kx > K/2 is read as conj(spec[(K - ky) mod K][K - kx]).  The warp walks the
// chunk 32 * kRun visibilities at a time, one per lane and kRun in flight per lane
// (metadata and epilogue loads issued before the window reload, coalesced):
//   v = w * sum_{t'} wy[t'] sum_t wx[t] win[cy + t'][cx + t]
// with the two J-tap weight rows from the block's shared table.  A cell's visibilities
// are consecutive, so neighbouring lanes often read the same window words.  No block-wide
// barrier after the table load.  `Epi` consumes (plan position, v).
template <int J, int TM, class Epi>
__global__ void __launch_bounds__(kThreads, degrid_occupancy(sizeof(typename Epi::real), J))
    k_degrid(VisGeom geo, const cplx<typename Epi::real>* __restrict__ spec, Epi epi) {
  using R = typename Epi::real;
  using C = cplx<R>;
  using E = typename Epi::SElem;
  extern __shared__ float4 smem_dg[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  static_assert(TM == kTapTable || TM == kTapFO, "table kernels (polynomial taps: k_degrid_fast)");
  R* sw = reinterpret_cast<R*>(smem_dg);
  const int S = 1 << geo.log2S;
  const int lane = threadIdx.x & 31;
  C* win = reinterpret_cast<C*>(sw + table_elems(S, J)) + (threadIdx.x >> 5) * (P * kWinPitch);
  copy_table_to_smem(sw, static_cast<const R*>(geo.wtab), table_elems(S, J));
  const int K = geo.K, H = (K >> 1) + 1;
  const E* streams[2] = {Epi::kStreams > 0 ? epi.stream(0) : nullptr, Epi::kStreams > 1 ? epi.stream(1) : nullptr};
  epi.init();  // includes a block barrier: the table is in place after it
  int cur_tile = -1;
  for (int c = blockIdx.x * W + (threadIdx.x >> 5); c < geo.n_chunks; c += gridDim.x * W) {
    const int4 ch = geo.chunks[c];
    const int lo = ch.y, cnt = ch.z;
    epi.begin_chunk(lo);  // warp-uniform
    for (int b0 = 0; b0 < cnt; b0 += 32 * kRun) {
      uint2 m[kRun];
      uint32_t fr[kRun];
      typename Epi::Pre pre[kRun];
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        const int i = b0 + lane + 32 * k;
        if (i < cnt && GBRI_DCHECK(geo.dbg, lo + i < geo.M, kDbgVis, lo + i)) {
          m[k] = geo.meta[lo + i];
          if constexpr (TM == kTapFO) fr[k] = geo.frac[lo + i];
          pre[k] = epi.pre_from(streams, lo + i);
        }
      }
      if (ch.x != cur_tile) {  // warp-uniform
        __syncwarp();
        const int ty = ch.x / geo.nT, tx = ch.x - ty * geo.nT;
        const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
        for (int i = lane; i < P * P; i += 32) {
          const int r = i / P, cc = i - r * P;
          const int ky = wrapK(oy + r, K), kx = wrapK(ox + cc, K);
          const bool mirror = kx > (K >> 1);
          const int sy = mirror ? (ky == 0 ? 0 : K - ky) : ky, sx = mirror ? K - kx : kx;
          const size_t q = (size_t)sy * H + sx;
          if (!GBRI_DCHECK(geo.dbg, q < (size_t)K * H, kDbgSpec, q)) continue;
          C v = __ldg(spec + q);
          if (mirror) v.y = -v.y;
          win[r * kWinPitch + cc] = v;
        }
        cur_tile = ch.x;
        __syncwarp();
      }
#pragma unroll
      for (int k = 0; k < kRun; ++k) {
        const int i = b0 + lane + 32 * k;
        if (i >= cnt) break;
        const int lx = m[k].x & 0xffff, ly = m[k].x >> 16;
        R wx[J], wy[J];
        if constexpr (TM == kTapFO) {
          load_taps_fo<J>(sw, lx & (S - 1), fr[k] & 0xff, S, wx);
          load_taps_fo<J>(sw, ly & (S - 1), fr[k] >> 8, S, wy);
        } else {
          load_taps<J>(sw, lx & (S - 1), S, wx);
          load_taps<J>(sw, ly & (S - 1), S, wy);
        }
        const bool in_win = GBRI_DCHECK(geo.dbg, (ly >> geo.log2S) < kTile && (lx >> geo.log2S) < kTile, kDbgWindow,
                                         lo + i);
        const C* base = win + (in_win ? (ly >> geo.log2S) * kWinPitch + (lx >> geo.log2S) : 0);
        R ar = 0, ai = 0;
#pragma unroll
        for (int tp = 0; tp < J; ++tp) {
          R rr = 0, ri = 0;
#pragma unroll
          for (int t = 0; t < J; ++t) {
            const C gv = base[tp * kWinPitch + t];
            rr = fma_r(wx[t], gv.x, rr);
            ri = fma_r(wx[t], gv.y, ri);
          }
          ar = fma_r(wy[tp], rr, ar);
          ai = fma_r(wy[tp], ri, ai);
        }
        const R w = (R)__uint_as_float(m[k].y);
        epi.store(lo + i, pre[k], mkc<R>(w * ar, w * ai));
      }
    }
  }
  epi.finish();
}

// Gridding (W^T then G^T, Sec. 2).  Every warp works alone: it takes whole tiles
// (heaviest first, warps striding over the tile list) and walks the tile's runs 32 at a
// time (each round of runs starts at a warp boundary, so the 32 lanes hold runs of 32
// distinct cells).  A lane takes one run (consecutive visibilities of one cell), loads it
// kRun visibilities at a time, sums w * v * wy[t'] wx[t] into a J x J register patch and
// adds the patch to the warp's private (T + J - 1)^2 accumulator in shared memory with
// plain read-modify-writes: the lanes of one instruction touch distinct cells and the
// warp's instructions are ordered, so no atomics are needed.  After the tile the warp
// writes its accumulator to the global grid (zeroing it for the next tile): plain stores
// for the cells no other tile touches, atomics for the border shared with the
// neighbouring tiles.  A heavy tile is cut into several items (whole 32-run groups, flag
// gt.w = 1), whose warps flush every cell with atomics.  No block-wide barrier after the
// table load.
// `Src` gives the visibility value at a plan position.
template <int J, int TM, class Src>
__global__ void __launch_bounds__(kThreads, grid_occupancy(sizeof(typename Src::real), J))
    k_grid(VisGeom geo, cplx<typename Src::real>* __restrict__ grid, Src src) {
  using R = typename Src::real;
  using C = cplx<R>;
  extern __shared__ float4 smem_gr[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  static_assert(TM == kTapTable || TM == kTapFO, "table kernels (polynomial taps: k_grid_fast)");
  const int S = 1 << geo.log2S;
  R* sw = reinterpret_cast<R*>(smem_gr);
  C* accs = reinterpret_cast<C*>(sw + table_elems(S, J));
  copy_table_to_smem(sw, static_cast<const R*>(geo.wtab), table_elems(S, J));
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) accs[i] = mkc<R>(0, 0);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  C* acc = accs + (threadIdx.x >> 5) * (P * kAccPitch2);
  const int K = geo.K;
  // accumulator rows / cols [lo_x, hi_x) belong to no other tile's window
  constexpr int lo_x = J - 1, hi_x = kTile;
  for (int it = blockIdx.x * W + (threadIdx.x >> 5); it < geo.n_gtiles; it += gridDim.x * W) {
    const int4 gt = geo.gtiles[it];
    const typename Src::Ctx sctx = src.ctx(geo.subruns[gt.y].x);  // a tile's first run is never padding
    for (int b0 = 0; b0 < gt.z; b0 += 32) {
      const int2 sr = geo.subruns[gt.y + b0 + lane];  // gt.z is a multiple of 32
      const bool active = sr.y > 0;
      C pt[J][J];
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) pt[tp][t] = mkc<R>(0, 0);
      int a0 = 0;
      bool in_acc = true;
      for (int k0 = 0; k0 < sr.y; k0 += kRun) {
        uint2 m[kRun];
        uint32_t fr[kRun];
        C v[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k)
          if (k0 + k < sr.y && GBRI_DCHECK(geo.dbg, sr.x + k0 + k < geo.M, kDbgVis, sr.x + k0 + k)) {
            m[k] = geo.meta[sr.x + k0 + k];
            if constexpr (TM == kTapFO) fr[k] = geo.frac[sr.x + k0 + k];
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
          R wx[J], wy[J];
          if constexpr (TM == kTapFO) {
            load_taps_fo<J>(sw, (m[k].x & 0xffff) & (S - 1), fr[k] & 0xff, S, wx);
            load_taps_fo<J>(sw, (m[k].x >> 16) & (S - 1), fr[k] >> 8, S, wy);
          } else {
            load_taps<J>(sw, (m[k].x & 0xffff) & (S - 1), S, wx);
            load_taps<J>(sw, (m[k].x >> 16) & (S - 1), S, wy);
          }
          const R w = (R)__uint_as_float(m[k].y);
          const R vr = w * v[k].x, vi = w * v[k].y;
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            const R br = wy[tp] * vr, bi = wy[tp] * vi;
#pragma unroll
            for (int t = 0; t < J; ++t) {
              pt[tp][t].x = fma_r(wx[t], br, pt[tp][t].x);
              pt[tp][t].y = fma_r(wx[t], bi, pt[tp][t].y);
            }
          }
        }
      }
      // all 32 lanes walk the taps in lockstep: within one tap the active lanes touch
      // distinct cells, and the warp barrier orders one tap's stores before the next
      // tap's loads (a neighbour cell's patch overlaps this one)
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (active && in_acc) {
            C* q = acc + a0 + tp * kAccPitch2 + t;
            const C o = *q;
            *q = mkc<R>(o.x + pt[tp][t].x, o.y + pt[tp][t].y);
          }
          __syncwarp();
        }
    }
    const int ty = gt.x / geo.nT, tx = gt.x - ty * geo.nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    for (int i = lane; i < P * P; i += 32) {
      const int r = i / P, cc = i - r * P;
      C* q = acc + r * kAccPitch2 + cc;
      const C a = *q;
      *q = mkc<R>(0, 0);
      if (geo.slots) {  // deterministic: the whole window to the item's slot
        if (GBRI_DCHECK(geo.dbg, it < geo.n_gtiles, kDbgSlot, it)) static_cast<C*>(geo.slots)[(size_t)it * (P * P) + i] = a;
        continue;
      }
      const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
      if (!GBRI_DCHECK(geo.dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
      C* dst = grid + gq;
      if (gt.w == 0 && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) {
        *dst = a;
      } else if (a.x != 0 || a.y != 0) {
        if constexpr (sizeof(R) == 4) {
          atomicAdd(dst, a);  // one vector atomic
        } else {
          atomicAdd(&dst->x, a.x);
          atomicAdd(&dst->y, a.y);
        }
      }
    }
    __syncwarp();  // the zeroed accumulator is visible to every lane before the next tile
  }
}

// Degridding fused with the gridding of the updated dual (primal-dual iteration, global
// ball; FISTA's residual; J = 4, FP32; FO: first-order table).  One warp per gridding work item (a tile, or a piece of
// a heavy tile), one lane per run (consecutive visibilities of one cell), as in k_grid.  A
// lane reads its cell's J x J window block from the warp's window once, then per
// visibility: the two tap rows (once, for both directions), v = w sum wy sum wx block,
// u <- c u + sigma2 (v - y) (stored; FP64 partials of ||u||^2), and the gridding patch
// += w u wy wx.  After the run the patch is added to the warp's accumulator; after the
// item the accumulator is flushed as in k_grid.  Gridding u as soon as it is updated is
// valid because Phi^dagger is applied to u itself (c scales the image later), so no global
// reduction separates the two passes.
template <int J, int TM, class Epi>
__global__ void __launch_bounds__(kThreads, 2)
    k_degrid_grid(VisGeom geo, const float2* __restrict__ spec, float2* __restrict__ grid, Epi epi) {
  static_assert(sizeof(typename Epi::real) == 4, "FP32 path only");
  using R = float;
  using C = float2;
  using E = typename Epi::SElem;
  extern __shared__ float4 smem_dgg[];
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  static_assert(TM == kTapTable || TM == kTapFO, "table kernels (polynomial taps: k_degrid_grid_fast)");
  R* sw = reinterpret_cast<R*>(smem_dgg);
  const int S = 1 << geo.log2S;
  const int lane = threadIdx.x & 31;
  C* wins = reinterpret_cast<C*>(sw + table_elems(S, J));
  C* win = wins + (threadIdx.x >> 5) * (P * kWinPitch);
  C* acc = wins + W * (P * kWinPitch) + (threadIdx.x >> 5) * (P * kAccPitch2);
  copy_table_to_smem(sw, static_cast<const R*>(geo.wtab), table_elems(S, J));
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) wins[W * P * kWinPitch + i] = mkc<R>(0, 0);
  const int K = geo.K, H = (K >> 1) + 1;
  const E* streams[2] = {Epi::kStreams > 0 ? epi.stream(0) : nullptr, Epi::kStreams > 1 ? epi.stream(1) : nullptr};
  epi.init();  // includes a block barrier: table and zeroed accumulators in place
  constexpr int lo_x = J - 1, hi_x = kTile;
  for (int it = blockIdx.x * W + (threadIdx.x >> 5); it < geo.n_gtiles; it += gridDim.x * W) {
    const int4 gt = geo.gtiles[it];
    const int ty = gt.x / geo.nT, tx = gt.x - ty * geo.nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    for (int i = lane; i < P * P; i += 32) {  // the tile's window of the half spectrum
      const int r = i / P, cc = i - r * P;
      const int ky = wrapK(oy + r, K), kx = wrapK(ox + cc, K);
      const bool mirror = kx > (K >> 1);
      const int sy = mirror ? (ky == 0 ? 0 : K - ky) : ky, sx = mirror ? K - kx : kx;
      const size_t q = (size_t)sy * H + sx;
      if (!GBRI_DCHECK(geo.dbg, q < (size_t)K * H, kDbgSpec, q)) continue;
      C v = __ldg(spec + q);
      if (mirror) v.y = -v.y;
      win[r * kWinPitch + cc] = v;
    }
    __syncwarp();
    for (int b0 = 0; b0 < gt.z; b0 += 32) {
      const int2 sr = geo.subruns[gt.y + b0 + lane];  // gt.z is a multiple of 32
      const bool active = sr.y > 0;
      C pt[J][J];
      C blk[J][J];
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) pt[tp][t] = mkc<R>(0, 0);
      int a0 = 0;
      bool in_acc = true;
      for (int k0 = 0; k0 < sr.y; k0 += kRun) {
        uint2 m[kRun];
        uint32_t fr[kRun];
        typename Epi::Pre pre[kRun];
#pragma unroll
        for (int k = 0; k < kRun; ++k)
          if (k0 + k < sr.y && GBRI_DCHECK(geo.dbg, sr.x + k0 + k < geo.M, kDbgVis, sr.x + k0 + k)) {
            m[k] = geo.meta[sr.x + k0 + k];
            if constexpr (TM == kTapFO) fr[k] = geo.frac[sr.x + k0 + k];
            pre[k] = epi.pre_from(streams, sr.x + k0 + k);
          }
        if (k0 == 0) {  // the run's cell: its J x J block of the window
          const int cy = (int)(m[0].x >> 16) >> geo.log2S, cx = (int)(m[0].x & 0xffff) >> geo.log2S;
          in_acc = GBRI_DCHECK(geo.dbg, cy < kTile && cx < kTile, kDbgWindow, sr.x);
          a0 = in_acc ? cy * kWinPitch + cx : 0;
#pragma unroll
          for (int tp = 0; tp < J; ++tp)
#pragma unroll
            for (int t = 0; t < J; ++t) blk[tp][t] = win[a0 + tp * kWinPitch + t];
        }
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
          if (k0 + k >= sr.y) break;
          R wx[J], wy[J];
          if constexpr (TM == kTapFO) {
            load_taps_fo<J>(sw, (m[k].x & 0xffff) & (S - 1), fr[k] & 0xff, S, wx);
            load_taps_fo<J>(sw, (m[k].x >> 16) & (S - 1), fr[k] >> 8, S, wy);
          } else {
            load_taps<J>(sw, (m[k].x & 0xffff) & (S - 1), S, wx);
            load_taps<J>(sw, (m[k].x >> 16) & (S - 1), S, wy);
          }
          R ar = 0, ai = 0;
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            R rr = 0, ri = 0;
#pragma unroll
            for (int t = 0; t < J; ++t) {
              rr = fma_r(wx[t], blk[tp][t].x, rr);
              ri = fma_r(wx[t], blk[tp][t].y, ri);
            }
            ar = fma_r(wy[tp], rr, ar);
            ai = fma_r(wy[tp], ri, ai);
          }
          const R w = __uint_as_float(m[k].y);
          const C un = epi.update(sr.x + k0 + k, pre[k], mkc<R>(w * ar, w * ai));
          const R vr = w * un.x, vi = w * un.y;
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            const R br = wy[tp] * vr, bi = wy[tp] * vi;
#pragma unroll
            for (int t = 0; t < J; ++t) {
              pt[tp][t].x = fma_r(wx[t], br, pt[tp][t].x);
              pt[tp][t].y = fma_r(wx[t], bi, pt[tp][t].y);
            }
          }
        }
      }
      // lanes hold distinct cells within one tap; the warp barrier orders neighbouring patches
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (active && in_acc) {
            C* q = acc + a0 + tp * kAccPitch2 + t;
            const C o = *q;
            *q = mkc<R>(o.x + pt[tp][t].x, o.y + pt[tp][t].y);
          }
          __syncwarp();
        }
    }
    for (int i = lane; i < P * P; i += 32) {
      const int r = i / P, cc = i - r * P;
      C* q = acc + r * kAccPitch2 + cc;
      const C a = *q;
      *q = mkc<R>(0, 0);
      if (geo.slots) {  // deterministic: the whole window to the item's slot
        if (GBRI_DCHECK(geo.dbg, it < geo.n_gtiles, kDbgSlot, it)) static_cast<C*>(geo.slots)[(size_t)it * (P * P) + i] = a;
        continue;
      }
      const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
      if (!GBRI_DCHECK(geo.dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
      C* dst = grid + gq;
      if (gt.w == 0 && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) *dst = a;
      else if (a.x != 0 || a.y != 0) atomicAdd(dst, a);
    }
    __syncwarp();  // window and zeroed accumulator visible to every lane before the next item
  }
  epi.finish();
}

inline size_t degrid_grid_smem(const gbri_plan* p) {
  return (size_t)smem_table_elems(p->tap_mode, p->S, p->J) * sizeof(float) +
         (size_t)(kThreads / 32) * (kTile + p->J - 1) * (kWinPitch + kAccPitch2) * sizeof(float2);
}

// Deterministic gridding, second pass: every grid cell is the sum of the item windows that
// cover it, in a fixed order (the tile above / left before the tile itself along each axis,
// a tile's items in index order); cells no window covers are zero.  The window of tile t
// starts at cell t T - (J/2 - 1) and spans T + J - 1 cells (periodic), so along one axis a
// cell lies in the window of tile t_a = floor((k + J/2 - 1) / T) at offset k + J/2 - 1 - t_a T,
// and also in tile t_a - 1's at that offset + T when the offset is below J - 1.
template <class R>
__global__ void k_grid_reduce(const cplx<R>* __restrict__ slots, const int32_t* __restrict__ toff,
                              const int32_t* __restrict__ titems, cplx<R>* __restrict__ grid, int K, int nT, int J) {
  const int P = kTile + J - 1, hb = J / 2 - 1;
  const int64_t cells = (int64_t)K * K;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < cells; q += (int64_t)gridDim.x * blockDim.x) {
    const int ky = (int)(q / K), kx = (int)(q - (int64_t)ky * K);
    int ty[2], oy[2], ny = 0, tx[2], ox[2], nx = 0;
    {
      const int ta = (ky + hb) / kTile, ra = ky + hb - ta * kTile;
      if (ra < J - 1) { ty[ny] = (ta - 1 + nT) % nT; oy[ny++] = ra + kTile; }
      ty[ny] = ta % nT; oy[ny++] = ra;
    }
    {
      const int ta = (kx + hb) / kTile, ra = kx + hb - ta * kTile;
      if (ra < J - 1) { tx[nx] = (ta - 1 + nT) % nT; ox[nx++] = ra + kTile; }
      tx[nx] = ta % nT; ox[nx++] = ra;
    }
    R sr = 0, si = 0;
    for (int a = 0; a < ny; ++a)
      for (int b = 0; b < nx; ++b) {
        const int t = ty[a] * nT + tx[b];
        const int w = oy[a] * P + ox[b];
        for (int j = toff[t]; j < toff[t + 1]; ++j) {
          const cplx<R> v = slots[(size_t)titems[j] * (P * P) + w];
          sr += v.x;
          si += v.y;
        }
      }
    grid[q] = mkc<R>(sr, si);
  }
}

template <class R>
int32_t launch_grid_reduce(gbri_plan* p, cudaStream_t s) {
  launch_begin(GBRI_K_GRID, s);
  const int64_t cells = (int64_t)p->K * p->K;
  const int blocks = (int)std::min<int64_t>(ceil_div(cells, 256), (int64_t)num_sms() * 16);
  k_grid_reduce<R><<<blocks, 256, 0, s>>>(p->as<const cplx<R>>(p->slots), p->tile_items_off, p->tile_items,
                                          p->as<cplx<R>>(p->grid), p->K, p->nT, p->J);
  return launch_end(GBRI_K_GRID, s);
}

template <class Epi>
int32_t launch_degrid(gbri_plan* p, Epi epi, cudaStream_t s) {
  using R = typename Epi::real;
  if constexpr (sizeof(R) == 4)
    if (p->tap_mode == kTapPoly) return launch_degrid_fast(p, epi, s);
  launch_begin(GBRI_K_DEGRID, s);
  const cplx<R>* g = p->as<cplx<R>>(p->spec);
  const size_t sm = degrid_smem(p);
  const VisGeom geo = vis_geom(p);
  const int tm = p->tap_mode;
  if (tm == kTapFO) {
    if (p->J == 4) k_degrid<4, kTapFO, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi);
    else k_degrid<6, kTapFO, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi);
  } else {
    if (p->J == 4) k_degrid<4, kTapTable, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi);
    else k_degrid<6, kTapTable, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi);
  }
  return launch_end(GBRI_K_DEGRID, s);
}

template <class Src>
int32_t launch_grid_generic(gbri_plan* p, Src src, cudaStream_t s);

template <class Src>
int32_t launch_grid(gbri_plan* p, Src src, cudaStream_t s, bool zeroed) {
  using R = typename Src::real;
  cplx<R>* g = p->as<cplx<R>>(p->grid);
  if (p->det) {  // the item windows go to slots; the fixed-order pass writes every cell
    if (p->n_gtiles > 0) {
      if constexpr (sizeof(R) == 4) {
        if (p->tap_mode == kTapPoly) GBRI_TRY(launch_grid_fast(p, src, s));
        else GBRI_TRY(launch_grid_generic(p, src, s));
      } else {
        GBRI_TRY(launch_grid_generic(p, src, s));
      }
    }
    return launch_grid_reduce<R>(p, s);
  }
  if (!zeroed) GBRI_CHECK_CUDA(cudaMemsetAsync(g, 0, sizeof(cplx<R>) * (size_t)p->K * p->K, s));
  if (p->n_gtiles == 0) return GBRI_OK;
  if constexpr (sizeof(R) == 4)
    if (p->tap_mode == kTapPoly) return launch_grid_fast(p, src, s);
  return launch_grid_generic(p, src, s);
}

template <class Src>
int32_t launch_grid_generic(gbri_plan* p, Src src, cudaStream_t s) {
  using R = typename Src::real;
  cplx<R>* g = p->as<cplx<R>>(p->grid);
  launch_begin(GBRI_K_GRID, s);
  const VisGeom geo = vis_geom(p);
  const int tm = p->tap_mode;
  if (tm == kTapFO) {
    if (p->J == 4) k_grid<4, kTapFO, Src><<<p->grid_blocks, kThreads, grid_smem(p), s>>>(geo, g, src);
    else k_grid<6, kTapFO, Src><<<p->grid_blocks, kThreads, grid_smem(p), s>>>(geo, g, src);
  } else {
    if (p->J == 4) k_grid<4, kTapTable, Src><<<p->grid_blocks, kThreads, grid_smem(p), s>>>(geo, g, src);
    else k_grid<6, kTapTable, Src><<<p->grid_blocks, kThreads, grid_smem(p), s>>>(geo, g, src);
  }
  return launch_end(GBRI_K_GRID, s);
}

// Shared-memory attributes of the FP32 polynomial-tap kernels (defined with them).
cudaError_t prepare_fast_kernels();

// Dynamic shared memory above 48 KB needs a per-kernel attribute; it is set once
// for every instantiation of one precision before any launch (so never inside a
// stream capture).
template <class R>
int32_t prepare_visibility_kernels() {
  static int32_t status = -100;
  static std::once_flag once;
  std::call_once(once, [] {
    const int lim = 220 * 1024;
    cudaError_t e = cudaSuccess;
#define GBRI_ATTR(kern) if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
#define GBRI_ATTR4(K, T) GBRI_ATTR((K<4, kTapTable, T<R>>)); GBRI_ATTR((K<6, kTapTable, T<R>>)); \
                         GBRI_ATTR((K<4, kTapFO, T<R>>)); GBRI_ATTR((K<6, kTapFO, T<R>>))
    GBRI_ATTR4(k_degrid, EpiStorePlan); GBRI_ATTR4(k_degrid, EpiStoreRaw); GBRI_ATTR4(k_degrid, EpiPD1);
    GBRI_ATTR4(k_degrid, EpiADMM1); GBRI_ATTR4(k_degrid, EpiResid); GBRI_ATTR4(k_degrid, EpiPD1L);
    GBRI_ATTR4(k_degrid, EpiADMM1L);
    GBRI_ATTR4(k_grid, SrcScaledL); GBRI_ATTR4(k_grid, SrcADMM2L); GBRI_ATTR4(k_grid, SrcPlan);
    GBRI_ATTR4(k_grid, SrcRaw); GBRI_ATTR4(k_grid, SrcADMM2);
#undef GBRI_ATTR4
    if constexpr (sizeof(R) == 4) {
      GBRI_ATTR((k_degrid_grid<4, kTapTable, EpiPD1<float>>));
      GBRI_ATTR((k_degrid_grid<4, kTapTable, EpiResid<float>>));
      GBRI_ATTR((k_degrid_grid<4, kTapFO, EpiPD1<float>>));
      GBRI_ATTR((k_degrid_grid<4, kTapFO, EpiResid<float>>));
    }
#undef GBRI_ATTR
    if constexpr (sizeof(R) == 4)
      if (e == cudaSuccess) e = prepare_fast_kernels();
    status = (e == cudaSuccess) ? GBRI_OK : cuda_error(e, "cudaFuncSetAttribute");
  });
  return status;
}

}  // namespace gbri

// Instantiates every visibility launch helper of real type R (one translation unit per R).
#define GBRI_INSTANTIATE_VIS(R)                                                              \
  namespace gbri {                                                                           \
  template int32_t launch_degrid<EpiStorePlan<R>>(gbri_plan*, EpiStorePlan<R>, cudaStream_t); \
  template int32_t launch_degrid<EpiStoreRaw<R>>(gbri_plan*, EpiStoreRaw<R>, cudaStream_t);   \
  template int32_t launch_degrid<EpiPD1<R>>(gbri_plan*, EpiPD1<R>, cudaStream_t);             \
  template int32_t launch_degrid<EpiADMM1<R>>(gbri_plan*, EpiADMM1<R>, cudaStream_t);         \
  template int32_t launch_degrid<EpiResid<R>>(gbri_plan*, EpiResid<R>, cudaStream_t);         \
  template int32_t launch_degrid<EpiPD1L<R>>(gbri_plan*, EpiPD1L<R>, cudaStream_t);           \
  template int32_t launch_degrid<EpiADMM1L<R>>(gbri_plan*, EpiADMM1L<R>, cudaStream_t);       \
  template int32_t launch_grid<SrcScaledL<R>>(gbri_plan*, SrcScaledL<R>, cudaStream_t, bool); \
  template int32_t launch_grid<SrcADMM2L<R>>(gbri_plan*, SrcADMM2L<R>, cudaStream_t, bool);   \
  template int32_t launch_grid<SrcPlan<R>>(gbri_plan*, SrcPlan<R>, cudaStream_t, bool);       \
  template int32_t launch_grid<SrcRaw<R>>(gbri_plan*, SrcRaw<R>, cudaStream_t, bool);         \
  template int32_t launch_grid<SrcADMM2<R>>(gbri_plan*, SrcADMM2<R>, cudaStream_t, bool);     \
  template int32_t prepare_visibility_kernels<R>();                                           \
  }
