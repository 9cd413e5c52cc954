// Step-major visibility kernels of Sec. 2 / Eq. 2 for FP32 plans with polynomial taps and
// J = 4 (the plan's "step layout").
//
// Layout.  A tile's runs (consecutive visibilities of one cell) are taken 32 at a time, as
// the plan lists them (round by round, banded by length, spread over bank slots): such a
// group is one warp's, a run per lane, 32 distinct cells.  The group's visibilities are
// stored step-major: step k holds the k-th visibility of every run longer than k, in lane
// order.  steps[s] = {pos | start << 31, mask}: the plan position of the first visibility of
// step s, bit 31 set on the first step of a group, and the lanes that hold a visibility at
// this step (the runs longer than k).  Lane j's visibility of step s is at
// pos + popc(mask & lanes below j).  So every step of a warp reads consecutive positions
// (one coalesced request per stream), and a warp walks its work item step by step.
//
// Staging.  The metadata and the plan-order streams a step needs (the epilogue's u and y,
// the gridding source) are copied into a per-warp ring of kStageDepth steps in shared
// memory with cp.async, that many steps ahead of their use; each lane copies and later
// reads only its own column, so a lane waits on its own copies only (cp.async.wait_group).
// Up to kStageDepth steps of loads are in flight per warp without holding registers.
//
// Modes: gridding only (a source gives the value at a position: Phi^dagger, the power
// method, ADMM and the local-ball dual) and gridding fused with degridding (the
// primal-dual dual update or FISTA's residual: each visibility's taps serve both
// directions).  Lanes keep their cell's J x J window block (fused) and J x J patch in
// registers for the whole run; the patch goes to the warp's shared accumulator at the end of
// the group, the accumulator to the grid at the end of the work item (plain stores inside
// the tile, vector atomics on the border and for pieces of a cut tile; deterministic plans
// write the whole window to the item's slot).  The operator's own degridding (Phi) keeps
// the chunk kernel k_degrid_fast, whose lanes take one visibility each in any order inside
// a tile: on the step layout's items it was 1.7x slower (one run per lane leaves lanes idle
// where runs differ in length, and the step bookkeeping adds instructions to a short loop).
#pragma once

#include "vis_fast.cuh"

namespace gbri {

enum StepMode { kStepGrid = 0, kStepFused = 1 };
// Steps in flight per warp (a power of two).  Depths 8 and 16 measured the same as 4: the
// kernels are bound by instruction issue once the loads are coalesced and staged.
constexpr int kStageDepth = 4;

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
template <class T>
__device__ __forceinline__ void cp_async_elem(void* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "staged elements are 4 or 8 bytes");
  if constexpr (sizeof(T) == 8) cp_async8(smem, gmem);
  else cp_async4(smem, gmem);
}

__device__ __forceinline__ int2 shfl_int2(int2 v, int src) {
  return make_int2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// A gridding source whose value at a position is one plan-order complex number (times a
// per-item factor) can be staged: SrcPlan (y[pos]) and SrcScaledL (c_j u[pos]).  Other
// sources are evaluated where the visibility is used.
template <class Src>
struct SrcStage {
  static constexpr bool kOn = false;
};
template <>
struct SrcStage<SrcPlan<float>> {
  static constexpr bool kOn = true;
  __device__ static const float2* ptr(const SrcPlan<float>& s) { return s.y; }
  __device__ static float2 value(const SrcPlan<float>&, float2 v, const NoCtx&) { return v; }
};
template <>
struct SrcStage<SrcScaledL<float>> {
  static constexpr bool kOn = true;
  __device__ static const float2* ptr(const SrcScaledL<float>& s) { return s.u; }
  __device__ static float2 value(const SrcScaledL<float>&, float2 v, const SrcScaledL<float>::Ctx& x) {
    return make_float2(x.c * v.x, x.c * v.y);
  }
};

// The per-item context of a gridding source (nothing for an epilogue).
template <class Op, bool IsSrc>
struct StepCtx {
  using type = typename Op::Ctx;
};
template <class Op>
struct StepCtx<Op, false> {
  struct type {};
};

// Streams staged beside the metadata: the epilogue's (degridding modes) or the source's.
template <int Mode, class Op>
constexpr int step_streams() {
  if constexpr (Mode == kStepFused) return Op::kStreams;
  else return SrcStage<Op>::kOn ? 1 : 0;
}

// Shared memory of a step kernel: per warp a window (fused mode), an accumulator and the
// staging ring (8-byte columns).
template <int Mode, class Op>
constexpr size_t step_smem() {
  constexpr int P = kTile + 4 - 1;
  constexpr int W = kThreads / 32;
  constexpr int NA = 1 + step_streams<Mode, Op>();
  return (size_t)W * ((Mode == kStepFused ? P * kWinPitch : 0) + P * kAccPitch2) * 8 +
         (size_t)W * kStageDepth * NA * 32 * 8;
}

template <int Mode, class Op>
__global__ void __launch_bounds__(kThreads, Mode == kStepGrid ? 3 : 2)
    k_steps(VisGeom geo, const float2* __restrict__ spec, float2* __restrict__ grid, Op op, unsigned int* ctr) {
  constexpr int J = 4;
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  constexpr int D = kStageDepth;
  constexpr bool kDg = Mode == kStepFused;  // degridding with the epilogue's update first
  constexpr int NS = step_streams<Mode, Op>();
  constexpr int NA = 1 + NS;
  static_assert(sizeof(typename Op::real) == 4, "FP32 path only");
  extern __shared__ float4 smem_steps[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* base = reinterpret_cast<float2*>(smem_steps);
  float2* win = base + warp * (P * kWinPitch);
  float2* accs = base + (kDg ? W * P * kWinPitch : 0);
  float2* acc = accs + warp * (P * kAccPitch2);
  uint2* stg = reinterpret_cast<uint2*>(accs + W * P * kAccPitch2) + warp * (D * NA * 32);
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) accs[i] = make_float2(0.f, 0.f);
  // the staged streams (element types of the epilogue or the source)
  const void* sp[2] = {nullptr, nullptr};
  if constexpr (kDg) {
    if constexpr (NS > 0) sp[0] = op.stream(0);
    if constexpr (NS > 1) sp[1] = op.stream(1);
  } else if constexpr (NS > 0) {
    sp[0] = SrcStage<Op>::ptr(op);
  }
  if constexpr (kDg) op.init();  // block barrier
  else __syncthreads();
  const int S = 1 << geo.log2S;
  const float two_over_S = 2.f / (float)S;
  const int K = geo.K;
  constexpr int lo_x = J - 1, hi_x = kTile;
  const unsigned lanes_below = (1u << lane) - 1u;
  const bool fixed = geo.slots != nullptr;  // deterministic plans: the same items per warp every run

  // copies of step descriptor d into ring slot q (this lane's column, if it holds a visibility)
  auto issue = [&](int q, int2 d) {
    if ((((unsigned)d.y) >> lane) & 1u) {
      const int pos = (d.x & 0x7fffffff) + __popc((unsigned)d.y & lanes_below);
      if (GBRI_DCHECK(geo.dbg, pos < geo.M, kDbgVis, pos)) {
        uint2* col = stg + (q * NA) * 32 + lane;
        cp_async8(col, geo.meta + pos);
        if constexpr (kDg) {
          using E = typename Op::SElem;
          if constexpr (NS > 0) cp_async_elem(col + 32, static_cast<const E*>(sp[0]) + pos);
          if constexpr (NS > 1) cp_async_elem(col + 64, static_cast<const E*>(sp[1]) + pos);
        } else if constexpr (NS > 0) {
          cp_async8(col + 32, static_cast<const float2*>(sp[0]) + pos);
        }
      }
    }
  };

  int it = first_item(ctr, fixed);
  while (it < geo.n_gtiles) {
    const int it_next = next_item(ctr, fixed, it);
    const int4 gt = geo.gtiles[it];  // {tile, first step, steps, split}
    const int s0 = gt.y, ns = gt.z;
    // step descriptors: lane j holds step 32 b + j of the current batch b and of the next
    int2 dcur = lane < ns ? geo.steps[s0 + lane] : make_int2(0, 0);
    int2 dnxt = 32 + lane < ns ? geo.steps[s0 + 32 + lane] : make_int2(0, 0);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const int2 d = shfl_int2(dcur, q);
      if (q < ns) issue(q, d);
      cp_async_commit();
    }
    if constexpr (kDg) {
      load_window_f32<J>(win, spec, gt.x, geo.nT, K, lane, geo.dbg);
      __syncwarp();
    }
    typename StepCtx<Op, !kDg>::type sctx{};
    if constexpr (!kDg) sctx = op.ctx(__shfl_sync(0xffffffffu, dcur.x, 0) & 0x7fffffff);
    if constexpr (kDg) op.begin_chunk(__shfl_sync(0xffffffffu, dcur.x, 0) & 0x7fffffff);
    float2 pt[J][J];
    float2 blk[J][J];
#pragma unroll
    for (int tp = 0; tp < J; ++tp)
#pragma unroll
      for (int t = 0; t < J; ++t) pt[tp][t] = make_float2(0.f, 0.f);
    int a0 = 0;
    bool has = false;  // this lane holds a run in the current group (and its cell is in the tile)
    // two steps per trip give the scheduler independent work from both (fused pass 172 -> 168 us,
    // gridding 123 -> 119 us; no spills)
#pragma unroll 2
    for (int i = 0; i < ns; ++i) {
      if (i > 0 && (i & 31) == 0) {  // next batch of descriptors (warp-uniform)
        dcur = dnxt;
        dnxt = i + 32 + lane < ns ? geo.steps[s0 + i + 32 + lane] : make_int2(0, 0);
      }
      const int2 d = shfl_int2(dcur, i & 31);
      const bool start = d.x < 0;
      {
        if (start && i > 0) {  // the previous group's patches into the accumulator
#pragma unroll
          for (int tp = 0; tp < J; ++tp)
#pragma unroll
            for (int t = 0; t < J; ++t) {
              if (has) {
                float2* q = acc + a0 + tp * kAccPitch2 + t;
                *q = add2(*q, pt[tp][t]);
              }
              pt[tp][t] = make_float2(0.f, 0.f);
              __syncwarp();
            }
        }
      }
      cp_async_wait<D - 1>();  // this lane's copies of step i have landed
      const int q = i & (D - 1);
      const bool act = ((((unsigned)d.y) >> lane) & 1u) != 0u;
      const uint2* col = stg + (q * NA) * 32 + lane;
      if (act) {
        const int pos = (d.x & 0x7fffffff) + __popc((unsigned)d.y & lanes_below);
        const uint2 m = col[0];
        if (start) {  // the run's cell: window block / accumulator offset
          const int cy = (int)(m.x >> 16) >> geo.log2S, cx = (int)(m.x & 0xffff) >> geo.log2S;
          has = GBRI_DCHECK(geo.dbg, cy < kTile && cx < kTile, kDbgAccum, pos);
          a0 = has ? cy * kWinPitch + cx : 0;
          if constexpr (kDg) {
#pragma unroll
            for (int tp = 0; tp < J; ++tp)
#pragma unroll
              for (int t = 0; t < J; ++t) blk[tp][t] = win[a0 + tp * kWinPitch + t];
          }
        }
        float2 w[J];
        taps_xy<J>(geo.poly, m.x, S, two_over_S, w);
        const float2 wt = f2(__uint_as_float(m.y));
        float2 wv;
        if constexpr (kDg) {
          float2 dg = make_float2(0.f, 0.f);
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            float2 row = mul2(f2(w[0].x), blk[tp][0]);
#pragma unroll
            for (int t = 1; t < J; ++t) row = fma2(f2(w[t].x), blk[tp][t], row);
            dg = fma2(f2(w[tp].y), row, dg);
          }
          using E = typename Op::SElem;
          const E* pe[2] = {reinterpret_cast<const E*>(col + 32), reinterpret_cast<const E*>(col + 64)};
          const typename Op::Pre pre = op.pre_from(pe, 0);
          wv = mul2(wt, op.update(pos, pre, mul2(wt, dg)));
        } else {
          float2 v;
          if constexpr (NS > 0) v = SrcStage<Op>::value(op, *reinterpret_cast<const float2*>(col + 32), sctx);
          else v = op(pos, sctx);
          wv = mul2(wt, v);
        }
        {
#pragma unroll
          for (int tp = 0; tp < J; ++tp) {
            const float2 b = mul2(f2(w[tp].y), wv);
#pragma unroll
            for (int t = 0; t < J; ++t) pt[tp][t] = fma2(f2(w[t].x), b, pt[tp][t]);
          }
        }
      } else if (start) {
        has = false;
      }
      // refill slot q with step i + D (its descriptor is in this batch or the next)
      const int i2 = i + D;
      const int2 d2 = shfl_int2(((i2 >> 5) == (i >> 5)) ? dcur : dnxt, i2 & 31);
      if (i2 < ns) issue(q, d2);
      cp_async_commit();
    }
    {
#pragma unroll
      for (int tp = 0; tp < J; ++tp)
#pragma unroll
        for (int t = 0; t < J; ++t) {
          if (has && ns > 0) {
            float2* q = acc + a0 + tp * kAccPitch2 + t;
            *q = add2(*q, pt[tp][t]);
          }
          __syncwarp();
        }
      const int ty = gt.x / geo.nT, tx = gt.x - ty * geo.nT;
      const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
      for (int e = lane; e < P * P; e += 32) {
        const int r = e / P, cc = e - r * P;
        float2* q = acc + r * kAccPitch2 + cc;
        const float2 a = *q;
        *q = make_float2(0.f, 0.f);
        if (geo.slots) {  // deterministic: the whole window to the item's slot
          if (GBRI_DCHECK(geo.dbg, it < geo.n_gtiles, kDbgSlot, it))
            static_cast<float2*>(geo.slots)[(size_t)it * (P * P) + e] = a;
          continue;
        }
        const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + cc, K);
        if (!GBRI_DCHECK(geo.dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
        float2* dst = grid + gq;
        if (gt.w == 0 && r >= lo_x && r < hi_x && cc >= lo_x && cc < hi_x) *dst = a;
        else if (a.x != 0.f || a.y != 0.f) atomicAdd(dst, a);
      }
    }
    __syncwarp();  // window, zeroed accumulator and ring visible to every lane before the next item
    it = it_next;
  }
  cp_async_wait<0>();
  release_items(ctr);
  if constexpr (kDg) op.finish();
}

}  // namespace gbri

namespace gbri {

// ---- the fused pass over several problems in one launch (batch executor) ----------------
// Every member is a primal-dual solver with a global l2 ball on an FP32 step-layout plan with
// the same kernel polynomial; its gridding work items are numbered after the previous
// members' (item0), and the warps take items of all members from one counter, heaviest
// members first.  Per visibility the arithmetic is the single-problem pass's (EpiPD1): u <- c u
// + sigma2 (Phi xhat - y), stored and gridded; each member's sum of |u|^2 is accumulated in
// FP64 per item and added to its slot of `sums`, and the launch's last block turns every
// slot into the member's ball scalar c = 1 - min(1, eps / dist), dist = sqrt(sum) / sigma2,
// and clears the slot.

__global__ void __launch_bounds__(kThreads, 2)
    k_steps_multi(const FusedMember* __restrict__ mem, int n_mem, int n_items, double* __restrict__ sums,
                  PolyTaps poly, unsigned int* ctr) {
  constexpr int J = 4;
  constexpr int P = kTile + J - 1;
  constexpr int W = kThreads / 32;
  constexpr int D = kStageDepth;
  constexpr int NA = 3;  // metadata, u, y
  extern __shared__ float4 smem_multi[];
  __shared__ int s_item0[kMaxFusedMembers + 1];
  __shared__ const void* s_ptr[W][3];  // the current item's member: meta, u, y
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2* base = reinterpret_cast<float2*>(smem_multi);
  float2* win = base + warp * (P * kWinPitch);
  float2* accs = base + W * P * kWinPitch;
  float2* acc = accs + warp * (P * kAccPitch2);
  uint2* stg = reinterpret_cast<uint2*>(accs + W * P * kAccPitch2) + warp * (D * NA * 32);
  for (int i = threadIdx.x; i < W * P * kAccPitch2; i += blockDim.x) accs[i] = make_float2(0.f, 0.f);
  for (int m = threadIdx.x; m < n_mem; m += blockDim.x) s_item0[m] = mem[m].item0;
  if (threadIdx.x == 0) s_item0[n_mem] = n_items;
  __syncthreads();
  constexpr int lo_x = J - 1, hi_x = kTile;
  const unsigned lanes_below = (1u << lane) - 1u;

  unsigned int* dbg = nullptr;  // the current member's error word (GBRI_DEBUG builds)
  long long M = 0;
  auto issue = [&](int q, int2 d) {
    if ((((unsigned)d.y) >> lane) & 1u) {
      const int pos = (d.x & 0x7fffffff) + __popc((unsigned)d.y & lanes_below);
      if (!GBRI_DCHECK(dbg, pos < M, kDbgVis, pos)) return;
      uint2* col = stg + (q * NA) * 32 + lane;
      cp_async8(col, static_cast<const uint2*>(s_ptr[warp][0]) + pos);
      cp_async8(col + 32, static_cast<const float2*>(s_ptr[warp][1]) + pos);
      cp_async8(col + 64, static_cast<const float2*>(s_ptr[warp][2]) + pos);
    }
  };

  int it = take_item(ctr);
  while (it < n_items) {
    const int it_next = take_item(ctr);
    int mi = 0;  // the member: the last whose first item is at most it
    {
      int hi = n_mem - 1;
      while (mi < hi) {
        const int mid = (mi + hi + 1) >> 1;
        if (s_item0[mid] <= it) mi = mid;
        else hi = mid - 1;
      }
    }
    const FusedMember& F = mem[mi];
    if (lane == 0) {
      s_ptr[warp][0] = F.meta;
      s_ptr[warp][1] = F.u;
      s_ptr[warp][2] = F.y;
    }
    __syncwarp();
    dbg = F.dbg;
    M = F.M;
    const int4 gt = F.gtiles[it - s_item0[mi]];  // {tile, first step, steps, split}
    const int2* steps = F.steps;
    const int K = F.K, nT = F.nT, log2S = F.log2S;
    const int S = 1 << log2S;
    const float two_over_S = 2.f / (float)S;
    const float cc = (float)*F.c;
    const float sigma2 = F.sigma2;
    float2* u = F.u;
    const int s0 = gt.y, ns = gt.z;
    int2 dcur = lane < ns ? steps[s0 + lane] : make_int2(0, 0);
    int2 dnxt = 32 + lane < ns ? steps[s0 + 32 + lane] : make_int2(0, 0);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const int2 d = shfl_int2(dcur, q);
      if (q < ns) issue(q, d);
      cp_async_commit();
    }
    load_window_f32<J>(win, F.spec, gt.x, nT, K, lane, dbg);
    __syncwarp();
    KahanF sum;
    float2 pt[J][J];
    float2 blk[J][J];
#pragma unroll
    for (int tp = 0; tp < J; ++tp)
#pragma unroll
      for (int t = 0; t < J; ++t) pt[tp][t] = make_float2(0.f, 0.f);
    int a0 = 0;
    bool has = false;
    for (int i = 0; i < ns; ++i) {
      if (i > 0 && (i & 31) == 0) {
        dcur = dnxt;
        dnxt = i + 32 + lane < ns ? steps[s0 + i + 32 + lane] : make_int2(0, 0);
      }
      const int2 d = shfl_int2(dcur, i & 31);
      const bool start = d.x < 0;
      if (start && i > 0) {  // the previous group's patches into the accumulator
#pragma unroll
        for (int tp = 0; tp < J; ++tp)
#pragma unroll
          for (int t = 0; t < J; ++t) {
            if (has) {
              float2* q = acc + a0 + tp * kAccPitch2 + t;
              *q = add2(*q, pt[tp][t]);
            }
            pt[tp][t] = make_float2(0.f, 0.f);
            __syncwarp();
          }
      }
      cp_async_wait<D - 1>();
      const int q = i & (D - 1);
      const bool act = ((((unsigned)d.y) >> lane) & 1u) != 0u;
      const uint2* col = stg + (q * NA) * 32 + lane;
      if (act) {
        const int pos = (d.x & 0x7fffffff) + __popc((unsigned)d.y & lanes_below);
        const uint2 m = col[0];
        if (start) {
          const int cy = (int)(m.x >> 16) >> log2S, cx = (int)(m.x & 0xffff) >> log2S;
          has = GBRI_DCHECK(dbg, cy < kTile && cx < kTile, kDbgWindow, pos);
          a0 = has ? cy * kWinPitch + cx : 0;
#pragma unroll
          for (int tp = 0; tp < J; ++tp)
#pragma unroll
            for (int t = 0; t < J; ++t) blk[tp][t] = win[a0 + tp * kWinPitch + t];
        }
        float2 w[J];
        taps_xy<J>(poly, m.x, S, two_over_S, w);
        const float2 wt = f2(__uint_as_float(m.y));
        float2 dg = make_float2(0.f, 0.f);
#pragma unroll
        for (int tp = 0; tp < J; ++tp) {
          float2 row = mul2(f2(w[0].x), blk[tp][0]);
#pragma unroll
          for (int t = 1; t < J; ++t) row = fma2(f2(w[t].x), blk[tp][t], row);
          dg = fma2(f2(w[tp].y), row, dg);
        }
        // u <- c u + sigma2 (w phi - y), as EpiPD1::update
        const float2 uo = *reinterpret_cast<const float2*>(col + 32);
        const float2 yo = *reinterpret_cast<const float2*>(col + 64);
        const float2 phi = mul2(wt, dg);
        const float2 un = make_float2(fmaf(cc, uo.x, sigma2 * (phi.x - yo.x)), fmaf(cc, uo.y, sigma2 * (phi.y - yo.y)));
        u[pos] = un;
        sum.add(fmaf(un.x, un.x, un.y * un.y));
        const float2 wv = mul2(wt, un);
#pragma unroll
        for (int tp = 0; tp < J; ++tp) {
          const float2 b = mul2(f2(w[tp].y), wv);
#pragma unroll
          for (int t = 0; t < J; ++t) pt[tp][t] = fma2(f2(w[t].x), b, pt[tp][t]);
        }
      } else if (start) {
        has = false;
      }
      const int i2 = i + D;
      const int2 d2 = shfl_int2(((i2 >> 5) == (i >> 5)) ? dcur : dnxt, i2 & 31);
      if (i2 < ns) issue(q, d2);
      cp_async_commit();
    }
#pragma unroll
    for (int tp = 0; tp < J; ++tp)
#pragma unroll
      for (int t = 0; t < J; ++t) {
        if (has && ns > 0) {
          float2* q = acc + a0 + tp * kAccPitch2 + t;
          *q = add2(*q, pt[tp][t]);
        }
        __syncwarp();
      }
    // the member's sum of |u|^2 over this item
    const double v = warp_sum(sum.value());
    if (lane == 0) atomicAdd(sums + mi, v);
    const int ty = gt.x / nT, tx = gt.x - ty * nT;
    const int oy = ty * kTile - (J / 2 - 1), ox = tx * kTile - (J / 2 - 1);
    float2* grid = F.grid;
    for (int e = lane; e < P * P; e += 32) {
      const int r = e / P, c2 = e - r * P;
      float2* qa = acc + r * kAccPitch2 + c2;
      const float2 a = *qa;
      *qa = make_float2(0.f, 0.f);
      const size_t gq = (size_t)wrapK(oy + r, K) * K + wrapK(ox + c2, K);
      if (!GBRI_DCHECK(dbg, gq < (size_t)K * K, kDbgGrid, gq)) continue;
      float2* dst = grid + gq;
      if (gt.w == 0 && r >= lo_x && r < hi_x && c2 >= lo_x && c2 < hi_x) *dst = a;
      else if (a.x != 0.f || a.y != 0.f) atomicAdd(dst, a);
    }
    __syncwarp();
    it = it_next;
  }
  cp_async_wait<0>();
  // the last block to finish turns every member's sum into its ball scalar and resets the
  // counters and sums for the next launch (stream order makes that visible to it)
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ctr + 1, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int m = threadIdx.x; m < n_mem; m += blockDim.x) {
    const double s = __ldcg(sums + m);
    const FusedMember& F = mem[m];
    const double dist = sqrt(s) / F.sigma2d;
    const double rho = dist > F.eps ? F.eps / dist : 1.0;
    *F.c = 1.0 - rho;
    *F.dist = dist;
    sums[m] = 0.0;
  }
  if (threadIdx.x == 0) {
    atomicExch(ctr, 0u);
    atomicExch(ctr + 1, 0u);
  }
}

// Shared memory of k_steps_multi (window, accumulator and a three-stream ring per warp).
constexpr size_t steps_multi_smem() {
  constexpr int P = kTile + 4 - 1;
  return (size_t)(kThreads / 32) * (P * kWinPitch + P * kAccPitch2) * 8 + (size_t)(kThreads / 32) * kStageDepth * 3 * 32 * 8;
}

}  // namespace gbri
