// Measurement operator Phi = W G F Z S (Sec. 2, Eq. 2) on one GPU: the plan
// object and the kernel templates shared by the operator calls and the solvers.
//
// Data layout in HBM (per plan):
//   meta   [M] uint2   plan (sorted) order: .x = (ly << 16) | lx, the tile-local
//                      fixed-point coordinates (cell-in-tile * S + fraction),
//                      .y = weight bits (float).  8 bytes per visibility.
//   perm   [M] int32   plan position -> caller's visibility index.
//   subruns [R] int2   runs {first plan position, count}: consecutive visibilities of one
//                      cell (at most the plan's run length); within a tile listed round by
//                      round (every cell's first run, then every second one, ...), each
//                      round padded to a multiple of 32 with empty runs {0, 0}.
//   gtiles [G] int4    gridding work items: {tile, first run, runs, split}; one per non-empty
//                      tile, or several (split = 1) for a tile heavier than twice a warp's
//                      share of the visibilities.
//   steps  [N] int2    step-layout plans only (FP32, polynomial taps, J = 4): the runs of
//                      every 32-run group are stored step-major (step k: the k-th visibility
//                      of each run longer than k, in lane order); steps[s] = {plan position
//                      of the step's first visibility | group start << 31, mask of the lanes
//                      holding one}; gtiles then list {tile, first step, steps, split}.
//   chunks [C] int4    degridding work items: {tile, first plan position, visibilities
//                      (<= kChunk), 0}: consecutive visibilities of one tile (any layout).
//   Visibilities are stored in run order: a tile's visibilities are contiguous, and so
//   are a run's (step-layout plans: a tile's and a group's are contiguous).
//   wtab   [S/2+1][J] R  tap weights by fractional offset f = k~ mod S: entry t is
//                      table[|f + (J/2 - 1 - t) S|] (Sec. 8.1 zeroth-order table,
//                      re-indexed so one visibility reads one row per axis).
//   frac   [M] uint16  first-order plans only: sub-sample fractions (fx | fy << 8) in
//                      1/256 of a table step, plan order.
//   corr   [n] R       1 / ghat(p'/K) (the S factor along one axis).
//   padded [K][K] R    real FFT input; zero outside the n x n image block (kept zero).
//   spec   [K][K/2+1] C  its real-to-complex FFT (half spectrum), read by degridding.
//   grid   [K][K] C    gridding accumulator; after the inverse its first half holds
//                       Re(F^H grid) as R [K][K].
// R is the plan's real type (float for GBRI_F32, double for GBRI_F64) and C the
// interleaved complex of R; the visibility order and metadata do not depend on it.
#pragma once

#include <cufft.h>

#include <vector>

#include "common.cuh"

namespace gbri {

constexpr int kTile = 16;      // grid tile side in cells (T * S <= 65536 keeps 16-bit local coords)
constexpr int kThreads = 256;  // threads per block of the visibility kernels
constexpr int kRun = 4;        // visibilities a thread has in flight (degridding: per chunk; gridding: per load round)
constexpr int kChunk = kThreads * kRun;  // visibilities per degridding chunk
constexpr int kDefaultRun = 64;  // default longest run of one cell's visibilities a gridding thread takes
constexpr int kMaxRun = 1024;
// complex-element row pitch of the degridding window and of the gridding accumulators
// (the plan's bank-slot map uses it)
constexpr int kWinPitch = 22;
// First-order interpolation: coordinates are quantised kFracSteps times finer than the
// table step; the fraction between two table samples is kept in 8 bits per axis.
constexpr int kLog2FracSteps = 8;
constexpr int kFracSteps = 1 << kLog2FracSteps;

// Bounds checks of the GBRI_DEBUG build: an index that would leave its buffer sets a bit in
// the plan's device error word (and the first such index beside it) and the access is
// skipped; nothing traps.  In the default build every check is the constant true.
enum DebugBit : unsigned {
  kDbgWindow = 1u,       // degridding window / shared spectrum block
  kDbgAccum = 2u,        // gridding accumulator
  kDbgGrid = 4u,         // grid cell of the flush
  kDbgVis = 8u,          // visibility position (metadata, streams)
  kDbgSpec = 16u,        // half-spectrum cell
  kDbgSlot = 32u,        // deterministic window slot
};
__device__ __forceinline__ bool debug_fail(unsigned int* word, unsigned int bit, long long idx) {
  if (word && atomicOr(word, bit) == 0u) *reinterpret_cast<long long*>(word + 2) = idx;
  return false;
}
#ifdef GBRI_DEBUG
#define GBRI_DCHECK(word, cond, bit, idx) ((cond) || ::gbri::debug_fail((word), (bit), (long long)(idx)))
#else
#define GBRI_DCHECK(word, cond, bit, idx) true
#endif

// How a visibility kernel gets its tap weights:
//   kTapTable: zeroth-order pre-sampled table in shared memory (Sec. 8.1);
//   kTapFO:    first-order interpolation between two table rows (Sec. 8.1, reading R13);
//   kTapPoly:  the kernel g on each unit segment [k, k + 1] of its support as a polynomial
//              fitted at plan time (FP32 plans, zeroth-order positions), evaluated in
//              registers at the same quantised positions the table is sampled at, so the
//              weights equal the table's to FP32 rounding.  It replaces the table's random
//              shared-memory rows (the pipe the visibility kernels are bound by) with FMAs.
enum TapMode { kTapTable = 0, kTapFO = 1, kTapPoly = 2 };

// Polynomial taps: on segment k (distance s in [k, k + 1] from the tap's cell) and with
// z = 2 (s - k) - 1 in [-1, 1], g = P_k(z) = E_k(z^2) + z O_k(z^2), E_k and O_k of degree
// kPolyHalf - 1 (P_k of degree 2 kPolyHalf - 1).
constexpr int kPolyHalf = 5;
struct PolyTaps {
  float e[3][kPolyHalf];  // even part of segment k, coefficient of (z^2)^i
  float o[3][kPolyHalf];  // odd part
};

// Resident blocks per SM the visibility kernels are compiled for (launch bounds) and
// launched with at most, by element size (4: FP32 path, 8: FP64 path) and support.  An FP32
// degridding block (kernel table + eight windows) takes about 60 KB of shared memory at
// J = 4, so three fit an SM; bounds of three leave 80 registers a thread, which measured
// faster than bounds of four (64 registers).
constexpr int degrid_occupancy(int rb, int J) { return rb == 4 ? 3 : 2; }
constexpr int grid_occupancy(int rb, int J) { return rb == 4 ? (J == 4 ? 3 : 2) : 1; }

}  // namespace gbri

struct gbri_plan {
  int n_side = 0, K = 0, J = 0, S = 0, log2S = 0, nT = 0, prec = 0;
  double beta = 0;
  int64_t M = 0;
  uint2* meta = nullptr;
  int32_t* perm = nullptr;
  int4* chunks = nullptr;
  int2* subruns = nullptr;  // runs {first plan position, count}: visibilities of one cell
  int4* gtiles = nullptr;   // gridding work items {tile, first run, runs}
  int64_t n_chunks = 0;
  int64_t n_gtiles = 0;
  int64_t n_tiles = 0;  // non-empty tiles
  int32_t* cell_off = nullptr;  // plan creation only
  void* wtab = nullptr;     // R
  void* corr = nullptr;     // R
  void* padded = nullptr;   // R [K][K]: Z S x (zero outside the image)
  void* spec = nullptr;     // C [K][K/2 + 1]: its real-to-complex FFT (half spectrum; Phi)
  void* grid = nullptr;     // C [K][K]: the gridded visibilities; then Re of their inverse FFT, R [K][K]
  void* vis_tmp = nullptr;  // C [M] plan-order scratch
  double* partials = nullptr;  // reduction partials
  double* scalars = nullptr;   // small device scalars
  int n_partials = 0;
  cufftHandle fft_r2c = 0;  // R2C / D2Z, forward (padded -> spec)
  cufftHandle fft_c2r = 0;  // C2R / Z2D, inverse of a Hermitian half spectrum (spec -> grid as R [K][K])
  bool fft_r2c_ok = false, fft_c2r_ok = false;
  int64_t device_bytes = 0;
  int64_t layout_bytes = 0;
  int degrid_blocks = 0, grid_blocks = 0;
  int run_len = gbri::kDefaultRun;  // longest run (visibilities of one cell a gridding thread takes)
  // first-order table interpolation: per visibility the sub-sample fractions of the two
  // coordinates in 1/kFracSteps of a table step, (fx | fy << 8), plan order; null for zeroth order
  uint16_t* frac = nullptr;
  uint16_t* frac_in = nullptr;  // plan creation only: the fractions in the caller's order
  int interp = 0;               // 0: zeroth-order table, 1: first order
  int tap_mode = gbri::kTapTable;  // how the visibility kernels get their tap weights
  gbri::PolyTaps poly{};        // kTapPoly coefficients
  // work counters of the kTapPoly kernels, a pair {next item, finished blocks} per kernel
  // (degridding, gridding, fused); zero between launches
  unsigned int* work = nullptr;
  unsigned int* dbg = nullptr;  // GBRI_DEBUG builds: {error bits, 0, first bad index (int64)}
  // deterministic gridding: every gridding work item writes its (T + J - 1)^2 window to
  // slots[item] (plan precision, complex), and k_grid_reduce sums, for every grid cell, the
  // windows covering it in a fixed order (tiles by position, a tile's items by index)
  int det = 0;
  void* slots = nullptr;             // C [n_gtiles][P][P]
  int32_t* tile_items_off = nullptr;  // [nT^2 + 1] CSR offsets: items of each tile
  int32_t* tile_items = nullptr;      // [n_gtiles] item indices, ascending per tile
  int autotune = 0;
  // step layout (FP32 polynomial-tap plans with J = 4): visibilities of every 32-run group
  // stored step-major, steps[s] = {first plan position | group start << 31, lanes holding a
  // visibility}; gtiles are then {tile, first step, steps, split}
  int step_layout = 0;
  int layout_req = 0;  // gbri_plan_desc.layout: 0 automatic, 1 the run layout
  int2* steps = nullptr;
  int64_t n_steps = 0;
  template <class T> T* as(void* q) const { return static_cast<T*>(q); }
};

namespace gbri {

__device__ __forceinline__ int wrapK(int v, int K) { return v < 0 ? v + K : (v >= K ? v - K : v); }

// Load the J tap weights of one axis for fractional offset f (0 <= f < S) from the
// shared table.  The table stores rows f = 0 .. S/2 only: row S - f is row f reversed
// (entry t of row f is table[|f + (J/2 - 1 - t) S|]).
template <int J, class R>
__device__ __forceinline__ void load_taps(const R* sw, int f, int S, R (&w)[J]) {
  const bool rev = f > (S >> 1);
  const int row = rev ? S - f : f;
  R v[J];
  if constexpr (J == 4 && sizeof(R) == 4) {
    const float4 q = reinterpret_cast<const float4*>(sw)[row];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (J % 2 == 0) {  // rows of J even elements are 2-element aligned
    using R2 = cplx<R>;
    const R2* p = reinterpret_cast<const R2*>(sw + row * J);
#pragma unroll
    for (int t = 0; t < J / 2; ++t) {
      const R2 a = p[t];
      v[2 * t] = a.x;
      v[2 * t + 1] = a.y;
    }
  } else {
#pragma unroll
    for (int t = 0; t < J; ++t) v[t] = sw[row * J + t];
  }
#pragma unroll
  for (int t = 0; t < J; ++t) w[t] = rev ? v[J - 1 - t] : v[t];
}

// First-order taps (Sec. 8.1 pre-sampling, first-order interpolation): the position lies
// phi / kFracSteps of a table step past sample f, so each tap interpolates linearly
// between rows f and f + 1 (0 <= f < S; row S is row 0 reversed, the next cell's row 0).
template <int J, class R>
__device__ __forceinline__ void load_taps_fo(const R* sw, int f, int phi, int S, R (&w)[J]) {
  R a[J], b[J];
  load_taps<J>(sw, f, S, a);
  load_taps<J>(sw, f + 1, S, b);
  const R t = (R)phi * ((R)1 / (R)kFracSteps);
#pragma unroll
  for (int j = 0; j < J; ++j) w[j] = fma_r(t, b[j] - a[j], a[j]);
}

// elements of the stored tap table (rows 0 .. S/2), rounded up to a multiple of 4
__host__ __device__ inline int table_elems(int S, int J) { return (((S / 2 + 1) * J) + 3) & ~3; }

template <class R>
__device__ __forceinline__ void copy_table_to_smem(R* sw, const R* __restrict__ g, int nelems) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float4* s4 = reinterpret_cast<float4*>(sw);
  const int n4 = nelems * (int)sizeof(R) / 16;
  for (int i = threadIdx.x; i < n4; i += blockDim.x) s4[i] = __ldg(g4 + i);
}

struct VisGeom {
  const uint2* __restrict__ meta;
  const int4* __restrict__ chunks;
  const int2* __restrict__ subruns;
  const int4* __restrict__ gtiles;
  const int2* __restrict__ steps;      // step layout: step descriptors (else null)
  const void* __restrict__ wtab;
  const uint16_t* __restrict__ frac;  // first-order fractions (null: zeroth order)
  void* slots;                         // deterministic gridding: per-item windows (null: atomics)
  unsigned int* dbg;                   // GBRI_DEBUG builds: the plan's error word (else null)
  int64_t M;                           // visibilities (bounds checks)
  int n_chunks, n_gtiles, K, log2S, nT;
  PolyTaps poly;                       // kTapPoly coefficients (kernel parameter space)
};

// shared-memory elements of the tap table a kernel of tap mode tm holds (none for kTapPoly)
inline int smem_table_elems(int tm, int S, int J) { return tm == kTapPoly ? 0 : table_elems(S, J); }
inline size_t degrid_smem(const gbri_plan* p) {  // the tap table and one window per warp
  const size_t rb = real_bytes(p->prec);
  return (size_t)smem_table_elems(p->tap_mode, p->S, p->J) * rb +
         (size_t)(kThreads / 32) * (kTile + p->J - 1) * kWinPitch * 2 * rb;
}
// warp-private gridding accumulators: complex cells, row pitch kAccPitch2 (>= T + J - 1)
constexpr int kAccPitch2 = kWinPitch;
inline size_t grid_smem(const gbri_plan* p) {
  const size_t rb = real_bytes(p->prec);
  const int P = kTile + p->J - 1;
  return (size_t)smem_table_elems(p->tap_mode, p->S, p->J) * rb + (size_t)(kThreads / 32) * P * kAccPitch2 * 2 * rb;
}

inline VisGeom vis_geom(const gbri_plan* p) {
  VisGeom g;
  g.meta = p->meta;
  g.chunks = p->chunks;
  g.subruns = p->subruns;
  g.gtiles = p->gtiles;
  g.steps = p->steps;
  g.wtab = p->wtab;
  g.frac = p->frac;
  g.slots = p->det ? p->slots : nullptr;
  g.dbg = p->dbg;
  g.M = p->M;
  g.n_chunks = (int)p->n_chunks;
  g.n_gtiles = (int)p->n_gtiles;
  g.K = p->K;
  g.log2S = p->log2S;
  g.nT = p->nT;
  g.poly = p->poly;
  return g;
}

// ---- epilogues / sources ------------------------------------------------------
// A degridding epilogue reads kStreams per-visibility input streams of element type
// SElem (stream(j), indexed by plan position); pre_from(st, pos) gathers element pos
// of every stream (issued with the metadata loads), and store(pos, pre, v) consumes
// the degridded value.  Each names its real type R (the plan's precision).
template <class R>
struct EpiStorePlan {  // y[pos] = v
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 0;
  cplx<R>* y;
  struct Pre {};
  __device__ __forceinline__ const SElem* stream(int) const { return nullptr; }
  __device__ __forceinline__ void init() { __syncthreads(); }
  __device__ __forceinline__ void begin_chunk(int) {}
  __device__ __forceinline__ Pre pre_from(const SElem* const*, int) const { return Pre{}; }
  __device__ __forceinline__ void store(int pos, const Pre&, cplx<R> v) { y[pos] = v; }
  __device__ __forceinline__ void finish() {}
};
template <class R>
struct EpiStoreRaw {  // y[perm[pos]] = v
  using real = R;
  using SElem = int32_t;
  static constexpr int kStreams = 1;
  cplx<R>* y;
  const int32_t* perm;
  struct Pre { int dst; };
  __device__ __forceinline__ const SElem* stream(int) const { return perm; }
  __device__ __forceinline__ void init() { __syncthreads(); }
  __device__ __forceinline__ void begin_chunk(int) {}
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i]}; }
  __device__ __forceinline__ void store(int, const Pre& p, cplx<R> v) { y[p.dst] = v; }
  __device__ __forceinline__ void finish() {}
};
// A gridding source gives the value at a plan position; ctx(pos) is evaluated once per
// tile (any position of the tile) and passed to every call of that tile.
struct NoCtx {};
template <class R>
struct SrcPlan {
  using real = R;
  using Ctx = NoCtx;
  const cplx<R>* y;
  __device__ __forceinline__ Ctx ctx(int) const { return Ctx{}; }
  __device__ __forceinline__ cplx<R> operator()(int pos, const Ctx&) const { return y[pos]; }
};
template <class R>
struct SrcRaw {
  using real = R;
  using Ctx = NoCtx;
  const cplx<R>* y;
  const int32_t* perm;
  __device__ __forceinline__ Ctx ctx(int) const { return Ctx{}; }
  __device__ __forceinline__ cplx<R> operator()(int pos, const Ctx&) const { return y[perm[pos]]; }
};

// Solver epilogues (fused dual updates; see solver.cu for the algebra).
template <class R>
struct EpiPD1 {
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 2;
  cplx<R>* u;
  const cplx<R>* y;
  const double* c;
  double* partials;
  R sigma2;
  acc_t<R> acc;
  R cc;  // *c rounded to R once per thread (a per-visibility conversion would run on the FP64 pipe)
  struct Pre { cplx<R> u, y; };
  __device__ __forceinline__ const SElem* stream(int j) const { return j == 0 ? u : y; }
  __device__ __forceinline__ void init() {
    cc = (R)*c;
    __syncthreads();
  }
  __device__ __forceinline__ void begin_chunk(int) {}
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i], st[1][i]}; }
  // u <- c u + sigma2 (phi - y), stored and returned (the fused degrid + grid pass grids it)
  __device__ __forceinline__ cplx<R> update(int pos, const Pre& p, cplx<R> phi) {
    const cplx<R> un = mkc<R>(fma_r(cc, p.u.x, sigma2 * (phi.x - p.y.x)), fma_r(cc, p.u.y, sigma2 * (phi.y - p.y.y)));
    u[pos] = un;
    acc.add(fma_r(un.x, un.x, un.y * un.y));
    return un;
  }
  __device__ __forceinline__ void store(int pos, const Pre& p, cplx<R> phi) { update(pos, p, phi); }
  // The l2-ball scalar of the next update, fused: the last block to finish (device-wide
  // counter, reset by that block) reduces the block partials in block order and stores
  // c = 1 - min(1, eps / dist), dist = sqrt(sum) / sigma2.  Every block has read the old c
  // (init) before it counts itself, so the store cannot race with a reader.  Without a
  // counter (done null) only the partials are written.
  double* c_out = nullptr;
  double* dist_out = nullptr;
  unsigned int* done = nullptr;
  double eps = 0.0, sigma2d = 1.0;
  __device__ __forceinline__ void finish() {
    __shared__ double sh[40];
    __shared__ bool last;
    const double v = block_sum(acc.value(), sh);
    if (done == nullptr) {
      if (threadIdx.x == 0) partials[blockIdx.x] = v;
      return;
    }
    if (threadIdx.x == 0) {
      partials[blockIdx.x] = v;
      __threadfence();
      last = atomicAdd(done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double sum = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) sum += __ldcg(partials + i);
    sum = block_sum(sum, sh);
    if (threadIdx.x == 0) {
      const double dist = sqrt(sum) / sigma2d;
      const double rho = dist > eps ? eps / dist : 1.0;
      *c_out = 1.0 - rho;
      *dist_out = dist;
      *done = 0u;
    }
  }
};

template <class R>
struct EpiADMM1 {  // w = Phi x + s - y, partial ||w||^2
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 2;
  cplx<R>* w;
  const cplx<R>* sv;
  const cplx<R>* y;
  double* partials;
  acc_t<R> acc;
  struct Pre { cplx<R> s, y; };
  __device__ __forceinline__ const SElem* stream(int j) const { return j == 0 ? sv : y; }
  __device__ __forceinline__ void init() { __syncthreads(); }
  __device__ __forceinline__ void begin_chunk(int) {}
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i], st[1][i]}; }
  __device__ __forceinline__ void store(int pos, const Pre& p, cplx<R> v) {
    const cplx<R> r = mkc<R>(v.x + p.s.x - p.y.x, v.y + p.s.y - p.y.y);
    w[pos] = r;
    acc.add(fma_r(r.x, r.x, r.y * r.y));
  }
  __device__ __forceinline__ void finish() {
    __shared__ double sh[40];
    const double v = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
};

template <class R>
struct EpiResid {  // r = Phi x - y, partial ||r||^2 (FISTA's gradient residual)
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 1;
  cplx<R>* r;
  const cplx<R>* y;
  double* partials;
  acc_t<R> acc;
  struct Pre { cplx<R> y; };
  __device__ __forceinline__ const SElem* stream(int) const { return y; }
  __device__ __forceinline__ void init() { __syncthreads(); }
  __device__ __forceinline__ void begin_chunk(int) {}
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i]}; }
  // r = v - y, stored and returned (the fused degrid + grid pass grids it)
  __device__ __forceinline__ cplx<R> update(int pos, const Pre& p, cplx<R> v) {
    const cplx<R> d = mkc<R>(v.x - p.y.x, v.y - p.y.y);
    r[pos] = d;
    acc.add(fma_r(d.x, d.x, d.y * d.y));
    return d;
  }
  __device__ __forceinline__ void store(int pos, const Pre& p, cplx<R> v) { update(pos, p, v); }
  __device__ __forceinline__ void finish() {
    __shared__ double sh[40];
    const double v = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
};

template <class R>
struct SrcADMM2 {  // s+ = s + varrho((1 - rho_b) w - s); source q = (1 - rho_b) w - s + s+
  using real = R;
  struct Ctx { R one_m; };  // 1 - rho_b rounded once per tile
  const cplx<R>* w;
  cplx<R>* sv;
  const double* rho_b;
  R varrho;
  __device__ __forceinline__ Ctx ctx(int) const { return Ctx{(R)(1.0 - *rho_b)}; }
  __device__ __forceinline__ cplx<R> operator()(int pos, const Ctx& x) const {
    const R one_m = x.one_m;
    const cplx<R> ww = w[pos], so = sv[pos];
    const cplx<R> pw = mkc<R>(one_m * ww.x, one_m * ww.y);
    const cplx<R> sn = mkc<R>(fma_r(varrho, pw.x - so.x, so.x), fma_r(varrho, pw.y - so.y, so.y));
    sv[pos] = sn;
    return mkc<R>(pw.x - so.x + sn.x, pw.y - so.y + sn.y);
  }
};

// ---- local l2 balls (Sec. 6.9) ----------------------------------------------------
// Ball j holds the plan positions [bstart[j], bstart[j + 1]) (whole tiles, so that a
// degridding chunk and a gridding tile lie in one ball).
constexpr int kMaxBalls = 64;
__device__ __forceinline__ int ball_of(const int32_t* bstart, int nb, int pos) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bstart[mid] <= pos) lo = mid;
    else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ double* ball_sums_smem() {
  __shared__ double b[kMaxBalls];
  return b;
}
__device__ __forceinline__ double* ball_red_smem() {
  __shared__ double b[40];
  return b;
}

// Per-ball sums of squares of one degridding launch: each thread accumulates into the
// current ball (compensated FP32 / FP64); when a warp's chunk enters another ball the warp
// sum is added to the block's per-ball shared sums; at the end every block writes
// partials[j * gridDim.x + blockIdx.x] for every ball j (fixed-order reduction later).
template <class R>
struct BallAcc {
  const int32_t* bstart;
  int nb;
  double* partials;
  acc_t<R> acc;
  int cur;
  __device__ __forceinline__ void init() {  // block-wide
    double* b = ball_sums_smem();
    for (int j = threadIdx.x; j < kMaxBalls; j += blockDim.x) b[j] = 0.0;
    acc = acc_t<R>{};
    cur = -1;
    __syncthreads();
  }
  __device__ __forceinline__ void flush() {  // warp-uniform
    if (cur < 0) return;
    const double v = warp_sum(acc.value());
    if ((threadIdx.x & 31) == 0) atomicAdd(ball_sums_smem() + cur, v);
    acc = acc_t<R>{};
  }
  __device__ __forceinline__ int enter(int lo) {  // warp-uniform
    const int b = ball_of(bstart, nb, lo);
    if (b != cur) {
      flush();
      cur = b;
    }
    return b;
  }
  __device__ __forceinline__ void finish() {  // block-wide
    flush();
    __syncthreads();
    const double* b = ball_sums_smem();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) partials[(size_t)j * gridDim.x + blockIdx.x] = b[j];
  }
};

template <class R>
struct EpiPD1L {  // EpiPD1 with one scale c_j per ball: u <- c_j u + sigma2 (Phi xhat - y)
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 2;
  cplx<R>* u;
  const cplx<R>* y;
  const double* cb;
  R sigma2;
  BallAcc<R> ba;
  R c;
  struct Pre { cplx<R> u, y; };
  __device__ __forceinline__ const SElem* stream(int j) const { return j == 0 ? u : y; }
  __device__ __forceinline__ void init() { ba.init(); }
  __device__ __forceinline__ void begin_chunk(int lo) { c = (R)cb[ba.enter(lo)]; }
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i], st[1][i]}; }
  __device__ __forceinline__ void store(int pos, const Pre& p, cplx<R> phi) {
    const cplx<R> un = mkc<R>(fma_r(c, p.u.x, sigma2 * (phi.x - p.y.x)), fma_r(c, p.u.y, sigma2 * (phi.y - p.y.y)));
    u[pos] = un;
    ba.acc.add(fma_r(un.x, un.x, un.y * un.y));
  }
  __device__ __forceinline__ void finish() { ba.finish(); }
};

template <class R>
struct EpiADMM1L {  // EpiADMM1 with per-ball sums of ||w_j||^2
  using real = R;
  using SElem = cplx<R>;
  static constexpr int kStreams = 2;
  cplx<R>* w;
  const cplx<R>* sv;
  const cplx<R>* y;
  BallAcc<R> ba;
  struct Pre { cplx<R> s, y; };
  __device__ __forceinline__ const SElem* stream(int j) const { return j == 0 ? sv : y; }
  __device__ __forceinline__ void init() { ba.init(); }
  __device__ __forceinline__ void begin_chunk(int lo) { ba.enter(lo); }
  __device__ __forceinline__ Pre pre_from(const SElem* const* st, int i) const { return Pre{st[0][i], st[1][i]}; }
  __device__ __forceinline__ void store(int pos, const Pre& p, cplx<R> v) {
    const cplx<R> r = mkc<R>(v.x + p.s.x - p.y.x, v.y + p.s.y - p.y.y);
    w[pos] = r;
    ba.acc.add(fma_r(r.x, r.x, r.y * r.y));
  }
  __device__ __forceinline__ void finish() { ba.finish(); }
};

template <class R>
struct SrcScaledL {  // z2 = c_j u (the PD dual with local balls)
  using real = R;
  struct Ctx { R c; };
  const cplx<R>* u;
  const double* cb;
  const int32_t* bstart;
  int nb;
  __device__ __forceinline__ Ctx ctx(int pos) const { return Ctx{(R)cb[ball_of(bstart, nb, pos)]}; }
  __device__ __forceinline__ cplx<R> operator()(int pos, const Ctx& x) const {
    const cplx<R> v = u[pos];
    return mkc<R>(x.c * v.x, x.c * v.y);
  }
};

template <class R>
struct SrcADMM2L {  // SrcADMM2 with one rho_j per ball
  using real = R;
  struct Ctx { R one_m; };
  const cplx<R>* w;
  cplx<R>* sv;
  const double* rho_b;
  const int32_t* bstart;
  int nb;
  R varrho;
  __device__ __forceinline__ Ctx ctx(int pos) const { return Ctx{(R)(1.0 - rho_b[ball_of(bstart, nb, pos)])}; }
  __device__ __forceinline__ cplx<R> operator()(int pos, const Ctx& x) const {
    const cplx<R> ww = w[pos], so = sv[pos];
    const cplx<R> pw = mkc<R>(x.one_m * ww.x, x.one_m * ww.y);
    const cplx<R> sn = mkc<R>(fma_r(varrho, pw.x - so.x, so.x), fma_r(varrho, pw.y - so.y, so.y));
    sv[pos] = sn;
    return mkc<R>(pw.x - so.x + sn.x, pw.y - so.y + sn.y);
  }
};

// ---- launch helpers (defined in the visibility translation units, vis_f32.cu and
// vis_f64.cu, with explicit instantiations, so that each kernel template is
// instantiated in exactly one translation unit) --------------------------------
// Degrids the forward FFT (the half spectrum p->spec) into the epilogue.
template <class Epi>
int32_t launch_degrid(gbri_plan* p, Epi epi, cudaStream_t s);
// Zeroes p->grid (unless the caller has, zeroed = true), then grids every visibility into it.
template <class Src>
int32_t launch_grid(gbri_plan* p, Src src, cudaStream_t s, bool zeroed = false);
// The FP32 kernels with polynomial taps (plans with tap_mode == kTapPoly; defined in the FP32
// visibility translation unit); launch_degrid / launch_grid dispatch to them.
template <class Epi>
int32_t launch_degrid_fast(gbri_plan* p, Epi epi, cudaStream_t s);
template <class Src>
int32_t launch_grid_fast(gbri_plan* p, Src src, cudaStream_t s);
// Degridding into an epilogue with an `update` (EpiPD1: the PD dual update; EpiResid: the
// FISTA residual) fused with the gridding of the values it returns (J = 4, FP32 plans of
// either table order): zeroes p->grid first unless zeroed.
int32_t launch_degrid_grid(gbri_plan* p, EpiPD1<float> epi, cudaStream_t s, bool zeroed);
int32_t launch_degrid_grid(gbri_plan* p, EpiResid<float> epi, cudaStream_t s, bool zeroed);
// Whether launch_degrid_grid applies to the plan.
inline bool fused_pd_applies(const gbri_plan* p) {
  return p->J == 4 && p->prec == GBRI_F32 && p->n_gtiles > 0;
}
// Bytes of p->grid.
inline size_t grid_bytes(const gbri_plan* p) { return (size_t)p->K * p->K * 2 * real_bytes(p->prec); }

// One member of the batch executor's fused pass over several problems (k_steps_multi):
// a primal-dual solver with a global l2 ball on an FP32 step-layout plan.
struct FusedMember {
  const uint2* meta;
  const int2* steps;
  const int4* gtiles;
  const float2* spec;  // the member's half spectrum (the forward FFT of its x-hat)
  float2* grid;        // its gridding target, zeroed before the pass
  float2* u;           // l2-ball dual (plan order), updated in place
  const float2* y;     // data (plan order)
  double* c;           // ball scalar: read by every item, written by the last block
  double* dist;        // ||u|| / sigma2 after the pass
  double eps, sigma2d;
  float sigma2;
  int K, nT, log2S;
  int item0;           // first item of this member in the launch's numbering
  long long M;         // visibilities (bounds checks)
  unsigned int* dbg;   // GBRI_DEBUG builds: the plan's error word (else null)
};
constexpr int kMaxFusedMembers = 256;  // members of one shared pass
// Runs the fused degridding + gridding pass of n_mem members in one launch (device table
// d_mem, items numbered member after member, n_items in all; d_sums[n_mem] zero on entry and
// on exit; d_ctr a zeroed counter pair).
int32_t launch_fused_multi(const FusedMember* d_mem, int n_mem, int n_items, double* d_sums, const PolyTaps& poly,
                           unsigned int* d_ctr, cudaStream_t s);

// Sets the shared-memory attributes of every visibility kernel of one precision
// (once per process).
template <class R>
int32_t prepare_visibility_kernels();
// Z S x into p->padded; optional extra scaling by 1 / *d_norm (device, may be null).
template <class R>
int32_t launch_pad(gbri_plan* p, const R* x, const double* d_norm, cudaStream_t s);
// F: padded -> spec (forward, unnormalised, real-to-complex).
int32_t fft_forward(gbri_plan* p, cudaStream_t s);
// Re(F^H grid) alone, as R [K][K] at the start of p->grid (unnormalised): the Hermitian part
// of the grid folded into p->spec, then the complex-to-real inverse (spec is overwritten).
int32_t fft_inverse_real(gbri_plan* p, cudaStream_t s);
// S^T Z^T Re(F^H grid) into x (after fft_inverse_real).
template <class R>
int32_t launch_crop(gbri_plan* p, R* x, cudaStream_t s);

}  // namespace gbri
