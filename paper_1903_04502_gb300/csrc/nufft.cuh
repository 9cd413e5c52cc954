// Measurement operator Phi = W G F Z S (Sec. 2, Eq. 2) on one GPU: the plan
// object and the kernel templates shared by the operator calls and the solvers.
//
// Data layout in HBM (per plan):
//   meta   [M] uint2   plan (sorted) order: .x = (ly << 16) | lx, the tile-local
//                      fixed-point coordinates (cell-in-tile * S + fraction),
//                      .y = weight bits (float).  8 bytes per visibility.
//   perm   [M] int32   plan position -> caller's visibility index.
//   subruns [R] int2   {first plan position, count <= kRun}: consecutive visibilities
//                      of one cell; within a tile listed rank-major (all cells' first
//                      sub-runs in cell order, then all second sub-runs, ...).
//   chunks [C] int4    {tile, first sub-run, sub-runs (<= kThreads), single}; single =
//                      the tile is one chunk.
//   Visibilities are sorted by (tile, cell row, cell column): a cell's visibilities
//   are contiguous.
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
constexpr int kThreads = 256;  // threads per block of the visibility kernels
constexpr int kRun = 4;        // consecutive visibilities a thread owns within a chunk
constexpr int kChunk = kThreads * kRun;  // visibilities per work chunk
constexpr int kWinPitch = 21;  // float2 pitch of the degridding window (same bank-slot map as the gridding accumulators)

}  // namespace gbri

struct gbri_plan {
  int n_side = 0, K = 0, J = 0, S = 0, log2S = 0, nT = 0, prec = 0;
  double beta = 0;
  int64_t M = 0;
  uint2* meta = nullptr;
  int32_t* perm = nullptr;
  int4* chunks = nullptr;
  int2* subruns = nullptr;  // {first plan position, count <= kRun}: visibilities of one cell
  int64_t n_chunks = 0;
  int64_t n_tiles = 0;  // non-empty tiles
  int32_t* cell_off = nullptr;  // plan creation only
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
  int64_t layout_bytes = 0;
  int degrid_blocks = 0, grid_blocks = 0;
  int run_len = 4;  // visibilities per sub-run (<= kRun)
  int autotune = 0;
};

namespace gbri {

__device__ __forceinline__ int wrapK(int v, int K) { return v < 0 ? v + K : (v >= K ? v - K : v); }

// Load the J tap weights of one axis for fractional offset f (0 <= f < S) from the
// shared table.  The table stores rows f = 0 .. S/2 only: row S - f is row f reversed
// (entry t of row f is table[|f + (J/2 - 1 - t) S|]).
template <int J>
__device__ __forceinline__ void load_taps(const float* sw, int f, int S, float (&w)[J]) {
  const bool rev = f > (S >> 1);
  const int row = rev ? S - f : f;
  float v[J];
  if constexpr (J == 4) {
    const float4 q = reinterpret_cast<const float4*>(sw)[row];
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (J == 6) {
    const float2* p = reinterpret_cast<const float2*>(sw + row * 6);
    const float2 a = p[0], b = p[1], c = p[2];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; v[4] = c.x; v[5] = c.y;
  } else {
#pragma unroll
    for (int t = 0; t < J; ++t) v[t] = sw[row * J + t];
  }
#pragma unroll
  for (int t = 0; t < J; ++t) w[t] = rev ? v[J - 1 - t] : v[t];
}

// floats of the stored tap table (rows 0 .. S/2), rounded up to a whole float4
__host__ __device__ inline int table_floats(int S, int J) { return (((S / 2 + 1) * J) + 3) & ~3; }

__device__ __forceinline__ void copy_table_to_smem(float* sw, const float* __restrict__ g, int nfloats) {
  const float4* g4 = reinterpret_cast<const float4*>(g);
  float4* s4 = reinterpret_cast<float4*>(sw);
  for (int i = threadIdx.x; i < nfloats / 4; i += blockDim.x) s4[i] = __ldg(g4 + i);
}

struct VisGeom {
  const uint2* __restrict__ meta;
  const int4* __restrict__ chunks;
  const int2* __restrict__ subruns;
  const float* __restrict__ wtab;
  int n_chunks, K, log2S, nT;
};

inline size_t degrid_smem(const gbri_plan* p) {
  return (size_t)table_floats(p->S, p->J) * sizeof(float) + (size_t)(kTile + p->J - 1) * kWinPitch * sizeof(float2);
}
// gridding accumulator: (T + J - 1) rows, planar re / im, row pitch kAccPitch (== 16 mod 32
// so that the two tile rows of a warp fall on disjoint banks)
constexpr int kAccPitch = 48;
// warp-private gridding accumulators: float2 cells, row pitch kAccPitch2 (>= T + J - 1)
constexpr int kAccPitch2 = 21;
inline size_t grid_smem(const gbri_plan* p) {
  const int P = kTile + p->J - 1;
  return (size_t)table_floats(p->S, p->J) * sizeof(float) + (size_t)(kThreads / 32) * P * kAccPitch2 * sizeof(float2);
}

inline VisGeom vis_geom(const gbri_plan* p) {
  VisGeom g;
  g.meta = p->meta;
  g.chunks = p->chunks;
  g.subruns = p->subruns;
  g.wtab = p->wtab;
  g.n_chunks = (int)p->n_chunks;
  g.K = p->K;
  g.log2S = p->log2S;
  g.nT = p->nT;
  return g;
}

// ---- epilogues / sources ------------------------------------------------------
// A degridding epilogue has two phases so that its global loads can be issued
// together with the metadata loads: Pre p = load(pos); ...; store(pos, p, v).
struct EpiStorePlan {  // y[pos] = v
  float2* y;
  struct Pre {};
  __device__ __forceinline__ Pre load(int) const { return Pre{}; }
  __device__ __forceinline__ void store(int pos, const Pre&, float2 v) { y[pos] = v; }
  __device__ __forceinline__ void finish() {}
};
struct EpiStoreRaw {  // y[perm[pos]] = v
  float2* y;
  const int32_t* perm;
  struct Pre { int dst; };
  __device__ __forceinline__ Pre load(int pos) const { return Pre{perm[pos]}; }
  __device__ __forceinline__ void store(int, const Pre& p, float2 v) { y[p.dst] = v; }
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

// Solver epilogues (fused dual updates; see solver.cu for the algebra).
struct EpiPD1 {
  float2* u;
  const float2* y;
  const double* c;
  double* partials;
  float sigma2;
  KahanF acc;
  struct Pre { float2 u, y; };
  __device__ __forceinline__ Pre load(int pos) const { return Pre{u[pos], y[pos]}; }
  __device__ __forceinline__ void store(int pos, const Pre& p, float2 phi) {
    const float cc = (float)*c;  // broadcast load, cached
    const float2 un = make_float2(fmaf(cc, p.u.x, sigma2 * (phi.x - p.y.x)), fmaf(cc, p.u.y, sigma2 * (phi.y - p.y.y)));
    u[pos] = un;
    acc.add(fmaf(un.x, un.x, un.y * un.y));
  }
  __device__ __forceinline__ void finish() {
    __shared__ double sh[40];
    const double v = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
};

struct EpiADMM1 {  // w = Phi x + s - y, partial ||w||^2
  float2* w;
  const float2* sv;
  const float2* y;
  double* partials;
  KahanF acc;
  struct Pre { float2 s, y; };
  __device__ __forceinline__ Pre load(int pos) const { return Pre{sv[pos], y[pos]}; }
  __device__ __forceinline__ void store(int pos, const Pre& p, float2 v) {
    const float2 r = make_float2(v.x + p.s.x - p.y.x, v.y + p.s.y - p.y.y);
    w[pos] = r;
    acc.add(fmaf(r.x, r.x, r.y * r.y));
  }
  __device__ __forceinline__ void finish() {
    __shared__ double sh[40];
    const double v = block_sum(acc.value(), sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
  }
};

struct SrcADMM2 {  // s+ = s + varrho((1 - rho_b) w - s); source q = (1 - rho_b) w - s + s+
  const float2* w;
  float2* sv;
  const double* rho_b;
  float varrho;
  __device__ __forceinline__ float2 operator()(int pos) const {
    const float one_m = (float)(1.0 - *rho_b);
    const float2 ww = w[pos], so = sv[pos];
    const float2 pw = make_float2(one_m * ww.x, one_m * ww.y);
    const float2 sn = make_float2(fmaf(varrho, pw.x - so.x, so.x), fmaf(varrho, pw.y - so.y, so.y));
    sv[pos] = sn;
    return make_float2(pw.x - so.x + sn.x, pw.y - so.y + sn.y);
  }
};

// ---- launch helpers (defined in nufft.cu with explicit instantiations, so that each
// kernel template is instantiated in exactly one translation unit) ----------------
template <class Epi>
int32_t launch_degrid(gbri_plan* p, const float2* grid, Epi epi, cudaStream_t s);
// Zeroes p->grid, then grids every visibility into it.
template <class Src>
int32_t launch_grid(gbri_plan* p, Src src, cudaStream_t s);

// Sets the shared-memory attributes of every visibility kernel (once per process).
int32_t prepare_visibility_kernels();
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
