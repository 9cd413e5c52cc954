// Plan creation (once per problem): FP64 quantisation of (u, v) to fixed-point
// grid coordinates, counting sort of the visibilities by (tile, cell), packed
// per-visibility metadata, work chunks, the pre-sampled Kaiser-Bessel table
// (Sec. 8.1) and the gridding correction (the S of Eq. 2), cuFFT plan.
//
// Kaiser-Bessel kernel (Sec. 7.3 names it, support J = 4; the formula is the
// standard one): g(t) = I0(beta sqrt(1 - (2t/J)^2)) / I0(beta) for |t| < J/2,
// 0 otherwise; its continuous Fourier transform is
// ghat(nu) = J sinh(sqrt(beta^2 - (pi J nu)^2)) / (I0(beta) sqrt(beta^2 - (pi J nu)^2)).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "nufft.cuh"

namespace gbri {
namespace {

double kb_g(double t, int J, double beta) {
  const double r = 2.0 * t / J;
  if (!(std::fabs(r) < 1.0)) return 0.0;
  return std::cyl_bessel_i(0.0, beta * std::sqrt(1.0 - r * r)) / std::cyl_bessel_i(0.0, beta);
}

double kb_ghat(double nu, int J, double beta) {
  const double s = beta * beta - (M_PI * J * nu) * (M_PI * J * nu);
  const double a = std::sqrt(std::fabs(s));
  double ratio = 1.0;
  if (a > 0.0) ratio = (s > 0.0) ? std::sinh(a) / a : std::sin(a) / a;
  return J * ratio / std::cyl_bessel_i(0.0, beta);
}

// Polynomial taps (kTapPoly): on each unit segment [k, k + 1] of the support, g(k + (z + 1) / 2)
// is interpolated at 32 Chebyshev nodes in z, truncated to degree 2 kPolyHalf - 1 and written
// in the monomial basis, split into its even and odd parts in z (FP64 on the host).  The fit is
// accepted when, with its coefficients rounded to FP32, it reproduces every sample of the
// zeroth-order table (the positions the kernels evaluate it at) to kPolyTol; otherwise the
// plan keeps the table.  g is an entire function of t (a power series in 1 - (2t/J)^2), so
// the Chebyshev coefficients fall off fast: degree 9 reaches ~5e-9 for J = 4 and 6 with
// beta = 2.34 J.  kPolyTol is near the FP32 table's own rounding (6e-8 of g(0) = 1).
constexpr double kPolyTol = 3e-7;

bool fit_poly_taps(gbri_plan* p) {
  if (p->prec != GBRI_F32 || p->interp != 0 || p->J / 2 > 3) return false;
  const int J = p->J, S = p->S;
  constexpr int N = 32, D = 2 * kPolyHalf - 1;
  PolyTaps pt{};
  for (int k = 0; k < J / 2; ++k) {
    double c[D + 1] = {};
    for (int m = 0; m <= D; ++m) {
      double acc = 0.0;
      for (int j = 0; j < N; ++j) {
        const double th = M_PI * (j + 0.5) / N;
        acc += kb_g(k + 0.5 * (std::cos(th) + 1.0), J, p->beta) * std::cos(m * th);
      }
      c[m] = acc * 2.0 / N;
    }
    c[0] *= 0.5;
    // monomial coefficients of sum_m c[m] T_m(z)
    double mono[D + 1] = {}, tprev[D + 1] = {}, tcur[D + 1] = {}, tnext[D + 1] = {};
    tprev[0] = 1.0;  // T_0
    tcur[1] = 1.0;   // T_1
    mono[0] += c[0];
    mono[1] += c[1];
    for (int m = 2; m <= D; ++m) {
      for (int i = 0; i <= D; ++i) tnext[i] = (i > 0 ? 2.0 * tcur[i - 1] : 0.0) - tprev[i];
      for (int i = 0; i <= D; ++i) {
        mono[i] += c[m] * tnext[i];
        tprev[i] = tcur[i];
        tcur[i] = tnext[i];
      }
    }
    for (int i = 0; i < kPolyHalf; ++i) {
      pt.e[k][i] = (float)mono[2 * i];
      pt.o[k][i] = (float)mono[2 * i + 1];
    }
  }
  // every table sample, from the FP32 coefficients (both taps of every segment)
  double worst = 0.0;
  for (int f = 0; f < S; ++f) {
    const double z = 2.0 * f / S - 1.0, u = z * z;
    for (int k = 0; k < J / 2; ++k) {
      double e = pt.e[k][kPolyHalf - 1], o = pt.o[k][kPolyHalf - 1];
      for (int i = kPolyHalf - 2; i >= 0; --i) {
        e = e * u + pt.e[k][i];
        o = o * u + pt.o[k][i];
      }
      const double lo = e + z * o, hi = e - z * o;  // distances k + f / S and k + 1 - f / S
      worst = std::max(worst, std::fabs(lo - kb_g(k + (double)f / S, J, p->beta)));
      if (!(k == J / 2 - 1 && f == 0))  // the edge tap at distance J / 2 is set to 0 explicitly
        worst = std::max(worst, std::fabs(hi - kb_g(k + 1 - (double)f / S, J, p->beta)));
    }
  }
  if (!(worst <= kPolyTol)) return false;
  p->poly = pt;
  return true;
}

// Per-visibility quantisation (Sec. 8.1, zeroth order): k~ = round_half_away(u * K S / (2 pi))
// in FP64, tile-major cell key, tile-local packed coordinates.
// lf = 0: zeroth order, q = k~ = round(k S); lf = kLog2FracSteps: first order, q = round(k S F)
// with F = 2^lf, the table sample floor(q / F) mod S packed like k~ and the fraction q mod F
// written to frac (caller's order).
__global__ void k_quantise(const float4* __restrict__ uvw, int64_t M, double scale, int K, int log2S, int lf,
                           int nT, int32_t* __restrict__ key, uint32_t* __restrict__ packed,
                           float* __restrict__ wt, uint16_t* __restrict__ frac, int32_t* __restrict__ counts,
                           int32_t* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int S = 1 << log2S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
    const float4 r = uvw[i];
    if (!isfinite(r.x) || !isfinite(r.y) || !isfinite(r.w)) {
      atomicOr(err, 1);
      key[i] = 0; packed[i] = 0; wt[i] = 0.f;
      if (frac) frac[i] = 0;
      continue;
    }
    if (fabsf(r.x) > 50.2654825f || fabsf(r.y) > 50.2654825f) {  // 16 pi
      atomicOr(err, 2);
      key[i] = 0; packed[i] = 0; wt[i] = 0.f;
      if (frac) frac[i] = 0;
      continue;
    }
    long long q[2];
    const float uv[2] = {r.x, r.y};
#pragma unroll
    for (int a = 0; a < 2; ++a) {
      const double prod = __dmul_rn((double)uv[a], scale);
      const double rnd = floor(__dadd_rn(fabs(prod), 0.5));
      q[a] = (long long)(prod < 0.0 ? -rnd : rnd);
    }
    // base cells floor(q / (S F)) (arithmetic shift = floor for negatives), table sample
    // floor(q / F) mod S, fraction q mod F
    const int bx = (int)(q[0] >> (log2S + lf)), by = (int)(q[1] >> (log2S + lf));
    const int fx = (int)((q[0] >> lf) & (S - 1)), fy = (int)((q[1] >> lf) & (S - 1));
    if (frac) frac[i] = (uint16_t)((q[0] & ((1 << lf) - 1)) | ((q[1] & ((1 << lf) - 1)) << 8));
    int cx = bx % K; if (cx < 0) cx += K;
    int cy = by % K; if (cy < 0) cy += K;
    const int tx = cx / kTile, ty = cy / kTile;
    const int lcx = cx - tx * kTile, lcy = cy - ty * kTile;
    const int k = ((ty * nT + tx) * kTile + lcy) * kTile + lcx;
    key[i] = k;
    packed[i] = (uint32_t)(lcx * S + fx) | ((uint32_t)(lcy * S + fy) << 16);
    wt[i] = r.w;
    atomicAdd(counts + k, 1);
  }
}

// ---- exclusive scan of int32 counts (3 phases) ---------------------------------
constexpr int kScanThreads = 1024, kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ int block_exclusive_scan(int v, int* sh, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += n;
  }
  if (lane == 31) sh[w] = x;
  __syncthreads();
  if (w == 0) {
    int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int n = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += n;
    }
    sh[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int warp_off = (w > 0) ? sh[w - 1] : 0;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

__global__ void k_scan_tile_sums(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int v = 0;
  for (int j = 0; j < kScanItems; ++j) v += (base + j < n) ? in[base + j] : 0;
  int tot;
  block_exclusive_scan(v, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t* __restrict__ sums, int n) {  // one block, in place, exclusive
  __shared__ int sh[32];
  int carry = 0;
  for (int b = 0; b < n; b += blockDim.x) {
    const int i = b + threadIdx.x;
    const int v = (i < n) ? sums[i] : 0;
    int tot;
    const int ex = block_exclusive_scan(v, sh, &tot);
    if (i < n) sums[i] = carry + ex;
    carry += tot;
  }
}

__global__ void k_scan_apply(const int32_t* __restrict__ in, int64_t n, const int32_t* __restrict__ sums,
                             int32_t* __restrict__ out /* n + 1 */) {
  __shared__ int sh[32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  int loc[kScanItems];
  int v = 0;
  for (int j = 0; j < kScanItems; ++j) {
    loc[j] = (base + j < n) ? in[base + j] : 0;
    v += loc[j];
  }
  int tot;
  int run = sums[blockIdx.x] + block_exclusive_scan(v, sh, &tot);
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < n) out[base + j] = run;
    run += loc[j];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[blockIdx.x] + tot;
}

__global__ void k_scatter(const int32_t* __restrict__ key, const uint32_t* __restrict__ packed,
                          const float* __restrict__ wt, int64_t M, int32_t* __restrict__ cursor,
                          uint2* __restrict__ meta, int32_t* __restrict__ perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += stride) {
    const int pos = atomicAdd(cursor + key[i], 1);
    meta[pos] = make_uint2(packed[i], __float_as_uint(wt[i]));
    perm[pos] = (int32_t)i;
  }
}

// Deterministic plans: the atomic scatter above leaves a cell's visibilities in a
// run-dependent order; sort every cell's segment by caller index (insertion sort, one thread
// per cell: segments are short, and this runs once per plan), so that the plan order, and
// with it every sum the kernels form, is the same in every run.
__global__ void k_sort_cells(const int32_t* __restrict__ off, int64_t cells, uint2* __restrict__ meta,
                             int32_t* __restrict__ perm) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
    const int lo = off[c], hi = off[c + 1];
    for (int i = lo + 1; i < hi; ++i) {
      const int32_t pk = perm[i];
      const uint2 mk = meta[i];
      int j = i - 1;
      while (j >= lo && perm[j] > pk) {
        perm[j + 1] = perm[j];
        meta[j + 1] = meta[j];
        --j;
      }
      perm[j + 1] = pk;
      meta[j + 1] = mk;
    }
  }
}

// out[pos] = in[perm[pos]]
__global__ void k_gather_u16(const uint16_t* __restrict__ in, const int32_t* __restrict__ perm,
                             uint16_t* __restrict__ out, int64_t M) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}

// Move every run (consecutive visibilities of one cell) from its cell-sorted place to
// its place in the run order: one thread per run.
__global__ void k_relayout(const int2* __restrict__ old_sub, const int32_t* __restrict__ new_start, int64_t n_sub,
                           const uint2* __restrict__ meta_in, const int32_t* __restrict__ perm_in,
                           uint2* __restrict__ meta_out, int32_t* __restrict__ perm_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sub; i += stride) {
    const int2 o = old_sub[i];
    const int d = new_start[i];
    for (int k = 0; k < o.y; ++k) {
      meta_out[d + k] = meta_in[o.x + k];
      perm_out[d + k] = perm_in[o.x + k];
    }
  }
}

// Step layout: move every run from its cell-sorted place to its step-major places.  Run i
// is lane i mod 32 of group i / 32, whose steps start at group_step[i / 32]; its k-th
// visibility goes to step k's first position plus the number of lanes below it holding a
// visibility at that step.  One thread per run.
__global__ void k_relayout_steps(const int2* __restrict__ old_sub, const int32_t* __restrict__ group_step,
                                 const int2* __restrict__ steps, int64_t n_sub, const uint2* __restrict__ meta_in,
                                 const int32_t* __restrict__ perm_in, uint2* __restrict__ meta_out,
                                 int32_t* __restrict__ perm_out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_sub; i += stride) {
    const int2 o = old_sub[i];
    const int32_t g0 = group_step[i >> 5];
    const unsigned below = (1u << (unsigned)(i & 31)) - 1u;
    for (int k = 0; k < o.y; ++k) {
      const int2 d = steps[g0 + k];
      const int dst = (d.x & 0x7fffffff) + __popc((unsigned)d.y & below);
      meta_out[dst] = meta_in[o.x + k];
      perm_out[dst] = perm_in[o.x + k];
    }
  }
}

__global__ void k_tile_starts(const int32_t* __restrict__ offsets, int n_tiles, int cells_per_tile,
                              int32_t* __restrict__ starts) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t <= n_tiles) starts[t] = offsets[(int64_t)t * cells_per_tile];
}

template <class T>
int32_t dmalloc(T** p, size_t n, int64_t* acct) {
  if (n == 0) n = 1;
  cudaError_t e = alloc_fault_injected() ? cudaErrorMemoryAllocation : cudaMalloc((void**)p, n * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_error(GBRI_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  if (acct) *acct += (int64_t)(n * sizeof(T));
  return GBRI_OK;
}

int32_t bmalloc(void** p, size_t bytes, int64_t* acct) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = alloc_fault_injected() ? cudaErrorMemoryAllocation : cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return set_error(GBRI_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  if (acct) *acct += (int64_t)bytes;
  return GBRI_OK;
}

// Device copy of an FP64 host table in the plan's precision (rounded once for FP32).
int32_t upload_real(void** dst, const std::vector<double>& v, int prec, int64_t* acct, cudaStream_t s) {
  const size_t rb = real_bytes(prec);
  GBRI_TRY(bmalloc(dst, v.size() * rb, acct));
  if (prec == GBRI_F64) {
    GBRI_CHECK_CUDA(cudaMemcpyAsync(*dst, v.data(), v.size() * rb, cudaMemcpyHostToDevice, s));
    GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
  } else {
    std::vector<float> f(v.begin(), v.end());
    GBRI_CHECK_CUDA(cudaMemcpyAsync(*dst, f.data(), f.size() * rb, cudaMemcpyHostToDevice, s));
    GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
  }
  return GBRI_OK;
}

int32_t scan_counts(const int32_t* counts, int64_t n, int32_t* offsets, cudaStream_t s) {
  const int64_t tiles = ceil_div(n, kScanTile);
  int32_t* sums = nullptr;
  GBRI_TRY(dmalloc(&sums, (size_t)tiles, nullptr));
  launch_begin(GBRI_K_OTHER, s);
  k_scan_tile_sums<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, n, sums);
  int32_t st = launch_end(GBRI_K_OTHER, s);
  if (st == GBRI_OK) {
    launch_begin(GBRI_K_OTHER, s);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, (int)tiles);
    st = launch_end(GBRI_K_OTHER, s);
  }
  if (st == GBRI_OK) {
    launch_begin(GBRI_K_OTHER, s);
    k_scan_apply<<<(unsigned)tiles, kScanThreads, 0, s>>>(counts, n, sums, offsets);
    st = launch_end(GBRI_K_OTHER, s);
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (st == GBRI_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize (scan)");
  cudaFree(sums);
  return st;
}

void destroy_plan(gbri_plan* p) {
  if (!p) return;
  cudaFree(p->meta);
  cudaFree(p->perm);
  cudaFree(p->frac);
  cudaFree(p->frac_in);
  cudaFree(p->chunks);
  cudaFree(p->subruns);
  cudaFree(p->steps);
  cudaFree(p->gtiles);
  cudaFree(p->wtab);
  cudaFree(p->corr);
  cudaFree(p->padded);
  cudaFree(p->spec);
  cudaFree(p->grid);
  cudaFree(p->vis_tmp);
  cudaFree(p->partials);
  cudaFree(p->scalars);
  cudaFree(p->work);
  cudaFree(p->dbg);
  cudaFree(p->slots);
  cudaFree(p->tile_items_off);
  cudaFree(p->tile_items);
  if (p->fft_r2c_ok) cufftDestroy(p->fft_r2c);
  if (p->fft_c2r_ok) cufftDestroy(p->fft_c2r);
  delete p;
}

// Band of a run of len visibilities: ceil(len / kBand).  The lanes of a warp take runs of one
// band where they can, so that they loop equally often (the fused pass takes two
// visibilities per step, gridding four; bands of two made both faster than bands of four:
// fused pass 207 -> 178 us with its dynamic items, gridding 118 -> 116 us).
constexpr int kBand = 2;
constexpr int kMaxBands = (kMaxRun + kBand - 1) / kBand;
inline int run_band(int len) { return (len + kBand - 1) / kBand; }

// Runs: at most R consecutive visibilities of one cell.  Within a tile they are listed
// round by round (every cell's first run, then every second one, ...; one round for
// tiles whose cells hold at most R visibilities), each round padded to a multiple of 32
// entries so that the lanes of a warp take runs of distinct cells.  Inside a round the
// runs go in bands of equal load rounds ceil(length / kBand), most first, so that the 32
// runs of a warp loop equally long; inside a band they are dealt round robin over the
// 16 eight-byte shared-memory bank slots of their cell's first accumulator / window word
// ((row * 21 + col) mod 16; cell order inside a slot), so that the 16 lanes of a
// half-warp hit distinct slots while enough slots are left.  Tiles are listed heaviest first.  The visibilities are
// stored in run order.  Work items: one gridding item per tile (its runs), and
// degridding chunks of at most kChunk consecutive visibilities of one tile.  (Re)builds
// p->meta, p->perm, p->subruns, p->gtiles, p->chunks from the cell-sorted arrays.
int32_t layout(gbri_plan* p, const std::vector<int32_t>& hoff, const std::vector<int32_t>& hst,
               const std::vector<int32_t>& order, int R, const uint2* meta_cell, const int32_t* perm_cell,
               cudaStream_t s) {
  const int64_t M = p->M;
  constexpr int NC = kTile * kTile;
  cudaFree(p->meta); cudaFree(p->perm); cudaFree(p->subruns); cudaFree(p->chunks); cudaFree(p->gtiles);
  p->meta = nullptr; p->perm = nullptr; p->subruns = nullptr; p->chunks = nullptr; p->gtiles = nullptr;
  cudaFree(p->slots); cudaFree(p->tile_items_off); cudaFree(p->tile_items);
  p->slots = nullptr; p->tile_items_off = nullptr; p->tile_items = nullptr;
  cudaFree(p->steps);
  p->steps = nullptr;
  p->n_steps = 0;
  // FP32 polynomial-tap plans with J = 4 store every 32-run group step-major (the step
  // kernels); the others keep each run's visibilities consecutive
  const bool steps = p->step_layout != 0;
  std::vector<int2> stp;         // step descriptors {first position | start << 31, lanes}
  std::vector<int32_t> gstep;    // first step of every 32-entry group of sub
  int64_t next_pos = 0;          // plan position of the next step's first visibility
  std::vector<int2> sub;
  sub.reserve((size_t)(M / std::max(R, 4) + order.size() * 64 + 16));
  std::vector<int4> ch, gt;
  int cnt[NC], nsub[NC];
  int64_t vis_base = 0;  // first plan position of the current tile
  // A gridding work item is one warp's: a tile heavier than twice a warp's share of the
  // visibilities (at full occupancy) is cut into items of whole 32-run groups of at most
  // that weight, which then flush with atomics on every cell (.w = 1); lighter tiles are one
  // item that writes its interior with plain stores.
  const int64_t warps = (int64_t)num_sms() * grid_occupancy((int)real_bytes(p->prec), p->J) * (kThreads / 32);
  const int64_t item_cap = std::max<int64_t>(1024, 2 * ((M + warps - 1) / warps));
  for (int t : order) {
    const int64_t base = (int64_t)t * NC;
    int maxsub = 0;
    for (int c = 0; c < NC; ++c) {
      cnt[c] = hoff[base + c + 1] - hoff[base + c];
      nsub[c] = (cnt[c] + R - 1) / R;
      maxsub = std::max(maxsub, nsub[c]);
    }
    const int64_t first = (int64_t)sub.size();
    for (int r = 0; r < maxsub; ++r) {
      int len[NC];
      int maxband = 0;
      int nin[kMaxBands + 1] = {0};
      for (int c = 0; c < NC; ++c) {
        len[c] = nsub[c] > r ? std::min(R, cnt[c] - r * R) : 0;
        if (len[c] > 0) {
          const int b = run_band(len[c]);
          maxband = std::max(maxband, b);
          ++nin[b];
        }
      }
      // cells by band, most rounds first, in cell order inside a band (counting sort) ...
      int start[kMaxBands + 2];
      start[maxband] = 0;
      for (int b = maxband; b >= 1; --b) start[b - 1] = start[b] + nin[b];
      int bycell[NC];
      {
        int fill[kMaxBands + 1];
        for (int b = 1; b <= maxband; ++b) fill[b] = start[b];
        for (int c = 0; c < NC; ++c)
          if (len[c] > 0) bycell[fill[run_band(len[c])]++] = c;
      }
      // ... and inside a band round robin over the bank slots, in cell order within a slot
      for (int band = maxband; band >= 1; --band) {
        int bucket[16][NC];
        int nb[16] = {0};
        for (int i = start[band]; i < start[band] + nin[band]; ++i) {
          const int c = bycell[i];
          const int slot = ((c / kTile) * kAccPitch2 + (c % kTile)) & 15;
          bucket[slot][nb[slot]++] = c;
        }
        int taken[16] = {0};
        for (bool any = true; any;) {
          any = false;
          for (int q = 0; q < 16; ++q)
            if (taken[q] < nb[q]) {
              const int c = bucket[q][taken[q]++];
              sub.push_back(make_int2(hoff[base + c] + r * R, len[c]));
              any = true;
            }
        }
      }
      while ((sub.size() - first) % 32) sub.push_back(make_int2(0, 0));
    }
    const int64_t nt = (int64_t)sub.size() - first;
    const int64_t nv_tile = hst[t + 1] - hst[t];
    if (steps) {  // the tile's groups step-major: step k holds the k-th visibility of each run
      for (int64_t g = first; g < first + nt; g += 32) {
        gstep.push_back((int32_t)stp.size());
        int maxlen = 0;
        for (int j = 0; j < 32; ++j) maxlen = std::max(maxlen, sub[g + j].y);
        for (int k = 0; k < maxlen; ++k) {
          unsigned mask = 0u;
          for (int j = 0; j < 32; ++j)
            if (sub[g + j].y > k) mask |= 1u << j;
          stp.push_back(make_int2((int)next_pos | (k == 0 ? (int)0x80000000u : 0), (int)mask));
          next_pos += __builtin_popcount(mask);
        }
      }
    }
    // an item's runs [a, b) of sub, as runs or (step layout) as steps
    auto item = [&](int64_t a, int64_t b, int split) {
      if (!steps) {
        gt.push_back(make_int4(t, (int)a, (int)(b - a), split));
        return;
      }
      const int64_t ga = a / 32, gb = b / 32;  // groups, relative to every group so far
      const int64_t sa = gstep[ga], sb = gb < (int64_t)gstep.size() ? gstep[gb] : (int64_t)stp.size();
      gt.push_back(make_int4(t, (int)sa, (int)(sb - sa), split));
    };
    if (nv_tile <= item_cap) {
      item(first, first + nt, 0);
    } else {
      int64_t g0 = first, w = 0;
      for (int64_t g = first; g < first + nt; g += 32) {
        int64_t wg = 0;
        for (int i = 0; i < 32; ++i) wg += sub[g + i].y;
        if (w > 0 && w + wg > item_cap) {
          item(g0, g, 1);
          g0 = g;
          w = 0;
        }
        w += wg;
      }
      item(g0, first + nt, 1);
    }
    const int64_t nv = hst[t + 1] - hst[t];
    const int64_t nch = (nv + kChunk - 1) / kChunk;
    for (int64_t k = 0; k < nch; ++k) {
      const int64_t a = vis_base + k * nv / nch, b = vis_base + (k + 1) * nv / nch;
      ch.push_back(make_int4(t, (int)a, (int)(b - a), 0));
    }
    vis_base += nv;
  }
  GBRI_CHECK((int64_t)sub.size() < ((int64_t)1 << 31), GBRI_EINVAL, "too many runs");
  std::vector<int32_t> nstart(sub.size());
  int64_t run = 0;
  for (size_t i = 0; i < sub.size(); ++i) {
    nstart[i] = (int32_t)run;
    run += sub[i].y;
  }
  p->n_chunks = (int64_t)ch.size();
  p->n_gtiles = (int64_t)gt.size();
  int32_t st = GBRI_OK;
  if ((st = dmalloc(&p->meta, (size_t)M, nullptr)) || (st = dmalloc(&p->perm, (size_t)M, nullptr)) ||
      (st = dmalloc(&p->chunks, ch.size(), nullptr)) ||
      (st = dmalloc(&p->subruns, steps ? 1 : sub.size(), nullptr)) || (st = dmalloc(&p->gtiles, gt.size(), nullptr)))
    return st;
  if (steps && !sub.empty()) {
    GBRI_CHECK(next_pos == M, GBRI_EINVAL, "step layout does not cover every visibility");
    p->n_steps = (int64_t)stp.size();
    if ((st = dmalloc(&p->steps, stp.size(), nullptr))) return st;
    int2* dold = nullptr;
    int32_t* dgs = nullptr;
    if ((st = dmalloc(&dold, sub.size(), nullptr)) || (st = dmalloc(&dgs, gstep.size(), nullptr))) {
      cudaFree(dold);
      return st;
    }
    cudaError_t e = cudaMemcpyAsync(p->steps, stp.data(), stp.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dold, sub.data(), sub.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dgs, gstep.data(), gstep.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "cudaMemcpyAsync (step layout)");
    } else {
      launch_begin(GBRI_K_OTHER, s);
      k_relayout_steps<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)sub.size(), 256), (int64_t)num_sms() * 16),
                         256, 0, s>>>(dold, dgs, p->steps, (int64_t)sub.size(), meta_cell, perm_cell, p->meta,
                                      p->perm);
      st = launch_end(GBRI_K_OTHER, s);
    }
    e = cudaStreamSynchronize(s);  // the host vectors are read by the copies
    if (st == GBRI_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize (step layout)");
    cudaFree(dold);
    cudaFree(dgs);
    if (st != GBRI_OK) return st;
  } else if (!sub.empty()) {
    int2* dold = nullptr;
    int32_t* dnew = nullptr;
    if ((st = dmalloc(&dold, sub.size(), nullptr)) || (st = dmalloc(&dnew, sub.size(), nullptr))) {
      cudaFree(dold);
      return st;
    }
    cudaError_t e = cudaMemcpyAsync(dold, sub.data(), sub.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dnew, nstart.data(), nstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "cudaMemcpyAsync (run layout)");
    } else {
      launch_begin(GBRI_K_OTHER, s);
      k_relayout<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)sub.size(), 256), (int64_t)num_sms() * 16), 256, 0,
                   s>>>(dold, dnew, (int64_t)sub.size(), meta_cell, perm_cell, p->meta, p->perm);
      st = launch_end(GBRI_K_OTHER, s);
    }
    // the host vectors are read by the copies: wait for them before anything goes out of scope
    e = cudaStreamSynchronize(s);
    if (st == GBRI_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize (run layout)");
    cudaFree(dold);
    cudaFree(dnew);
    if (st != GBRI_OK) return st;
    for (size_t i = 0; i < sub.size(); ++i) sub[i].x = nstart[i];
    GBRI_CHECK_CUDA(cudaMemcpyAsync(p->subruns, sub.data(), sub.size() * sizeof(int2), cudaMemcpyHostToDevice, s));
  }
  if (!ch.empty())
    GBRI_CHECK_CUDA(cudaMemcpyAsync(p->chunks, ch.data(), ch.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  if (!gt.empty())
    GBRI_CHECK_CUDA(cudaMemcpyAsync(p->gtiles, gt.data(), gt.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  p->layout_bytes = (int64_t)((steps ? stp.size() : sub.size()) * sizeof(int2) + (ch.size() + gt.size()) * sizeof(int4));
  std::vector<int32_t> toff, titems;
  if (p->det) {  // per-tile item lists (CSR over every tile, items ascending) and the window slots
    const int64_t ntiles = (int64_t)p->nT * p->nT;
    toff.assign((size_t)ntiles + 1, 0);
    for (const int4& g : gt) ++toff[(size_t)g.x + 1];
    for (int64_t t = 0; t < ntiles; ++t) toff[t + 1] += toff[t];
    titems.resize(gt.size());
    std::vector<int32_t> cur(toff.begin(), toff.end() - 1);
    for (size_t i = 0; i < gt.size(); ++i) titems[cur[gt[i].x]++] = (int32_t)i;
    const int P = kTile + p->J - 1;
    const size_t slot_bytes = (size_t)gt.size() * P * P * 2 * real_bytes(p->prec);
    if ((st = bmalloc(&p->slots, slot_bytes, nullptr)) || (st = dmalloc(&p->tile_items_off, toff.size(), nullptr)) ||
        (st = dmalloc(&p->tile_items, titems.size(), nullptr)))
      return st;
    GBRI_CHECK_CUDA(cudaMemcpyAsync(p->tile_items_off, toff.data(), toff.size() * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
    if (!titems.empty())
      GBRI_CHECK_CUDA(cudaMemcpyAsync(p->tile_items, titems.data(), titems.size() * sizeof(int32_t),
                                      cudaMemcpyHostToDevice, s));
    p->layout_bytes += (int64_t)(slot_bytes + (toff.size() + titems.size()) * sizeof(int32_t));
  }
  GBRI_CHECK_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  return GBRI_OK;
}

// Autotuner results per problem shape (grid size, support, table density, visibility
// count, non-empty tiles): run length and resident blocks per SM of both kernels.
struct TuneKey {
  int K, J, S, prec, interp;
  int64_t M, tiles;
  bool operator<(const TuneKey& o) const {
    return std::tie(K, J, S, prec, interp, M, tiles) < std::tie(o.K, o.J, o.S, o.prec, o.interp, o.M, o.tiles);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::array<int, 3>> g_tune;

bool tune_cache_get(const TuneKey& k, int* run, int* dg, int* gr) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(k);
  if (it == g_tune.end()) return false;
  *run = it->second[0];
  *dg = it->second[1];
  *gr = it->second[2];
  return true;
}

void tune_cache_put(const TuneKey& k, int run, int dg, int gr) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = {run, dg, gr};
}

// Plain degridding / gridding of the plan's scratch (autotuner timing).
void plain_degrid(gbri_plan* p, cudaStream_t s) {
  if (p->prec == GBRI_F64) launch_degrid(p, EpiStorePlan<double>{p->as<double2>(p->vis_tmp)}, s);
  else launch_degrid(p, EpiStorePlan<float>{p->as<float2>(p->vis_tmp)}, s);
}
void plain_grid(gbri_plan* p, cudaStream_t s) {
  if (p->prec == GBRI_F64) launch_grid(p, SrcPlan<double>{p->as<const double2>(p->vis_tmp)}, s);
  else launch_grid(p, SrcPlan<float>{p->as<const float2>(p->vis_tmp)}, s);
}

int32_t build_plan(gbri_plan* p, const float* d_uvw, cudaStream_t s) {
  GBRI_TRY(p->prec == GBRI_F64 ? prepare_visibility_kernels<double>() : prepare_visibility_kernels<float>());
  const int K = p->K, S = p->S;
  const int64_t M = p->M;
  const int64_t cells = (int64_t)K * K;
  const int n_tiles = p->nT * p->nT;

  // tables on the host in FP64, stored in the plan's precision (Sec. 8.1; the S factor of Eq. 2)
  const size_t rb = real_bytes(p->prec);
  {
    const int half = (p->J / 2) * S;
    std::vector<double> tab(half + 1);
    for (int i = 0; i <= half; ++i) tab[i] = kb_g((double)i / S, p->J, p->beta);
    std::vector<double> w((size_t)table_elems(S, p->J), 0.0);
    for (int f = 0; f <= S / 2; ++f)
      for (int t = 0; t < p->J; ++t) {
        const int d = std::abs(f + (p->J / 2 - 1 - t) * S);
        w[(size_t)f * p->J + t] = (d <= half) ? tab[d] : 0.0;
      }
    std::vector<double> corr(p->n_side);
    for (int i = 0; i < p->n_side; ++i) corr[i] = 1.0 / kb_ghat((double)(i - p->n_side / 2) / K, p->J, p->beta);
    GBRI_TRY(upload_real(&p->wtab, w, p->prec, &p->device_bytes, s));
    GBRI_TRY(upload_real(&p->corr, corr, p->prec, &p->device_bytes, s));
    // FP32 zeroth-order plans evaluate the kernel from its polynomial fit unless
    // GBRI_TAP_TABLE=1 asks for the shared-memory table (both give the table's weights)
    const char* force_table = std::getenv("GBRI_TAP_TABLE");
    const bool table_only = force_table && force_table[0] == '1';
    p->tap_mode = p->interp ? kTapFO : (!table_only && fit_poly_taps(p)) ? kTapPoly : kTapTable;
    // FP32 polynomial-tap plans with J = 4 take the step layout and its kernels unless the
    // caller asks for the run layout (each run's visibilities consecutive; the run kernels)
    p->step_layout = p->tap_mode == kTapPoly && p->J == 4 && p->layout_req == 0;
  }

  GBRI_TRY(dmalloc(&p->meta, (size_t)M, &p->device_bytes));
  GBRI_TRY(dmalloc(&p->perm, (size_t)M, &p->device_bytes));
  GBRI_TRY(bmalloc(&p->vis_tmp, (size_t)M * 2 * rb, &p->device_bytes));
  GBRI_TRY(bmalloc(&p->padded, (size_t)cells * rb, &p->device_bytes));
  GBRI_TRY(bmalloc(&p->spec, (size_t)K * (K / 2 + 1) * 2 * rb, &p->device_bytes));
  GBRI_TRY(bmalloc(&p->grid, (size_t)cells * 2 * rb, &p->device_bytes));
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->padded, 0, (size_t)cells * rb, s));

  // work arrays for the sort
  int32_t *key = nullptr, *counts = nullptr, *err = nullptr, *starts = nullptr;
  int32_t*& offsets = p->cell_off;  // kept: per-cell visibility ranges
  uint32_t* packed = nullptr;
  float* wt = nullptr;
  int32_t st = GBRI_OK;
  auto cleanup = [&]() {
    cudaFree(key); cudaFree(counts); cudaFree(err); cudaFree(packed); cudaFree(wt);
    cudaFree(starts);
  };
  if (p->interp) {  // caller-order fractions, gathered into plan order after the layout
    GBRI_TRY(dmalloc(&p->frac_in, (size_t)M, nullptr));
  }
  uint16_t* frac_in = p->frac_in;
  if ((st = dmalloc(&key, (size_t)M, nullptr)) || (st = dmalloc(&packed, (size_t)M, nullptr)) ||
      (st = dmalloc(&wt, (size_t)M, nullptr)) || (st = dmalloc(&counts, (size_t)cells, nullptr)) ||
      (st = dmalloc(&offsets, (size_t)cells + 1, &p->device_bytes)) || (st = dmalloc(&err, 1, nullptr)) ||
      (st = dmalloc(&starts, (size_t)n_tiles + 1, nullptr))) {
    cleanup();
    return st;
  }
  {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int32_t) * cells, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) {
      cleanup();
      return cuda_error(e, "cudaMemsetAsync (plan counts)");
    }
  }
  const int lf = p->interp ? kLog2FracSteps : 0;
  const double scale = (double)((int64_t)K * S << lf) / (2.0 * M_PI);
  const int vb = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(M, 256), 1), (int64_t)num_sms() * 16);
  launch_begin(GBRI_K_OTHER, s);
  k_quantise<<<vb, 256, 0, s>>>(reinterpret_cast<const float4*>(d_uvw), M, scale, K, p->log2S, lf, p->nT, key,
                                packed, wt, frac_in, counts, err);
  st = launch_end(GBRI_K_OTHER, s);
  if (st == GBRI_OK) st = scan_counts(counts, cells, offsets, s);
  int32_t herr = 0;
  if (st == GBRI_OK) {
    cudaError_t e = cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "quantise status");
    else if (herr & 1) st = set_error(GBRI_ENONFINITE, "non-finite u, v or weight");
    else if (herr & 2) st = set_error(GBRI_EINVAL, "|u| or |v| exceeds 16 pi");
  }
  if (st == GBRI_OK) {
    // cursor = offsets (reuse counts as the cursor array)
    const cudaError_t e = cudaMemcpyAsync(counts, offsets, sizeof(int32_t) * cells, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      st = cuda_error(e, "cudaMemcpyAsync (sort cursor)");
    } else {
      launch_begin(GBRI_K_OTHER, s);
      k_scatter<<<vb, 256, 0, s>>>(key, packed, wt, M, counts, p->meta, p->perm);
      st = launch_end(GBRI_K_OTHER, s);
      if (st == GBRI_OK && p->det) {
        launch_begin(GBRI_K_OTHER, s);
        k_sort_cells<<<(unsigned)std::min<int64_t>(ceil_div(cells, 256), (int64_t)num_sms() * 16), 256, 0, s>>>(
            offsets, cells, p->meta, p->perm);
        st = launch_end(GBRI_K_OTHER, s);
      }
    }
  }
  std::vector<int32_t> hst(n_tiles + 1);
  if (st == GBRI_OK) {
    launch_begin(GBRI_K_OTHER, s);
    k_tile_starts<<<(n_tiles + 1 + 255) / 256, 256, 0, s>>>(offsets, n_tiles, kTile * kTile, starts);
    st = launch_end(GBRI_K_OTHER, s);
  }
  if (st == GBRI_OK) {
    cudaError_t e = cudaMemcpyAsync(hst.data(), starts, sizeof(int32_t) * (n_tiles + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_error(e, "tile starts");
  }
  cleanup();
  if (st != GBRI_OK) return st;

  std::vector<int32_t> tiles;
  for (int t = 0; t < n_tiles; ++t)
    if (hst[t + 1] > hst[t]) tiles.push_back(t);
  p->n_tiles = (int64_t)tiles.size();
  std::vector<int32_t> hoff((size_t)cells + 1);
  {
    cudaError_t e = cudaMemcpyAsync(hoff.data(), p->cell_off, sizeof(int32_t) * (cells + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cell offsets");
  }
  cudaFree(p->cell_off);  // the kernels only need the sub-runs and chunks
  p->cell_off = nullptr;
  p->device_bytes -= (int64_t)(cells + 1) * (int64_t)sizeof(int32_t);
  std::vector<int32_t> order(tiles);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return hst[a + 1] - hst[a] > hst[b + 1] - hst[b]; });
  // the cell-sorted arrays stay the source of every layout tried below
  uint2* meta_cell = p->meta;
  int32_t* perm_cell = p->perm;
  p->meta = nullptr;
  p->perm = nullptr;
  p->device_bytes -= (int64_t)M * 12;
  const int sms = num_sms();
  const int lim_dg =
      std::min(std::max(1, (int)((227 * 1024) / (degrid_smem(p) + 1024))), degrid_occupancy((int)rb, p->J));
  // the pipelined FP32 polynomial-tap gridding kernel of the run layout is compiled for two
  // blocks per SM, the step layout's for three (80 registers; at M = 1e7: 126.9 us at two
  // blocks, 123.4 at three, 118.7 at three with the step loop unrolled by two)
  const int lim_gr = std::min(std::min(std::max(1, (int)((227 * 1024) / (grid_smem(p) + 1024))),
                                       grid_occupancy((int)rb, p->J)),
                              p->tap_mode == kTapPoly ? (p->step_layout ? 3 : 2) : 1 << 20);
  p->n_partials = std::max(sms * 8, 1024);
  GBRI_TRY(dmalloc(&p->partials, (size_t)p->n_partials * 4, &p->device_bytes));
  GBRI_TRY(dmalloc(&p->scalars, 64, &p->device_bytes));
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->scalars, 0, 64 * sizeof(double), s));
  GBRI_TRY(dmalloc(&p->work, 16, &p->device_bytes));
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->work, 0, 16 * sizeof(unsigned int), s));
#ifdef GBRI_DEBUG
  GBRI_TRY(dmalloc(&p->dbg, 4, &p->device_bytes));
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->dbg, 0, 4 * sizeof(unsigned int), s));
#endif
  // the padded image is real: the forward transform is real-to-complex (half the work of
  // C2C); degridding reads the other half through G[-k] = conj(G[k])
  if (cufftPlan2d(&p->fft_r2c, K, K, p->prec == GBRI_F64 ? CUFFT_D2Z : CUFFT_R2C) != CUFFT_SUCCESS) {
    cudaFree(meta_cell); cudaFree(perm_cell);
    return set_error(GBRI_ECUFFT, "cufftPlan2d (real-to-complex) failed");
  }
  p->fft_r2c_ok = true;
  // every reader of the adjoint's inverse transform (crop, the solvers' updates) takes only
  // its real part: the complex-to-real inverse of the grid's Hermitian part gives it with
  // about half the work of the complex inverse
  if (cufftPlan2d(&p->fft_c2r, K, K, p->prec == GBRI_F64 ? CUFFT_Z2D : CUFFT_C2R) != CUFFT_SUCCESS) {
    cudaFree(meta_cell); cudaFree(perm_cell);
    return set_error(GBRI_ECUFFT, "cufftPlan2d (complex-to-real) failed");
  }
  p->fft_c2r_ok = true;
  {
    size_t ws1 = 0, ws2 = 0;
    if (cufftGetSize(p->fft_r2c, &ws1) == CUFFT_SUCCESS && cufftGetSize(p->fft_c2r, &ws2) == CUFFT_SUCCESS)
      p->device_bytes += (int64_t)(ws1 + ws2);
  }

  auto set_blocks = [&](int bpm_dg, int bpm_gr) {
    // one degridding chunk per warp
    p->degrid_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(p->n_chunks, kThreads / 32), (int64_t)sms * bpm_dg));
    // one gridding work item per warp
    p->grid_blocks =
        (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(p->n_gtiles, kThreads / 32), (int64_t)sms * bpm_gr));
  };
  int best_run = p->run_len, best_dg = lim_dg, best_gr = lim_gr;
  const TuneKey tkey{K, p->J, S, p->prec, p->interp, M, p->n_tiles};
  bool cached = false;
  if (p->autotune) cached = tune_cache_get(tkey, &best_run, &best_dg, &best_gr);
  if (p->autotune && !cached && M > 0) {
    // time the plain degridding and gridding kernels for every run length and
    // persistent-grid size, keep the pair with the smallest summed time
    float best = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      st = set_error(GBRI_ECUDA, "cudaEventCreate (autotune)");
    const int runs[3] = {8, 16, 64};
    for (int R : runs) {
      if (st != GBRI_OK) break;
      st = layout(p, hoff, hst, order, R, meta_cell, perm_cell, s);
      if (st != GBRI_OK) break;
      float tdg[8] = {0}, tgr[8] = {0};
      for (int b = 1; b <= std::max(lim_dg, lim_gr); ++b) {
        set_blocks(std::min(b, lim_dg), std::min(b, lim_gr));
        for (int rep = 0; rep < 3; ++rep) {  // rep 0 warms up
          float ms = 0.f;
          cudaEventRecord(e0, s);
          if (b <= lim_dg) plain_degrid(p, s);
          cudaEventRecord(e1, s);
          cudaError_t e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (rep) tdg[b] += ms;
          cudaEventRecord(e0, s);
          if (b <= lim_gr) plain_grid(p, s);
          cudaEventRecord(e1, s);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (rep) tgr[b] += ms;
          if (e != cudaSuccess && st == GBRI_OK) st = cuda_error(e, "autotune timing");
        }
      }
      int bd = 1, bg = 1;
      for (int b = 1; b <= lim_dg; ++b)
        if (tdg[b] < tdg[bd]) bd = b;
      for (int b = 1; b <= lim_gr; ++b)
        if (tgr[b] < tgr[bg]) bg = b;
      if (tdg[bd] + tgr[bg] < best) {
        best = tdg[bd] + tgr[bg];
        best_run = R;
        best_dg = bd;
        best_gr = bg;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st == GBRI_OK) tune_cache_put(tkey, best_run, best_dg, best_gr);
  }
  if (st == GBRI_OK) st = layout(p, hoff, hst, order, best_run, meta_cell, perm_cell, s);
  {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st == GBRI_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize (plan layout)");
  }
  cudaFree(meta_cell);
  cudaFree(perm_cell);
  if (st == GBRI_OK && p->interp) {  // first-order fractions into plan order
    st = dmalloc(&p->frac, (size_t)M, &p->device_bytes);
    if (st == GBRI_OK && M > 0) {
      launch_begin(GBRI_K_OTHER, s);
      k_gather_u16<<<(unsigned)std::min<int64_t>(ceil_div(M, 256), (int64_t)num_sms() * 16), 256, 0, s>>>(
          p->frac_in, p->perm, p->frac, M);
      st = launch_end(GBRI_K_OTHER, s);
    }
    const cudaError_t e = cudaStreamSynchronize(s);
    if (st == GBRI_OK && e != cudaSuccess) st = cuda_error(e, "cudaStreamSynchronize (fractions)");
    cudaFree(p->frac_in);
    p->frac_in = nullptr;
  }
  if (st != GBRI_OK) return st;
  p->run_len = best_run;
  set_blocks(best_dg, best_gr);
  p->device_bytes += (int64_t)M * 12 + p->layout_bytes;
  GBRI_CHECK_CUDA(cudaMemsetAsync(p->grid, 0, (size_t)cells * 2 * rb, s));
  GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
  return GBRI_OK;
}

}  // namespace
}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_plan_create(gbri_plan** out, const gbri_plan_desc* d, const float* d_uvw, void* stream) {
  GBRI_CHECK(out && d, GBRI_EINVAL, "null argument");
  *out = nullptr;
  GBRI_CHECK(d->deterministic == 0 || d->deterministic == 1, GBRI_EINVAL, "deterministic must be 0 or 1");
  GBRI_CHECK(d->layout == 0 || d->layout == 1, GBRI_EINVAL, "layout must be 0 or 1");
  GBRI_CHECK(d->precision == GBRI_F32 || d->precision == GBRI_F64, GBRI_EINVAL, "precision must be GBRI_F32 or GBRI_F64");
  GBRI_CHECK(d->n_side >= 16 && d->n_side % 2 == 0, GBRI_EINVAL, "n_side must be even and >= 16");
  GBRI_CHECK(d->oversample >= 2 && d->oversample <= 4, GBRI_EINVAL, "oversample must be in [2, 4]");
  GBRI_CHECK(d->J == 4 || d->J == 6, GBRI_EINVAL, "J must be 4 or 6");
  const int S = d->samples_per_unit;
  GBRI_CHECK(S >= 16 && S <= 4096 && (S & (S - 1)) == 0, GBRI_EINVAL,
             "samples_per_unit must be a power of two in [16, 4096]");
  GBRI_CHECK(d->M >= 0 && d->M < (int64_t)1 << 31, GBRI_EINVAL, "M must be in [0, 2^31)");
  GBRI_CHECK(d->M == 0 || d_uvw, GBRI_EINVAL, "null uvw");
  const int64_t K = (int64_t)d->oversample * d->n_side;
  GBRI_CHECK(K % kTile == 0, GBRI_EINVAL, "oversample * n_side must be a multiple of 16");
  GBRI_CHECK(K <= 16384, GBRI_EINVAL, "grid larger than 16384^2 is not supported");
  GBRI_CHECK(d->vis_per_run >= 0 && d->vis_per_run <= kMaxRun, GBRI_EINVAL, "vis_per_run must be in [0, 1024]");
  GBRI_CHECK(d->autotune == 0 || d->autotune == 1, GBRI_EINVAL, "autotune must be 0 or 1");
  GBRI_CHECK(d->interp_order == 0 || d->interp_order == 1, GBRI_EINVAL, "interp_order must be 0 or 1");
  gbri_plan* p = new (std::nothrow) gbri_plan();
  GBRI_CHECK(p, GBRI_ENOMEM, "host allocation");
  p->n_side = d->n_side;
  p->K = (int)K;
  p->J = d->J;
  p->S = S;
  p->log2S = 0;
  while ((1 << p->log2S) < S) ++p->log2S;
  p->nT = (int)(K / kTile);
  p->beta = d->kb_beta > 0 ? d->kb_beta : 2.34 * d->J;
  p->M = d->M;
  p->prec = d->precision;
  p->run_len = d->vis_per_run ? d->vis_per_run : kDefaultRun;
  p->interp = d->interp_order;
  p->det = d->deterministic;
  p->layout_req = d->layout;
  p->autotune = d->deterministic ? 0 : d->autotune;  // timed choices would make the layout vary
  const int32_t st = build_plan(p, d_uvw, (cudaStream_t)stream);
  if (st != GBRI_OK) {
    destroy_plan(p);
    return st;
  }
  *out = p;
  return GBRI_OK;
}

int32_t gbri_plan_destroy(gbri_plan* p) {
  if (p) cudaDeviceSynchronize();
  destroy_plan(p);
  return GBRI_OK;
}

int32_t gbri_plan_launch_config(const gbri_plan* p, int32_t* run, int32_t* dg, int32_t* gr) {
  GBRI_CHECK(p, GBRI_EINVAL, "null plan");
  if (run) *run = p->run_len;
  if (dg) *dg = p->degrid_blocks;
  if (gr) *gr = p->grid_blocks;
  return GBRI_OK;
}

int32_t gbri_plan_debug_word(const gbri_plan* p, uint32_t* bits, int64_t* first_index, int32_t reset,
                             void* stream) {
  GBRI_CHECK(p && bits, GBRI_EINVAL, "null argument");
  GBRI_CHECK(p->dbg, GBRI_EINVAL, "the library was built without GBRI_DEBUG bounds checks");
  uint32_t h[4] = {0, 0, 0, 0};
  cudaStream_t s = (cudaStream_t)stream;
  GBRI_CHECK_CUDA(cudaMemcpyAsync(h, p->dbg, sizeof(h), cudaMemcpyDeviceToHost, s));
  if (reset) GBRI_CHECK_CUDA(cudaMemsetAsync(p->dbg, 0, sizeof(h), s));
  GBRI_CHECK_CUDA(cudaStreamSynchronize(s));
  *bits = h[0];
  if (first_index) {
    int64_t v = 0;
    std::memcpy(&v, &h[2], sizeof(v));
    *first_index = v;
  }
  return GBRI_OK;
}

int32_t gbri_plan_tap_mode(const gbri_plan* p, int32_t* mode) {
  GBRI_CHECK(p && mode, GBRI_EINVAL, "null argument");
  *mode = p->tap_mode;
  return GBRI_OK;
}

int32_t gbri_plan_info(const gbri_plan* p, int64_t* K, int64_t* M, int64_t* n_tiles, int64_t* bytes) {
  GBRI_CHECK(p, GBRI_EINVAL, "null plan");
  if (K) *K = p->K;
  if (M) *M = p->M;
  if (n_tiles) *n_tiles = p->n_tiles;
  if (bytes) *bytes = p->device_bytes;
  return GBRI_OK;
}

int32_t gbri_plan_permutation(const gbri_plan* p, int32_t* d_perm, void* stream) {
  GBRI_CHECK(p && (d_perm || p->M == 0), GBRI_EINVAL, "null argument");
  if (p->M == 0) return GBRI_OK;
  GBRI_CHECK_CUDA(cudaMemcpyAsync(d_perm, p->perm, sizeof(int32_t) * p->M, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
  return GBRI_OK;
}

}  // extern "C"
