// SARA dictionary kernels: periodic 2-D Daubechies analysis (Psi^dagger) and
// synthesis (Psi), rows then columns per level, Mallat layout, batched over the
// non-Dirac bases (blockIdx.y); the Dirac basis is an elementwise copy.
//
// One level of the 1-D periodic analysis of a length-m signal:
//   a[k] = sum_i h[i] x[(2k + i) mod m],   d[k] = sum_i g[i] x[(2k + i) mod m],
// g[i] = (-1)^i h[L-1-i]; the synthesis is its transpose.
#include <cmath>
#include <cstdint>
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

template <class R>
__device__ __forceinline__ void emit(R* __restrict__ out, size_t q, R v, const EpiR<R>& e) {
  if (e.mode == 0) {
    out[q] = v;
  } else {
    const R u = fma_r(e.ca, out[q], e.cb * v);
    const R lim = e.w ? e.lim * e.w[q] : e.lim;
    out[q] = min_r(max_r(u, -lim), lim) * e.ce;
  }
}

// The epilogue's value for v given the output's current value prev and weight wq (mode 0:
// v itself); emit_pre() stores it.  The current value is read ahead of the filtering, so that
// the load's latency overlaps the block's work; the same arithmetic as emit().
template <class R>
__device__ __forceinline__ R epi_value(R v, const EpiR<R>& e, R prev, R wq) {
  if (e.mode == 0) return v;
  const R u = fma_r(e.ca, prev, e.cb * v);
  const R lim = e.w ? e.lim * wq : e.lim;
  return min_r(max_r(u, -lim), lim) * e.ce;
}
template <class R>
__device__ __forceinline__ void emit_pre(R* __restrict__ out, size_t q, R v, const EpiR<R>& e, R prev, R wq) {
  out[q] = epi_value(v, e, prev, wq);
}

constexpr int kAB = 16;                         // analysis: output coefficients per block side (per quadrant)
constexpr int kATile = 2 * kAB + kMaxTaps - 2;  // input rows / cols a block reads
constexpr int kSB = 32;                         // synthesis: output samples per block side
constexpr int kSK = kSB / 2 + kMaxTaps / 2 - 1; // coefficient rows / cols per half a block reads

template <class R>
struct AnaSmem {
  R tin[kATile][kATile + 1];
  R trow[kATile][2 * kAB + 1];
};
// Row pitch of the column-synthesis output: 16 (mod 32) words, so that the two rows a
// warp reads in the row synthesis (16 lanes each) fall on disjoint banks.
constexpr int kTmPitch = 2 * kSK <= 48 ? 48 : 80;
template <class R>
struct SynSmem {
  R tc[2 * kSK][2 * kSK + 1];  // [a|d rows][a|d cols]
  R tm[kSB][kTmPitch];         // after the column synthesis
};

// One analysis level of one basis with an L-tap filter pair (unrolled), block
// (blockIdx.x, blockIdx.y) = 16 x 16 output coefficients of each quadrant.  Written for
// latency: every element of the input window and the epilogue's current outputs are
// loaded into registers before the first use, so that the block waits for one round of
// L2 / HBM latency instead of one per loop trip; the row and column filters are
// register-blocked (a thread filters two neighbouring outputs from one sliding window of
// L + 2 samples).  Each output's sum runs over the taps in the same order as a plain
// loop, so the coefficients are those of the one-output-per-thread form.
template <int L, class R>
__device__ __forceinline__ void dwt_block(AnaSmem<R>& sm, const R* __restrict__ src, R* __restrict__ carry,
                                          R* __restrict__ dst, int m, int n, bool last, R scale,
                                          const R* __restrict__ hf, const R* __restrict__ gf, const EpiR<R>& e) {
  constexpr int T = 2 * kAB + L - 2;
  constexpr int NL = (T * T + 255) / 256;  // window elements per thread
  static_assert(kAB == 16 && T <= kATile, "block shape");
  const int half = m >> 1;
  const int k0 = blockIdx.y * kAB, l0 = blockIdx.x * kAB;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const bool interior = 2 * k0 + T <= m && 2 * l0 + T <= m;  // no periodic wrap
  // interior blocks of an FP32 level whose window rows start 16-byte aligned and end inside
  // the image row load the window as float4 (a quarter of the load and index instructions)
  constexpr int T4 = (T + 3) / 4;
  constexpr int NL4 = (T * T4 + 255) / 256;
  bool vec = false;
  if constexpr (sizeof(R) == 4)
    vec = interior && (n & 3) == 0 && 2 * l0 + 4 * T4 <= m && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  R v[NL];
  float4 v4[NL4];
  if (vec) {
#pragma unroll
    for (int k = 0; k < NL4; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < T * T4) {
        const int rr = idx / T4, c4 = idx - rr * T4;
        v4[k] = *reinterpret_cast<const float4*>(src + (size_t)(2 * k0 + rr) * n + 2 * l0 + 4 * c4);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < T * T) {
        const int rr = idx / T, cc = idx - rr * T;
        int gr = 2 * k0 + rr, gc = 2 * l0 + cc;
        if (!interior) {
          gr = gr < m ? gr : gr % m;
          gc = gc < m ? gc : gc % m;
        }
        v[k] = src[(size_t)gr * n + gc];
      }
    }
  }
  // this thread's outputs: column c of the [a | d] halves, rows kA and kA + 1 of the block
  const int c = tx;
  const int kA = 2 * ty;
  const int ll_ = l0 + (c & (kAB - 1));
  const int col = (c < kAB) ? ll_ : half + ll_;
  const bool lo_final = !(c < kAB && !last);  // else the LL value is carried to the next level
  R pv[4] = {0, 0, 0, 0}, pw[4] = {0, 0, 0, 0};
  if (e.mode != 0) {
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int kk = k0 + kA + i;
      if (kk < half && ll_ < half) {
        const size_t qlo = (size_t)kk * n + col, qhi = (size_t)(half + kk) * n + col;
        if (lo_final) pv[2 * i] = dst[qlo];
        pv[2 * i + 1] = dst[qhi];
        if (e.w) {
          if (lo_final) pw[2 * i] = e.w[qlo];
          pw[2 * i + 1] = e.w[qhi];
        }
      }
    }
  }
  R h[L], g[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    h[i] = hf[i];
    g[i] = gf[i];
  }
  if (vec) {
#pragma unroll
    for (int k = 0; k < NL4; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < T * T4) {
        const int rr = idx / T4, c4 = idx - rr * T4;
        const float e4[4] = {v4[k].x, v4[k].y, v4[k].z, v4[k].w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (4 * c4 + j < T) sm.tin[rr][4 * c4 + j] = (R)e4[j];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < T * T) {
        const int rr = idx / T;
        sm.tin[rr][idx - rr * T] = v[k];
      }
    }
  }
  __syncthreads();
  {  // rows: thread (row rr, pair p) -> a and d of outputs 2p, 2p + 1 from samples 4p .. 4p + L + 1
    const int p = threadIdx.x & 7;
    for (int rr = threadIdx.x >> 3; rr < T; rr += 32) {
      const R* row = &sm.tin[rr][4 * p];
      R a0 = 0, a1 = 0, d0 = 0, d1 = 0;
#pragma unroll
      for (int i = 0; i < L + 2; ++i) {
        const R x = row[i];
        if (i < L) {
          a0 = fma_r(h[i], x, a0);
          d0 = fma_r(g[i], x, d0);
        }
        if (i >= 2) {
          a1 = fma_r(h[i - 2], x, a1);
          d1 = fma_r(g[i - 2], x, d1);
        }
      }
      sm.trow[rr][2 * p] = a0;
      sm.trow[rr][2 * p + 1] = a1;
      sm.trow[rr][kAB + 2 * p] = d0;
      sm.trow[rr][kAB + 2 * p + 1] = d1;
    }
  }
  __syncthreads();
  // columns: rows 2 kA .. 2 kA + L + 1 of column c give outputs kA and kA + 1
  R lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
  for (int i = 0; i < L + 2; ++i) {
    const R x = sm.trow[2 * kA + i][c];
    if (i < L) {
      lo0 = fma_r(h[i], x, lo0);
      hi0 = fma_r(g[i], x, hi0);
    }
    if (i >= 2) {
      lo1 = fma_r(h[i - 2], x, lo1);
      hi1 = fma_r(g[i - 2], x, hi1);
    }
  }
  const R lo[2] = {lo0, lo1}, hi[2] = {hi0, hi1};
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int kk = k0 + kA + i;
    if (kk >= half || ll_ >= half) continue;
    const size_t qlo = (size_t)kk * n + col;
    if (!lo_final) carry[qlo] = lo[i];
    else emit_pre(dst, qlo, scale * lo[i], e, pv[2 * i], pw[2 * i]);
    emit_pre(dst, (size_t)(half + kk) * n + col, scale * hi[i], e, pv[2 * i + 1], pw[2 * i + 1]);
  }
}

// One analysis level at block size m (pitch n) for basis blockIdx.z, fused rows + columns:
// the block reads the (2*16 + L - 2)^2 input window (periodic), filters its rows into
// [a | d] halves in shared memory, then its columns, and writes a 16 x 16 block of each
// quadrant.  The LL quadrant goes to the carry buffer unless this is the last level;
// every other coefficient is final and goes through the epilogue.
template <class R>
__global__ void __launch_bounds__(256) k_dwt_level(const R* __restrict__ in, size_t in_stride, R* __restrict__ ll,
                                                   R* __restrict__ out, int m, int n, bool last, R scale,
                                                   const Filters<R> F, const EpiR<R> e) {
  __shared__ AnaSmem<R> sm;
  const int j = blockIdx.z;
  const R* src = in + in_stride * j;
  R* carry = ll + (size_t)n * n * j;
  R* dst = out + (size_t)n * n * F.aidx[j];
  EpiR<R> ej = e;  // the weights plane of this basis
  if (ej.w) ej.w += (size_t)n * n * F.aidx[j];
#define GBRI_DWT_CASE(LL) \
  case LL: dwt_block<LL, R>(sm, src, carry, dst, m, n, last, scale, F.h[j], F.g[j], ej); break;
  switch (F.len[j]) {
    GBRI_DWT_CASE(2) GBRI_DWT_CASE(4) GBRI_DWT_CASE(6) GBRI_DWT_CASE(8) GBRI_DWT_CASE(10) GBRI_DWT_CASE(12)
    GBRI_DWT_CASE(14) GBRI_DWT_CASE(16) GBRI_DWT_CASE(18) GBRI_DWT_CASE(20)
    default: break;
  }
#undef GBRI_DWT_CASE
}

// One synthesis level of one basis with an L-tap filter pair (the transpose of the
// analysis): reconstructs a 32 x 32 window of the m x m block from the
// 2 x (16 + L/2 - 1) coefficient rows and columns it touches (periodic).  Every
// coefficient of the window is loaded into registers before the first shared-memory store
// (one round of load latency per block).
template <int L, class R>
__device__ __forceinline__ void idwt_block(SynSmem<R>& sm, const R* __restrict__ coef, const R* __restrict__ llsrc,
                                           R* __restrict__ dst, int m, int n, const R* __restrict__ hf,
                                           const R* __restrict__ gf) {
  constexpr int KB = kSB / 2 + L / 2 - 1;
  const int half = m >> 1;
  const int r0 = blockIdx.y * kSB, c0 = blockIdx.x * kSB;
  const int kr_lo = r0 / 2 - L / 2 + 1, kc_lo = c0 / 2 - L / 2 + 1;
  R h[L], g[L];
#pragma unroll
  for (int i = 0; i < L; ++i) {
    h[i] = hf[i];
    g[i] = gf[i];
  }
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // coefficient indexes stay within [-half, 2 half) once half >= 16 and half >= L: one
  // conditional wrap instead of an integer modulo per element
  const bool small = half < 16 || half < L;
  const bool interior = kr_lo >= 0 && kr_lo + KB <= half && kc_lo >= 0 && kc_lo + KB <= half;
  constexpr int NW = 4 * KB * KB;         // the window: [a | d rows] x [a | d cols]
  constexpr int NL = (NW + 255) / 256;    // elements per thread
  // interior blocks of an FP32 level read each window row's two column segments (KB
  // coefficients of the a and of the d half) as float4 from the 16-byte boundary at or below
  // the segment's start, when the last float4 ends inside the row: a quarter of the load and
  // index instructions
  constexpr int S4 = (KB + 6) / 4;             // float4 per segment (start up to 3 below)
  constexpr int NV4 = 2 * KB * 2 * S4;
  constexpr int NL4 = (NV4 + 255) / 256;
  const int dlt = kc_lo & 3;
  bool vec = false;
  if constexpr (sizeof(R) == 4)
    vec = interior && (n & 3) == 0 && (half & 3) == 0 && kc_lo - dlt + 4 * S4 <= half &&
          ((reinterpret_cast<uintptr_t>(coef) | reinterpret_cast<uintptr_t>(llsrc)) & 15) == 0;
  float4 v4[NL4];
  if (vec) {
#pragma unroll
    for (int k = 0; k < NL4; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < NV4) {
        const int sr = idx / (2 * S4), rem = idx - sr * (2 * S4);
        const int pc = rem >= S4 ? 1 : 0, c4 = rem - pc * S4;
        const int pr = sr >= KB ? 1 : 0;
        const int kr = kr_lo + sr - pr * KB;
        const R* srcp = (pr == 0 && pc == 0) ? llsrc : coef;
        v4[k] = *reinterpret_cast<const float4*>(srcp + (size_t)(pr * half + kr) * n + pc * half + kc_lo - dlt +
                                                 4 * c4);
      }
    }
  }
  R v[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int idx = threadIdx.x + 256 * k;
    if (!vec && idx < NW) {
      const int sr = idx / (2 * KB), sc = idx - sr * (2 * KB);
      const int pr = sr >= KB ? 1 : 0, pc = sc >= KB ? 1 : 0;
      int kr = kr_lo + sr - pr * KB, kc = kc_lo + sc - pc * KB;
      if (!interior) {
        if (small) {
          kr %= half;
          kc %= half;
        }
        if (kr < 0) kr += half;
        if (kr >= half) kr -= half;
        if (kc < 0) kc += half;
        if (kc >= half) kc -= half;
      }
      const R* srcp = (pr == 0 && pc == 0) ? llsrc : coef;
      v[k] = srcp[(size_t)(pr * half + kr) * n + pc * half + kc];
    }
  }
  if (vec) {
#pragma unroll
    for (int k = 0; k < NL4; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < NV4) {
        const int sr = idx / (2 * S4), rem = idx - sr * (2 * S4);
        const int pc = rem >= S4 ? 1 : 0, c4 = rem - pc * S4;
        const float e4[4] = {v4[k].x, v4[k].y, v4[k].z, v4[k].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int e = 4 * c4 + j - dlt;
          if (e >= 0 && e < KB) sm.tc[sr][pc * KB + e] = (R)e4[j];
        }
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < NL; ++k) {
      const int idx = threadIdx.x + 256 * k;
      if (idx < NW) {
        const int sr = idx / (2 * KB);
        sm.tc[sr][idx - sr * (2 * KB)] = v[k];
      }
    }
  }
  __syncthreads();
  // column synthesis, register-blocked: an item is one coefficient column sc and two output
  // row pairs (2 pr, 2 pr + 1), pr = 2 pg, 2 pg + 1, which read the L/2 + 1 coefficient rows
  // kq = pr .. pr + L/2 of the a and d halves they share once
  for (int sc = tx; sc < 2 * KB; sc += 32) {
    const int pr0 = 2 * ty;  // pg = ty: 8 warps cover the kSB / 4 = 8 pair groups
    R a[L / 2 + 1], d[L / 2 + 1];
#pragma unroll
    for (int j = 0; j <= L / 2; ++j) {
      a[j] = sm.tc[pr0 + j][sc];
      d[j] = sm.tc[KB + pr0 + j][sc];
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      R ve = 0, vo = 0;
#pragma unroll
      for (int q = 0; q < L / 2; ++q) {
        const int j = p + L / 2 - 1 - q;
        ve = fma_r(h[2 * q], a[j], fma_r(g[2 * q], d[j], ve));
        vo = fma_r(h[2 * q + 1], a[j], fma_r(g[2 * q + 1], d[j], vo));
      }
      sm.tm[2 * (pr0 + p)][sc] = ve;
      sm.tm[2 * (pr0 + p) + 1][sc] = vo;
    }
  }
  __syncthreads();
  // row synthesis, register-blocked: an item is one output row r and two output column
  // pairs (four consecutive samples), reading the L/2 + 1 a and d values they share once
  {
    const int r = threadIdx.x >> 3, pc0 = 2 * (threadIdx.x & 7);  // kSB * kSB / 4 = 256 items
    R a[L / 2 + 1], d[L / 2 + 1];
#pragma unroll
    for (int j = 0; j <= L / 2; ++j) {
      a[j] = sm.tm[r][pc0 + j];
      d[j] = sm.tm[r][KB + pc0 + j];
    }
    R o[4];
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      R ve = 0, vo = 0;
#pragma unroll
      for (int q = 0; q < L / 2; ++q) {
        const int j = p + L / 2 - 1 - q;
        ve = fma_r(h[2 * q], a[j], fma_r(g[2 * q], d[j], ve));
        vo = fma_r(h[2 * q + 1], a[j], fma_r(g[2 * q + 1], d[j], vo));
      }
      o[2 * p] = ve;
      o[2 * p + 1] = vo;
    }
    const int Rr = r0 + r, Cc = c0 + 2 * pc0;
    if (Rr < m) {
      R* q = dst + (size_t)Rr * n + Cc;
      bool v4 = false;
      if constexpr (sizeof(R) == 4) v4 = Cc + 3 < m && (n & 3) == 0;  // Cc is a multiple of 4
      if (v4) {  // one 16-byte store
        *reinterpret_cast<float4*>(q) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (Cc + i < m) q[i] = o[i];
      }
    }
  }
}

// One synthesis level at block size m for basis blockIdx.z: writes the reconstruction
// of the m x m block into rec_out[basis].  The LL quadrant is read from rec_in (the
// coarser level's reconstruction, from_rec) or from the coefficients.
template <class R>
__global__ void __launch_bounds__(256) k_idwt_level(const R* __restrict__ alpha, const R* __restrict__ rec_in,
                                                    bool from_rec, R* __restrict__ rec_out, int m, int n,
                                                    const Filters<R> F) {
  __shared__ SynSmem<R> sm;
  const int j = blockIdx.z;
  const R* coef = alpha + (size_t)n * n * F.aidx[j];
  const R* llsrc = from_rec ? rec_in + (size_t)n * n * j : coef;
  R* dst = rec_out + (size_t)n * n * j;
#define GBRI_IDWT_CASE(LL) \
  case LL: idwt_block<LL, R>(sm, coef, llsrc, dst, m, n, F.h[j], F.g[j]); break;
  switch (F.len[j]) {
    GBRI_IDWT_CASE(2) GBRI_IDWT_CASE(4) GBRI_IDWT_CASE(6) GBRI_IDWT_CASE(8) GBRI_IDWT_CASE(10) GBRI_IDWT_CASE(12)
    GBRI_IDWT_CASE(14) GBRI_IDWT_CASE(16) GBRI_IDWT_CASE(18) GBRI_IDWT_CASE(20)
    default: break;
  }
#undef GBRI_IDWT_CASE
}

// x[q] = scale * (sum_j rec[j][q] + dirac[q]), summed in that order; V = 4 consecutive
// samples per thread (float4) on the FP32 path when N % 4 == 0 and the pointers are 16-byte
// aligned, else V = 1.
template <class R, int V>
__global__ void k_psi_sum(const R* __restrict__ rec, int nb, const R* __restrict__ dirac, R* __restrict__ x,
                          int64_t N, R scale) {
  static_assert(V == 1 || (V == 4 && sizeof(R) == 4), "vector path is FP32 only");
  const int64_t G = N / V;
  for (int64_t gq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gq < G; gq += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (V == 4) {
      float4 v = dirac ? *reinterpret_cast<const float4*>(dirac + 4 * gq) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
      for (int j = 0; j < nb; ++j) {
        const float4 r = *reinterpret_cast<const float4*>(rec + (size_t)N * j + 4 * gq);
        v.x += r.x;
        v.y += r.y;
        v.z += r.z;
        v.w += r.w;
      }
      *reinterpret_cast<float4*>(x + 4 * gq) = make_float4(scale * v.x, scale * v.y, scale * v.z, scale * v.w);
    } else {
      R v = dirac ? dirac[gq] : (R)0;
#pragma unroll 8
      for (int j = 0; j < nb; ++j) v += rec[(size_t)N * j + gq];
      x[gq] = scale * v;
    }
  }
}

// Dirac basis of the analysis: out[q] = epi(scale * x[q]); V as in k_psi_sum.
template <class R, int V>
__global__ void k_dirac(const R* __restrict__ x, R* __restrict__ out, int64_t N, R scale, const EpiR<R> e) {
  static_assert(V == 1 || (V == 4 && sizeof(R) == 4), "vector path is FP32 only");
  const int64_t G = N / V;
  for (int64_t gq = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; gq < G; gq += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (V == 4) {
      const float4 xv = *reinterpret_cast<const float4*>(x + 4 * gq);
      float4 pv = make_float4(0.f, 0.f, 0.f, 0.f), wv = pv;
      if (e.mode != 0) pv = *reinterpret_cast<const float4*>(out + 4 * gq);
      if (e.w) wv = *reinterpret_cast<const float4*>(e.w + 4 * gq);
      *reinterpret_cast<float4*>(out + 4 * gq) =
          make_float4(epi_value(scale * xv.x, e, pv.x, wv.x), epi_value(scale * xv.y, e, pv.y, wv.y),
                      epi_value(scale * xv.z, e, pv.z, wv.z), epi_value(scale * xv.w, e, pv.w, wv.w));
    } else {
      emit(out, (size_t)gq, scale * x[gq], e);
    }
  }
}

// x[q] = scale * dirac[q] (a dictionary that holds only the Dirac basis)
template <class R>
__global__ void k_scale_copy(const R* __restrict__ a, R* __restrict__ x, int64_t N, R scale) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x)
    x[q] = scale * a[q];
}

// float4 access: FP32, a length that is a multiple of 4 and 16-byte aligned pointers
// (null pointers are not accessed)
template <class R>
bool vec4_ok(int64_t N, const void* a, const void* b, const void* c) {
  auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return sizeof(R) == 4 && N % 4 == 0 && al(a) && al(b) && al(c);
}

int blocks_for(int64_t work) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(work, 256), (int64_t)num_sms() * 8));
}

template <class R> const Filters<R>& filters(const gbri_wavelet* w);
template <> const Filters<float>& filters<float>(const gbri_wavelet* w) { return w->F; }
template <> const Filters<double>& filters<double>(const gbri_wavelet* w) { return w->Fd; }

}  // namespace

template <class R>
int32_t psi_adjoint_apply(gbri_wavelet* w, const R* x, R* out, DualEpi epi, cudaStream_t s) {
  const int n = w->n;
  const int64_t N = (int64_t)n * n;
  const R scale = (R)w->scale;
  if (w->dirac_idx >= 0) {
    launch_begin(GBRI_K_PSI_ADJ, s);
    EpiR<R> ed(epi);
    if (ed.w) ed.w += (size_t)N * w->dirac_idx;
    R* od = out + (size_t)N * w->dirac_idx;
    if (vec4_ok<R>(N, x, od, ed.w))
      k_dirac<R, (sizeof(R) == 4 ? 4 : 1)><<<blocks_for(N / 4), 256, 0, s>>>(x, od, N, scale, ed);
    else
      k_dirac<R, 1><<<blocks_for(N), 256, 0, s>>>(x, od, N, scale, ed);
    GBRI_TRY(launch_end(GBRI_K_PSI_ADJ, s));
  }
  if (w->nb == 0) return GBRI_OK;
  // the LL carry ping-pongs between the two buffers: a level must not overwrite the
  // window another block of the same level still has to read
  R* carry[2] = {static_cast<R*>(w->ll), static_cast<R*>(w->tmp)};
  for (int lev = 0; lev < w->levels; ++lev) {
    const int m = n >> lev;
    const int bq = (int)ceil_div(m / 2, kAB);
    const R* in = (lev == 0) ? x : carry[(lev - 1) & 1];
    const size_t in_stride = (lev == 0) ? 0 : (size_t)N;
    launch_begin(GBRI_K_PSI_ADJ, s);
    k_dwt_level<R><<<dim3(bq, bq, w->nb), 256, 0, s>>>(in, in_stride, carry[lev & 1], out, m, n,
                                                       lev == w->levels - 1, scale, filters<R>(w), EpiR<R>(epi));
    GBRI_TRY(launch_end(GBRI_K_PSI_ADJ, s));
  }
  return GBRI_OK;
}

template <class R>
int32_t psi_apply(gbri_wavelet* w, const R* alpha, R* x, cudaStream_t s) {
  const int n = w->n;
  const int64_t N = (int64_t)n * n;
  const R scale = (R)w->scale;
  const R* dirac = w->dirac_idx >= 0 ? alpha + (size_t)N * w->dirac_idx : nullptr;
  if (w->nb == 0) {
    launch_begin(GBRI_K_PSI, s);
    k_scale_copy<R><<<blocks_for(N), 256, 0, s>>>(dirac, x, N, scale);
    return launch_end(GBRI_K_PSI, s);
  }
  // ping-pong reconstruction buffers: level l reads the coarser level's output
  R* bufs[2] = {static_cast<R*>(w->ll), static_cast<R*>(w->tmp)};
  int cur = 0;
  for (int lev = w->levels - 1; lev >= 0; --lev) {
    const int m = n >> lev;
    const int bs = (int)ceil_div(m, kSB);
    launch_begin(GBRI_K_PSI, s);
    k_idwt_level<R><<<dim3(bs, bs, w->nb), 256, 0, s>>>(alpha, bufs[cur ^ 1], lev != w->levels - 1, bufs[cur], m, n,
                                                        filters<R>(w));
    GBRI_TRY(launch_end(GBRI_K_PSI, s));
    cur ^= 1;
  }
  launch_begin(GBRI_K_PSI, s);
  if (vec4_ok<R>(N, bufs[cur ^ 1], x, dirac))
    k_psi_sum<R, (sizeof(R) == 4 ? 4 : 1)><<<blocks_for(N / 4), 256, 0, s>>>(bufs[cur ^ 1], w->nb, dirac, x, N, scale);
  else
    k_psi_sum<R, 1><<<blocks_for(N), 256, 0, s>>>(bufs[cur ^ 1], w->nb, dirac, x, N, scale);
  return launch_end(GBRI_K_PSI, s);
}

template int32_t psi_adjoint_apply<float>(gbri_wavelet*, const float*, float*, DualEpi, cudaStream_t);
template int32_t psi_adjoint_apply<double>(gbri_wavelet*, const double*, double*, DualEpi, cudaStream_t);
template int32_t psi_apply<float>(gbri_wavelet*, const float*, float*, cudaStream_t);
template int32_t psi_apply<double>(gbri_wavelet*, const double*, double*, cudaStream_t);

}  // namespace gbri

using namespace gbri;

extern "C" {

int32_t gbri_wavelet_create(gbri_wavelet** out, int32_t n_side, int32_t levels, const int32_t* db_orders,
                            int32_t n_w, int32_t precision) {
  GBRI_CHECK(out && db_orders, GBRI_EINVAL, "null argument");
  *out = nullptr;
  GBRI_CHECK(precision == GBRI_F32 || precision == GBRI_F64, GBRI_EINVAL, "precision must be GBRI_F32 or GBRI_F64");
  GBRI_CHECK(n_w >= 1 && n_w <= kMaxBases, GBRI_EINVAL, "n_w must be in [1, 16]");
  GBRI_CHECK(levels >= 1 && levels <= 12, GBRI_EINVAL, "levels must be in [1, 12]");
  GBRI_CHECK(n_side >= 4 && n_side % (1 << levels) == 0 && (n_side >> levels) >= 2, GBRI_EINVAL,
             "n_side must be divisible by 2^levels with n_side >> levels >= 2");
  gbri_wavelet* w = new (std::nothrow) gbri_wavelet();
  GBRI_CHECK(w, GBRI_ENOMEM, "host allocation");
  w->n = n_side;
  w->levels = levels;
  w->nw = n_w;
  w->prec = precision;
  w->scale = 1.0 / std::sqrt((double)n_w);
  for (int b = 0; b < n_w; ++b) {
    const int N = db_orders[b];
    if (N < 0 || N > kMaxTaps / 2 || (N == 0 && w->dirac_idx >= 0)) {
      delete w;
      return set_error(GBRI_EINVAL, "db order must be 0 (once) or 1..10");
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
      const double hv = i < L ? h[i] : 0.0;
      const double gv = i < L ? (i % 2 ? -1.0 : 1.0) * h[L - 1 - i] : 0.0;
      w->F.h[j][i] = (float)hv;
      w->F.g[j][i] = (float)gv;
      w->Fd.h[j][i] = hv;
      w->Fd.g[j][i] = gv;
    }
    w->F.len[j] = w->Fd.len[j] = L;
    w->F.aidx[j] = w->Fd.aidx[j] = b;
  }
  const size_t bytes = real_bytes(precision) * (size_t)std::max(1, w->nb) * n_side * n_side;
  if (cudaMalloc(&w->tmp, bytes) != cudaSuccess || cudaMalloc(&w->ll, bytes) != cudaSuccess) {
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

int32_t gbri_psi(gbri_wavelet* w, const void* d_alpha, void* d_x, void* stream) {
  GBRI_CHECK(w && d_alpha && d_x, GBRI_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  if (w->prec == GBRI_F64) return psi_apply(w, static_cast<const double*>(d_alpha), static_cast<double*>(d_x), s);
  return psi_apply(w, static_cast<const float*>(d_alpha), static_cast<float*>(d_x), s);
}

int32_t gbri_psi_adjoint(gbri_wavelet* w, const void* d_x, void* d_alpha, void* stream) {
  GBRI_CHECK(w && d_alpha && d_x, GBRI_EINVAL, "null argument");
  DualEpi e{0, 0.0, 0.0, 0.0, 0.0};
  cudaStream_t s = (cudaStream_t)stream;
  if (w->prec == GBRI_F64)
    return psi_adjoint_apply(w, static_cast<const double*>(d_x), static_cast<double*>(d_alpha), e, s);
  return psi_adjoint_apply(w, static_cast<const float*>(d_x), static_cast<float*>(d_alpha), e, s);
}

}  // extern "C"
