// SARA wavelet dictionary (Sec. 3.1, Sec. 6.4, Sec. 7.5): Dirac basis plus 2-D
// separable periodic Daubechies transforms, batched over the bases in each launch.
#pragma once

#include <vector>

#include "common.cuh"

namespace gbri {

constexpr int kMaxTaps = 20;   // db10
constexpr int kMaxBases = 16;

// Filter bank of the non-Dirac bases in real type R, passed to the kernels by value.
template <class R>
struct Filters {
  R h[kMaxBases][kMaxTaps];
  R g[kMaxBases][kMaxTaps];
  int len[kMaxBases];
  int aidx[kMaxBases];  // position of the basis in the coefficient stack
};

// How the analysis writes a final coefficient v (already scaled by 1/sqrt(n_w)):
//   mode 0: out[q] = v
//   mode 1: out[q] = clip(ca * out[q] + cb * v, [-lim w_q, lim w_q]) * ce   (dual updates of
//           PD / DualFB; w = per-coefficient l1 weights of the stack layout, real type of the
//           kernels, or null for w = 1)
// (constants in FP64; rounded once to the kernels' real type)
struct DualEpi {
  int mode;
  double ca, cb, lim, ce;
  const void* w = nullptr;
};

// DualEpi rounded to the kernels' real type once, on the host (a per-thread conversion
// from double would run on the FP64 pipe).
template <class R>
struct EpiR {
  int mode;
  R ca, cb, lim, ce;
  const R* w;  // weights of the plane written (offset like the output), or null
  __host__ __device__ explicit EpiR(const DualEpi& e)
      : mode(e.mode), ca((R)e.ca), cb((R)e.cb), lim((R)e.lim), ce((R)e.ce), w(static_cast<const R*>(e.w)) {}
};

// Daubechies low-pass filter dbN (2N taps, minimum phase, sum = sqrt 2) by
// spectral factorisation of the Daubechies polynomial (host, long double).
std::vector<double> daubechies_lowpass(int N);

}  // namespace gbri

struct gbri_wavelet {
  int n = 0, levels = 0, nw = 0, nb = 0;  // nb = number of non-Dirac bases
  int dirac_idx = -1;
  int prec = 0;                            // GBRI_F32 or GBRI_F64: element type of every buffer
  double scale = 1.0;                      // 1 / sqrt(n_w)
  std::vector<int> orders;
  gbri::Filters<float> F;                  // FP32 path
  gbri::Filters<double> Fd;                // FP64 path
  void* tmp = nullptr;  // R [nb][n][n]
  void* ll = nullptr;   // R [nb][n][n] LL carry (analysis) / reconstruction (synthesis)
};

namespace gbri {
// Psi^dagger x with the epilogue applied to every final coefficient of the stack `out` [n_w][n][n].
template <class R>
int32_t psi_adjoint_apply(gbri_wavelet* w, const R* x, R* out, DualEpi epi, cudaStream_t s);
// x = Psi alpha (overwrites x).
template <class R>
int32_t psi_apply(gbri_wavelet* w, const R* alpha, R* x, cudaStream_t s);
}  // namespace gbri
