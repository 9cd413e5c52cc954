// Solvers of the constrained analysis problem (Sec. 3.1, Sec. 5):
//     min ||Psi^dagger x||_1  s.t.  ||y - Phi x||_2 <= eps,  x >= 0.
//
// Primal-dual (Appendix A.4, Algorithm 7) with L = [Psi^dagger; Phi],
// f = gamma ||.||_1 (+) iota_B(y, eps), g = iota_{R+}.  With the Moreau
// decomposition the dual step is z1 <- clip(z1 + sigma1 Psi^dagger xhat, gamma) and
// z2 <- t - sigma2 P_B(t / sigma2), t = z2 + sigma2 Phi xhat.  Writing
// u = t - sigma2 y, the projection gives z2 = (1 - rho) u with
// rho = min(1, eps / ||u / sigma2||), so the device keeps u and the scalar
// c = 1 - rho instead of z2:
//   degrid epilogue:  u <- c u + sigma2 (Phi xhat - y), partial ||u||^2  (FP64 block sums);
//                     its last block: c <- 1 - min(1, eps sigma2 / ||u||)
//   gridding source:  u (Phi^dagger is linear; c scales the image)
//   image epilogue:   x+ = max(x - tau (Psi z1 + c Re Phi^dagger u), 0), xhat = x+ + theta (x+ - x);
//                     its last block: ||x+ - x|| / ||x+||
// The wavelet half (z1 and Psi z1) runs on a second stream beside the measurement half.
//
// Dual Forward-Backward ADMM (Sec. 5, Algorithm 1), with w = v + s - y, v = Phi x:
//   r = y + rho_b w, rho_b = min(1, eps / ||w||)  (projection onto the ball around y)
//   s+ = s + varrho (v - r) = s + varrho ((1 - rho_b) w - s)
//   xt = x - rho Re Phi^dagger (v - r + s+),  v - r + s+ = (1 - rho_b) w - s + s+
//   DualFB(xt): zbar = P_C(xt); repeat { d = clip(eta d + Psi^dagger zbar, gamma) / eta;
//               zbar = P_C(xt - Psi d) }; x = zbar.
//
// FISTA (Algorithm 4) on the unconstrained analysis problem (Sec. 3.1):
//   r = Phi xhat - y;  z = xhat - lambda Re Phi^dagger r;  x+ = DualFB(z, lambda gamma);
//   theta+ = (1 + sqrt(1 + 4 theta^2)) / 2;  xhat = x+ + (theta - 1) / theta+ (x+ - x).
// theta lives on the device (graph replays need no host work).
// All global norms are FP64 (FP32 path: per-thread compensated FP32 partials, FP64
// block sums).  Every kernel is templated on the real type R of the plan: float for
// the mixed-precision path, double for the plain FP64 path.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <new>
#include <vector>

#include "nufft.cuh"
#include "prox.cuh"
#include "solver.cuh"
#include "wavelet.cuh"

namespace gbri {
namespace {

enum {
  SC_C = 0, SC_DIST = 1, SC_REL = 2, SC_XN = 3, SC_RES = 4, SC_MAX = 5, SC_THETA = 6, SC_ALPHA = 7, SC_ONE = 8,
  SC_N = 16
};

// c = 1 - min(1, eps / (||u|| / sigma2))  (PD)   or   rho_b = min(1, eps / ||w||)  (ADMM, sigma2 = 1, want_rho)
__global__ void k_ball_scalar(const double* __restrict__ partials, int n, double eps, double sigma2, bool want_rho,
                              double* __restrict__ sc) {
  __shared__ double sh[40];
  const double dist = sqrt(reduce_partials(partials, n, sh)) / sigma2;
  if (threadIdx.x == 0) {
    const double rho = dist > eps ? eps / dist : 1.0;
    sc[SC_C] = want_rho ? rho : 1.0 - rho;
    sc[SC_DIST] = dist;
  }
}

// Local balls: block j of the grid reduces ball j's partials in a fixed order;
// rho_j = min(1, eps_j / dist_j), dist_j = sqrt(sum) / sigma2; out[j] = rho_j or 1 - rho_j.
__global__ void k_ball_scalar_local(const double* __restrict__ partials, int n, const double* __restrict__ eps,
                                    double sigma2, bool want_rho, double* __restrict__ out) {
  __shared__ double sh[40];
  const int j = blockIdx.x;
  const double dist = sqrt(reduce_partials(partials + (size_t)j * n, n, sh)) / sigma2;
  if (threadIdx.x == 0) {
    const double rho = dist > eps[j] ? eps[j] / dist : 1.0;
    out[j] = want_rho ? rho : 1.0 - rho;
  }
}

// PD primal update fused with S^T Z^T of img = Re(F^H grid) of the gridded dual (real
// [K][K], from the complex-to-real inverse; scaled by *cp, the l2-ball scalar c; 1 with local
// balls, whose scalars the gridding source applied) and the
// relative-change reduction: each block writes its FP64 sums of (x+ - x)^2 and x+^2; the
// last block to finish (device-wide counter, reset by that block) reduces them in block
// order into sc[SC_REL] = ||x+ - x|| / ||x+|| and sc[SC_XN] = ||x+||.
// A thread takes V consecutive pixels of one row: V = 4 on the FP32 path when n % 8 == 0
// (a group never straddles the periodic wrap at column n/2, and every vector access is
// 16-byte aligned), else V = 1.
template <class R, int V>
__global__ void k_pd_update(const R* __restrict__ img, const R* __restrict__ corr, const R* __restrict__ psiz,
                            R* __restrict__ x, R* __restrict__ xhat, int n, int K, R tau, R theta,
                            const double* __restrict__ cp, double* __restrict__ sc, double* __restrict__ partials,
                            unsigned int* __restrict__ done) {
  static_assert(V == 1 || (V == 4 && sizeof(R) == 4), "vector path is FP32 only");
  __shared__ double sh[40];
  __shared__ bool last;
  const R c = (R)*cp;
  acc_t<R> dd, xx;
  const int groups = n * n / V;
  const int stride = gridDim.x * blockDim.x;
  // U grid-stride steps per pass with all their loads issued first (one round of load
  // latency per pass); the steps are applied in grid-stride order, so the per-thread sums
  // take their terms in the same order as a one-step loop
  constexpr int U = 4;
  for (int g0 = blockIdx.x * blockDim.x + threadIdx.x; g0 < groups; g0 += U * stride) {
    R gr[U][V], cr[U][V], ps[U][V], xo[U][V], cq[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int gi = g0 + u * stride;
      if (gi >= groups) break;
      const int i = gi * V;
      const int q = i / n, p = i - q * n;
      int r = q - n / 2; if (r < 0) r += K;
      int cc = p - n / 2; if (cc < 0) cc += K;
      if constexpr (V == 4) {
        const float4 g4 = *reinterpret_cast<const float4*>(img + (size_t)r * K + cc);
        gr[u][0] = g4.x; gr[u][1] = g4.y; gr[u][2] = g4.z; gr[u][3] = g4.w;
        const float4 c4 = *reinterpret_cast<const float4*>(corr + p);
        cr[u][0] = c4.x; cr[u][1] = c4.y; cr[u][2] = c4.z; cr[u][3] = c4.w;
        const float4 p4 = *reinterpret_cast<const float4*>(psiz + i);
        ps[u][0] = p4.x; ps[u][1] = p4.y; ps[u][2] = p4.z; ps[u][3] = p4.w;
        const float4 x4 = *reinterpret_cast<const float4*>(x + i);
        xo[u][0] = x4.x; xo[u][1] = x4.y; xo[u][2] = x4.z; xo[u][3] = x4.w;
      } else {
        gr[u][0] = img[(size_t)r * K + cc];
        cr[u][0] = corr[p];
        ps[u][0] = psiz[i];
        xo[u][0] = x[i];
      }
      cq[u] = corr[q];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int gi = g0 + u * stride;
      if (gi >= groups) break;
      const int i = gi * V;
      R xn[V], xh[V];
#pragma unroll
      for (int j = 0; j < V; ++j) {
        const R phit = c * cr[u][j] * cq[u] * gr[u][j];
        xn[j] = max_r(xo[u][j] - tau * (ps[u][j] + phit), (R)0);
        xh[j] = fma_r(theta, xn[j] - xo[u][j], xn[j]);
        dd.add((xn[j] - xo[u][j]) * (xn[j] - xo[u][j]));
        xx.add(xn[j] * xn[j]);
      }
      if constexpr (V == 4) {
        *reinterpret_cast<float4*>(xhat + i) = make_float4(xh[0], xh[1], xh[2], xh[3]);
        *reinterpret_cast<float4*>(x + i) = make_float4(xn[0], xn[1], xn[2], xn[3]);
      } else {
        xhat[i] = xh[0];
        x[i] = xn[0];
      }
    }
  }
  const double a = block_sum(dd.value(), sh);
  const double b = block_sum(xx.value(), sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
    __threadfence();  // the partials are visible device-wide before the count says so
    last = atomicAdd(done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    sa += __ldcg(partials + 2 * i);
    sb += __ldcg(partials + 2 * i + 1);
  }
  sa = block_sum(sa, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    const double dn = sqrt(sa), xn = sqrt(sb);
    sc[SC_REL] = xn > 0 ? dn / xn : (dn == 0 ? 0.0 : INFINITY);
    sc[SC_XN] = xn;
    *done = 0u;
  }
}

__global__ void k_rel_change(const double* __restrict__ partials, int n, double* __restrict__ sc) {
  __shared__ double sh[40];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a += partials[2 * i];
    b += partials[2 * i + 1];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    const double dn = sqrt(a), xn = sqrt(b);
    sc[SC_REL] = xn > 0 ? dn / xn : (dn == 0 ? 0.0 : INFINITY);
    sc[SC_XN] = xn;
  }
}

// ADMM: xt = x - rho * S^T Z^T img, img = Re(F^H grid) (real [K][K]); zbar = max(xt, 0)
template <class R>
__global__ void k_admm_xt(const R* __restrict__ img, const R* __restrict__ corr, const R* __restrict__ x,
                          R* __restrict__ xt, R* __restrict__ zbar, int n, int K, R rho) {
  const int total = n * n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int q = i / n, p = i - q * n;
    int r = q - n / 2; if (r < 0) r += K;
    int cc = p - n / 2; if (cc < 0) cc += K;
    const R v = x[i] - rho * corr[p] * corr[q] * img[(size_t)r * K + cc];
    xt[i] = v;
    zbar[i] = max_r(v, (R)0);
  }
}

// zbar = max(xt - Psi d, 0); on the last inner iteration also x = zbar with change partials.
template <class R>
__global__ void k_admm_zbar(const R* __restrict__ xt, const R* __restrict__ psid, R* __restrict__ zbar,
                            R* __restrict__ x, int64_t N, bool last, double* __restrict__ partials) {
  __shared__ double sh[40];
  acc_t<R> dd, xx;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const R z = max_r(xt[i] - psid[i], (R)0);
    zbar[i] = z;
    if (last) {
      const R xo = x[i];
      dd.add((z - xo) * (z - xo));
      xx.add(z * z);
      x[i] = z;
    }
  }
  if (!last) return;
  const double a = block_sum(dd.value(), sh);
  const double b = block_sum(xx.value(), sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

// FISTA momentum: alpha = (theta - 1) / theta+, theta <- theta+ (theta starts at 1)
__global__ void k_fista_theta(double* __restrict__ sc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    const double t = sc[SC_THETA];
    const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
    sc[SC_ALPHA] = (t - 1.0) / tn;
    sc[SC_THETA] = tn;
  }
}

// Last DualFB step of FISTA: x+ = max(z - Psi d, 0); xhat = x+ + alpha (x+ - x); x = x+; change partials.
template <class R>
__global__ void k_fista_last(const R* __restrict__ z, const R* __restrict__ psid, R* __restrict__ xhat,
                             R* __restrict__ x, int64_t N, const double* __restrict__ sc,
                             double* __restrict__ partials) {
  __shared__ double sh[40];
  const R alpha = (R)sc[SC_ALPHA];
  acc_t<R> dd, xx;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const R xn = max_r(z[i] - psid[i], (R)0);
    const R xo = x[i];
    xhat[i] = fma_r(alpha, xn - xo, xn);
    x[i] = xn;
    dd.add((xn - xo) * (xn - xo));
    xx.add(xn * xn);
  }
  const double a = block_sum(dd.value(), sh);
  const double b = block_sum(xx.value(), sh);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
  }
}

template <class R>
__global__ void k_absmax_partials(const R* __restrict__ a, int64_t n, double* __restrict__ partials) {
  __shared__ R sh[32];
  R m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max_r(m, abs_r(a[i]));
  for (int o = 16; o > 0; o >>= 1) m = max_r(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    R r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max_r(r, sh[w]);
    partials[blockIdx.x] = r;
  }
}

// SARA weights in place: w = delta / (delta + |w|) (w holds Psi^dagger x on entry)
template <class R>
__global__ void k_sara_weights(R* __restrict__ w, int64_t n, R delta) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = delta / (delta + abs_r(w[i]));
}

__global__ void k_max_finish(const double* __restrict__ partials, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, partials[i]);
    *out = m;
  }
}

template <class R>
__global__ void k_residual_partials(const cplx<R>* __restrict__ a, const cplx<R>* __restrict__ b, int64_t M,
                                    double* __restrict__ partials) {
  __shared__ double sh[40];
  acc_t<R> acc;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    const R dr = a[i].x - b[i].x, di = a[i].y - b[i].y;
    acc.add(fma_r(dr, dr, di * di));
  }
  const double v = block_sum(acc.value(), sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

__global__ void k_sqrt_sum(const double* __restrict__ partials, int n, double* __restrict__ out) {
  __shared__ double sh[40];
  const double v = reduce_partials(partials, n, sh);
  if (threadIdx.x == 0) *out = sqrt(v);
}

int img_blocks(int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, 256), (int64_t)num_sms() * 8));
}

}  // namespace
}  // namespace gbri

using namespace gbri;

struct gbri_solver {
  gbri_plan* plan = nullptr;
  gbri_wavelet* wav = nullptr;
  gbri_solve_params p{};
  int prec = 0;  // the plan's precision: element type R of every vector below
  void *yp = nullptr, *u = nullptr, *w = nullptr;                            // complex [M], plan order
  void *x = nullptr, *xhat = nullptr, *psiz = nullptr, *z1 = nullptr, *xt = nullptr;  // real images / stacks
  void* zb = nullptr;  // FISTA: the DualFB iterate zbar (image)
  void* wts = nullptr;  // per-coefficient l1 weights [n_w][n][n] (after gbri_solver_reweight), or null
  int64_t graph_version = 0;
  // local l2 balls (n_balls >= 2): plan-position starts [nb + 1], radii [nb], per-ball
  // scalars [nb] (PD: c_j = 1 - rho_j; ADMM: rho_j), per-ball block partials [nb][degrid blocks]
  int nb = 0;
  int32_t* bstart = nullptr;
  double *beps = nullptr, *bsc = nullptr, *bpart = nullptr;
  double* partials = nullptr;
  double* sc = nullptr;
  int n_partials = 0;
  int iters = 0;
  double ms_total = 0.0;
  // primal-dual: the wavelet branch of an iteration runs on aux_stream, forked from and
  // joined back to the iteration's stream by the two events
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_zero = nullptr;
  unsigned int* done = nullptr;  // last-block counters: [0] degridding (ball scalar), [1] primal-dual update
  // one iteration captured as a CUDA graph and replayed (no host work per kernel)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int64_t launches_per_iter = 0;
  bool graph_failed = false;
};

namespace {

void free_solver(gbri_solver* s) {
  if (!s) return;
  if (s->graph_exec) cudaGraphExecDestroy(s->graph_exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->aux_stream) cudaStreamDestroy(s->aux_stream);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  if (s->ev_zero) cudaEventDestroy(s->ev_zero);
  cudaFree(s->yp); cudaFree(s->u); cudaFree(s->w);
  cudaFree(s->x); cudaFree(s->xhat); cudaFree(s->psiz); cudaFree(s->z1); cudaFree(s->xt); cudaFree(s->zb);
  cudaFree(s->wts);
  cudaFree(s->partials); cudaFree(s->sc); cudaFree(s->done);
  cudaFree(s->bstart); cudaFree(s->beps); cudaFree(s->bsc); cudaFree(s->bpart);
  delete s;
}

template <class R> R* vec(void* p) { return static_cast<R*>(p); }
template <class R> cplx<R>* cvec(void* p) { return static_cast<cplx<R>*>(p); }

// phase 0: the whole iteration; 1: up to the forward FFT (the stream then also waits for the
// zeroed grid); 2: from the inverse FFT on.  Phases 1 and 2 leave the fused degridding +
// gridding pass between them to the batch executor's pass over several problems.
template <class R>
int32_t pd_iteration(gbri_solver* S, cudaStream_t st, int phase = 0) {
  gbri_plan* P = S->plan;
  gbri_wavelet* W = S->wav;
  const auto& p = S->p;
  const int n = P->n_side;
  const int64_t N = (int64_t)n * n;
  // The wavelet branch (the dual update of z1, then Psi z1) and the measurement branch
  // (the dual update of u, then Phi^dagger u) of Algorithm 7 read only xhat and their own
  // dual variable until the primal update joins them: the wavelet branch runs on the
  // auxiliary stream, so its small coarse-level launches fill the SMs the visibility
  // kernels and the FFT leave idle.  (Captured, the fork and join are graph edges.)  With
  // kernel-by-kernel profiling on, both branches run on the one stream, so that the events
  // around each kernel time that kernel alone.
  const bool fork = !profiling_enabled();
  cudaStream_t sw = fork ? S->aux_stream : st;
  if (phase == 2) goto after_pass;
  if (fork) {
    GBRI_CHECK_CUDA(cudaEventRecord(S->ev_fork, st));
    GBRI_CHECK_CUDA(cudaStreamWaitEvent(sw, S->ev_fork, 0));
    // the gridding target is free once the previous update has read it: zero it here, off
    // the measurement branch (which reads the separate half spectrum until the gridding)
    GBRI_CHECK_CUDA(cudaMemsetAsync(P->grid, 0, grid_bytes(P), sw));
    GBRI_CHECK_CUDA(cudaEventRecord(S->ev_zero, sw));
  }
  // z1 <- clip(z1 + sigma1 Psi^dagger xhat, gamma)
  GBRI_TRY(psi_adjoint_apply<R>(W, vec<R>(S->xhat), vec<R>(S->z1), DualEpi{1, 1.0, p.sigma1, p.gamma, 1.0, S->wts},
                                sw));
  // Psi z1
  GBRI_TRY(psi_apply<R>(W, vec<R>(S->z1), vec<R>(S->psiz), sw));
  if (fork) GBRI_CHECK_CUDA(cudaEventRecord(S->ev_join, sw));
  // u <- c u + sigma2 (Phi xhat - y), ||u||^2
  GBRI_TRY(launch_pad<R>(P, vec<R>(S->xhat), nullptr, st));
  GBRI_TRY(fft_forward(P, st));
  if (phase == 1) {
    if (fork) GBRI_CHECK_CUDA(cudaStreamWaitEvent(st, S->ev_zero, 0));
    return GBRI_OK;
  }
  if (S->nb == 0) {
    // (the degridding's last block also stores the ball scalar c of this iteration)
    EpiPD1<R> e1{cvec<R>(S->u), cvec<R>(S->yp), S->sc + SC_C, S->partials, (R)p.sigma2, acc_t<R>{}, (R)0,
                 S->sc + SC_C, S->sc + SC_DIST, S->done, p.eps, p.sigma2};
    bool fused = false;
    if constexpr (sizeof(R) == 4) {
      if (fused_pd_applies(P)) {  // degridding + gridding of the updated u in one pass
        if (fork) GBRI_CHECK_CUDA(cudaStreamWaitEvent(st, S->ev_zero, 0));
        GBRI_TRY(launch_degrid_grid(P, e1, st, fork));
        fused = true;
      }
    }
    if (!fused) {
      GBRI_TRY(launch_degrid(P, e1, st));
      // Phi^dagger u (scaled by c in the update)
      if (fork) GBRI_CHECK_CUDA(cudaStreamWaitEvent(st, S->ev_zero, 0));
      GBRI_TRY(launch_grid(P, SrcPlan<R>{cvec<R>(S->u)}, st, fork));
    }
  } else {  // local balls: c_j per ball, applied inside the gridding source
    EpiPD1L<R> e1{cvec<R>(S->u), cvec<R>(S->yp), S->bsc, (R)p.sigma2,
                  BallAcc<R>{S->bstart, S->nb, S->bpart, acc_t<R>{}, -1}, (R)0};
    GBRI_TRY(launch_degrid(P, e1, st));
    launch_begin(GBRI_K_OTHER, st);
    k_ball_scalar_local<<<S->nb, 256, 0, st>>>(S->bpart, P->degrid_blocks, S->beps, p.sigma2, false, S->bsc);
    GBRI_TRY(launch_end(GBRI_K_OTHER, st));
    if (fork) GBRI_CHECK_CUDA(cudaStreamWaitEvent(st, S->ev_zero, 0));
    GBRI_TRY(launch_grid(P, SrcScaledL<R>{cvec<R>(S->u), S->bsc, S->bstart, S->nb}, st, fork));
  }
after_pass:
  GBRI_TRY(fft_inverse_real(P, st));
  if (fork) GBRI_CHECK_CUDA(cudaStreamWaitEvent(st, S->ev_join, 0));
  const bool v4 = sizeof(R) == 4 && n % 8 == 0;
  // two blocks per SM looping over the image: fewer block reductions and counter atomics
  // than one group per thread (16.5 against 21.2 us per update at 1024^2)
  const int ib = std::min(std::min(img_blocks(v4 ? N / 4 : N), num_sms() * 2), S->n_partials / 2);
  const double* cp = S->nb ? S->sc + SC_ONE : S->sc + SC_C;
  launch_begin(GBRI_K_UPDATE, st);
  if (v4)
    k_pd_update<R, (sizeof(R) == 4 ? 4 : 1)><<<ib, 256, 0, st>>>(
        P->as<const R>(P->grid), P->as<const R>(P->corr), vec<R>(S->psiz), vec<R>(S->x), vec<R>(S->xhat), n,
        P->K, (R)p.tau, (R)p.theta, cp, S->sc, S->partials + S->n_partials, S->done + 1);
  else
    k_pd_update<R, 1><<<ib, 256, 0, st>>>(P->as<const R>(P->grid), P->as<const R>(P->corr), vec<R>(S->psiz),
                                          vec<R>(S->x), vec<R>(S->xhat), n, P->K, (R)p.tau, (R)p.theta, cp, S->sc,
                                          S->partials + S->n_partials, S->done + 1);
  return launch_end(GBRI_K_UPDATE, st);
}

template <class R>
int32_t admm_iteration(gbri_solver* S, cudaStream_t st) {
  gbri_plan* P = S->plan;
  gbri_wavelet* W = S->wav;
  const auto& p = S->p;
  const int n = P->n_side;
  const int64_t N = (int64_t)n * n;
  GBRI_TRY(launch_pad<R>(P, vec<R>(S->x), nullptr, st));
  GBRI_TRY(fft_forward(P, st));
  if (S->nb == 0) {
    EpiADMM1<R> e1{cvec<R>(S->w), cvec<R>(S->u), cvec<R>(S->yp), S->partials, acc_t<R>{}};
    GBRI_TRY(launch_degrid(P, e1, st));
    launch_begin(GBRI_K_OTHER, st);
    k_ball_scalar<<<1, 256, 0, st>>>(S->partials, P->degrid_blocks, p.eps, 1.0, true, S->sc);
    GBRI_TRY(launch_end(GBRI_K_OTHER, st));
    GBRI_TRY(launch_grid(P, SrcADMM2<R>{cvec<R>(S->w), cvec<R>(S->u), S->sc + SC_C, (R)p.varrho}, st));
  } else {  // local balls: rho_j per ball
    EpiADMM1L<R> e1{cvec<R>(S->w), cvec<R>(S->u), cvec<R>(S->yp), BallAcc<R>{S->bstart, S->nb, S->bpart, acc_t<R>{}, -1}};
    GBRI_TRY(launch_degrid(P, e1, st));
    launch_begin(GBRI_K_OTHER, st);
    k_ball_scalar_local<<<S->nb, 256, 0, st>>>(S->bpart, P->degrid_blocks, S->beps, 1.0, true, S->bsc);
    GBRI_TRY(launch_end(GBRI_K_OTHER, st));
    GBRI_TRY(launch_grid(P, SrcADMM2L<R>{cvec<R>(S->w), cvec<R>(S->u), S->bsc, S->bstart, S->nb, (R)p.varrho},
                         st));
  }
  GBRI_TRY(fft_inverse_real(P, st));
  const int ib = std::min(img_blocks(N), S->n_partials / 2);
  launch_begin(GBRI_K_UPDATE, st);
  k_admm_xt<R><<<ib, 256, 0, st>>>(P->as<const R>(P->grid), P->as<const R>(P->corr), vec<R>(S->x),
                                   vec<R>(S->xt), vec<R>(S->xhat) /* zbar */, n, P->K, (R)p.rho);
  GBRI_TRY(launch_end(GBRI_K_UPDATE, st));
  for (int k = 0; k < p.dualfb_iters; ++k) {
    GBRI_TRY(psi_adjoint_apply<R>(W, vec<R>(S->xhat), vec<R>(S->z1) /* d */,
                                  DualEpi{1, p.eta, 1.0, p.gamma, 1.0 / p.eta, S->wts}, st));
    GBRI_TRY(psi_apply<R>(W, vec<R>(S->z1), vec<R>(S->psiz), st));
    const bool last = (k == p.dualfb_iters - 1);
    launch_begin(GBRI_K_UPDATE, st);
    k_admm_zbar<R><<<ib, 256, 0, st>>>(vec<R>(S->xt), vec<R>(S->psiz), vec<R>(S->xhat), vec<R>(S->x), N, last,
                                       S->partials);
    GBRI_TRY(launch_end(GBRI_K_UPDATE, st));
  }
  launch_begin(GBRI_K_OTHER, st);
  k_rel_change<<<1, 256, 0, st>>>(S->partials, ib, S->sc);
  return launch_end(GBRI_K_OTHER, st);
}

template <class R>
int32_t fista_iteration(gbri_solver* S, cudaStream_t st) {
  gbri_plan* P = S->plan;
  gbri_wavelet* W = S->wav;
  const auto& p = S->p;
  const int n = P->n_side;
  const int64_t N = (int64_t)n * n;
  // r = Phi xhat - y (into u)
  GBRI_TRY(launch_pad<R>(P, vec<R>(S->xhat), nullptr, st));
  GBRI_TRY(fft_forward(P, st));
  const EpiResid<R> er{cvec<R>(S->u), cvec<R>(S->yp), S->partials, acc_t<R>{}};
  bool fused = false;
  if constexpr (sizeof(R) == 4) {
    if (fused_pd_applies(P)) {  // degridding + gridding of the residual in one pass
      GBRI_TRY(launch_degrid_grid(P, er, st, false));
      fused = true;
    }
  }
  if (!fused) {
    GBRI_TRY(launch_degrid(P, er, st));
    // z = xhat - lambda Re Phi^dagger r (into xt); zbar = P_C(z) (into zb)
    GBRI_TRY(launch_grid(P, SrcPlan<R>{cvec<R>(S->u)}, st));
  }
  GBRI_TRY(fft_inverse_real(P, st));
  const int ib = std::min(img_blocks(N), S->n_partials / 2);
  launch_begin(GBRI_K_UPDATE, st);
  k_admm_xt<R><<<ib, 256, 0, st>>>(P->as<const R>(P->grid), P->as<const R>(P->corr), vec<R>(S->xhat),
                                   vec<R>(S->xt), vec<R>(S->zb), n, P->K, (R)p.rho);
  GBRI_TRY(launch_end(GBRI_K_UPDATE, st));
  launch_begin(GBRI_K_OTHER, st);
  k_fista_theta<<<1, 32, 0, st>>>(S->sc);
  GBRI_TRY(launch_end(GBRI_K_OTHER, st));
  // x+ = DualFB(z, lambda gamma), d warm-started in z1; the last step also extrapolates
  const double thr = p.rho * p.gamma;
  for (int k = 0; k < p.dualfb_iters; ++k) {
    GBRI_TRY(psi_adjoint_apply<R>(W, vec<R>(S->zb), vec<R>(S->z1) /* d */,
                                  DualEpi{1, p.eta, 1.0, thr, 1.0 / p.eta, S->wts}, st));
    GBRI_TRY(psi_apply<R>(W, vec<R>(S->z1), vec<R>(S->psiz), st));
    launch_begin(GBRI_K_UPDATE, st);
    if (k < p.dualfb_iters - 1)
      k_admm_zbar<R><<<ib, 256, 0, st>>>(vec<R>(S->xt), vec<R>(S->psiz), vec<R>(S->zb), vec<R>(S->x), N, false,
                                         S->partials);
    else
      k_fista_last<R><<<ib, 256, 0, st>>>(vec<R>(S->xt), vec<R>(S->psiz), vec<R>(S->xhat), vec<R>(S->x), N, S->sc,
                                          S->partials);
    GBRI_TRY(launch_end(GBRI_K_UPDATE, st));
  }
  launch_begin(GBRI_K_OTHER, st);
  k_rel_change<<<1, 256, 0, st>>>(S->partials, ib, S->sc);
  return launch_end(GBRI_K_OTHER, st);
}

int32_t iteration(gbri_solver* S, cudaStream_t st) {
  const int a = S->p.algo;
  if (S->prec == GBRI_F64)
    return a == GBRI_ALGO_PD ? pd_iteration<double>(S, st)
                             : (a == GBRI_ALGO_ADMM ? admm_iteration<double>(S, st) : fista_iteration<double>(S, st));
  return a == GBRI_ALGO_PD ? pd_iteration<float>(S, st)
                           : (a == GBRI_ALGO_ADMM ? admm_iteration<float>(S, st) : fista_iteration<float>(S, st));
}

// ||y - Phi x|| into sc[SC_RES] (uses the plan's visibility scratch)
template <class R>
int32_t residual(gbri_solver* S, cudaStream_t st) {
  gbri_plan* P = S->plan;
  GBRI_TRY(launch_pad<R>(P, vec<R>(S->x), nullptr, st));
  GBRI_TRY(fft_forward(P, st));
  if (P->M > 0) GBRI_TRY(launch_degrid(P, EpiStorePlan<R>{P->as<cplx<R>>(P->vis_tmp)}, st));
  const int b = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(ceil_div(P->M, 2048), S->n_partials),
                                                             (int64_t)num_sms() * 4));
  launch_begin(GBRI_K_OTHER, st);
  k_residual_partials<R><<<b, 256, 0, st>>>(P->as<const cplx<R>>(P->vis_tmp), cvec<R>(S->yp), P->M, S->partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, st));
  launch_begin(GBRI_K_OTHER, st);
  k_sqrt_sum<<<1, 256, 0, st>>>(S->partials, b, S->sc + SC_RES);
  return launch_end(GBRI_K_OTHER, st);
}

// gamma = 1e-3 max|Psi^dagger Phi^dagger y| / ||Phi||^2
template <class R>
int32_t default_gamma(gbri_solver* S, cudaStream_t st, double* out) {
  gbri_plan* P = S->plan;
  const int64_t N = (int64_t)P->n_side * P->n_side;
  GBRI_TRY(launch_grid(P, SrcPlan<R>{cvec<R>(S->yp)}, st));
  GBRI_TRY(fft_inverse_real(P, st));
  GBRI_TRY(launch_crop<R>(P, vec<R>(S->psiz), st));
  GBRI_TRY(psi_adjoint_apply<R>(S->wav, vec<R>(S->psiz), vec<R>(S->z1), DualEpi{0, 0.0, 0.0, 0.0, 0.0}, st));
  const int64_t tot = N * S->wav->nw;
  const int b = std::min(img_blocks(tot), S->n_partials);
  launch_begin(GBRI_K_OTHER, st);
  k_absmax_partials<R><<<b, 256, 0, st>>>(vec<R>(S->z1), tot, S->partials);
  GBRI_TRY(launch_end(GBRI_K_OTHER, st));
  launch_begin(GBRI_K_OTHER, st);
  k_max_finish<<<1, 32, 0, st>>>(S->partials, b, S->sc + SC_MAX);
  GBRI_TRY(launch_end(GBRI_K_OTHER, st));
  double m = 0;
  GBRI_CHECK_CUDA(cudaMemcpyAsync(&m, S->sc + SC_MAX, sizeof(double), cudaMemcpyDeviceToHost, st));
  GBRI_CHECK_CUDA(cudaStreamSynchronize(st));
  *out = 1e-3 * m / S->p.op_norm_sq;
  return GBRI_OK;
}

bool use_graphs() {
  const char* e = getenv("GBRI_GRAPHS");
  return !(e && e[0] == '0');
}

// Capture one iteration on a private stream (the caller's stream may be the legacy
// default stream, which cannot be captured) and instantiate it.
int32_t capture_iteration(gbri_solver* S) {
  if (!S->cap_stream) GBRI_CHECK_CUDA(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
  const int64_t before = launch_counter();
  GBRI_CHECK_CUDA(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeThreadLocal));
  const int32_t r = iteration(S, S->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(S->cap_stream, &g);
  const int64_t captured = launch_counter() - before;
  add_launches(-captured);  // capturing launches nothing
  if (r != GBRI_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_error(e2, "cudaGraphInstantiate");
  }
  S->graph = g;
  S->graph_exec = ex;
  S->launches_per_iter = captured;
  return GBRI_OK;
}

template <class T>
int32_t zalloc(T** p, size_t n, cudaStream_t s) {
  if (n == 0) n = 1;
  if (alloc_fault_injected() || cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) {
    *p = nullptr;
    return set_error(GBRI_ENOMEM, "cudaMalloc solver state");
  }
  GBRI_CHECK_CUDA(cudaMemsetAsync(*p, 0, n * sizeof(T), s));
  return GBRI_OK;
}

// zeroed device buffer of `bytes` bytes
int32_t zalloc_bytes(void** p, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (alloc_fault_injected() || cudaMalloc(p, bytes) != cudaSuccess) {
    *p = nullptr;
    return set_error(GBRI_ENOMEM, "cudaMalloc solver state");
  }
  GBRI_CHECK_CUDA(cudaMemsetAsync(*p, 0, bytes, s));
  return GBRI_OK;
}

// Local l2 balls: cut the plan order at tile boundaries (the plan's degridding chunks are
// tile-contiguous and ascending) into S->nb ranges; ball j < nb - 1 ends after the first
// tile at which C * nb >= (j + 1) * M (C = cumulative count), at most one ball per tile;
// radius eps_j = eps sqrt(M_j / M).
int32_t setup_balls(gbri_solver* S, cudaStream_t st) {
  gbri_plan* P = S->plan;
  const int nb = S->nb;
  const int64_t M = P->M;
  std::vector<int4> ch((size_t)P->n_chunks);
  if (!ch.empty()) {
    GBRI_CHECK_CUDA(cudaMemcpyAsync(ch.data(), P->chunks, ch.size() * sizeof(int4), cudaMemcpyDeviceToHost, st));
    GBRI_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int32_t> start(1, 0);
  int64_t cum = 0;
  for (size_t k = 0; k < ch.size(); ++k) {
    cum += ch[k].z;
    const bool tile_end = (k + 1 == ch.size()) || ch[k + 1].x != ch[k].x;
    const int j = (int)start.size() - 1;
    if (tile_end && j < nb - 1 && cum * nb >= (int64_t)(j + 1) * M) start.push_back((int32_t)cum);
  }
  start.push_back((int32_t)M);
  GBRI_CHECK((int)start.size() == nb + 1, GBRI_EINVAL, "too few tiles for the requested number of l2 balls");
  std::vector<double> eps(nb);
  for (int j = 0; j < nb; ++j) {
    GBRI_CHECK(start[j + 1] > start[j], GBRI_EINVAL, "empty l2 ball");
    eps[j] = S->p.eps * std::sqrt((double)(start[j + 1] - start[j]) / (double)M);
  }
  GBRI_TRY(zalloc(&S->bstart, (size_t)nb + 1, st));
  GBRI_TRY(zalloc(&S->beps, (size_t)nb, st));
  GBRI_TRY(zalloc(&S->bsc, (size_t)nb, st));
  GBRI_TRY(zalloc(&S->bpart, (size_t)nb * P->degrid_blocks, st));
  GBRI_CHECK_CUDA(cudaMemcpyAsync(S->bstart, start.data(), start.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  GBRI_CHECK_CUDA(cudaMemcpyAsync(S->beps, eps.data(), eps.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  GBRI_CHECK_CUDA(cudaStreamSynchronize(st));  // host vectors go out of scope
  return GBRI_OK;
}

int32_t create_solver(gbri_solver* S, const void* d_y, uint32_t flags, cudaStream_t st) {
  gbri_plan* P = S->plan;
  const int64_t N = (int64_t)P->n_side * P->n_side;
  const int64_t M = P->M;
  const int nw = S->wav->nw;
  const size_t rb = real_bytes(S->prec);
  auto& p = S->p;
  S->n_partials = std::max(std::max(P->degrid_blocks, 2 * img_blocks(N * nw)), 2048);
  {  // the wavelet branch at the highest stream priority: its blocks are dispatched first
     // as visibility-kernel blocks retire, so the shorter branch does not trail the longer
    int least = 0, greatest = 0;
    GBRI_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    GBRI_CHECK_CUDA(cudaStreamCreateWithPriority(&S->aux_stream, cudaStreamNonBlocking, greatest));
  }
  GBRI_CHECK_CUDA(cudaEventCreateWithFlags(&S->ev_fork, cudaEventDisableTiming));
  GBRI_CHECK_CUDA(cudaEventCreateWithFlags(&S->ev_join, cudaEventDisableTiming));
  GBRI_CHECK_CUDA(cudaEventCreateWithFlags(&S->ev_zero, cudaEventDisableTiming));
  GBRI_TRY(zalloc(&S->partials, (size_t)S->n_partials * 2, st));
  GBRI_TRY(zalloc(&S->done, 2, st));
  GBRI_TRY(zalloc(&S->sc, SC_N, st));
  GBRI_TRY(zalloc_bytes(&S->yp, (size_t)M * 2 * rb, st));
  GBRI_TRY(zalloc_bytes(&S->u, (size_t)M * 2 * rb, st));
  if (p.algo == GBRI_ALGO_ADMM) GBRI_TRY(zalloc_bytes(&S->w, (size_t)M * 2 * rb, st));
  GBRI_TRY(zalloc_bytes(&S->x, (size_t)N * rb, st));
  GBRI_TRY(zalloc_bytes(&S->xhat, (size_t)N * rb, st));
  GBRI_TRY(zalloc_bytes(&S->psiz, (size_t)N * rb, st));
  GBRI_TRY(zalloc_bytes(&S->xt, (size_t)N * rb, st));
  if (p.algo == GBRI_ALGO_FISTA) GBRI_TRY(zalloc_bytes(&S->zb, (size_t)N * rb, st));
  GBRI_TRY(zalloc_bytes(&S->z1, (size_t)(N * nw) * rb, st));
  if (M > 0) {
    if (flags & GBRI_PLAN_ORDER)
      GBRI_CHECK_CUDA(cudaMemcpyAsync(S->yp, d_y, (size_t)M * 2 * rb, cudaMemcpyDeviceToDevice, st));
    else
      GBRI_TRY(gbri_vis_reorder(P, d_y, S->yp, 1, st));
  }
  // resolve defaults
  if (p.max_iter < 0) return set_error(GBRI_EINVAL, "max_iter < 0");
  if (p.reserved != 0) return set_error(GBRI_EINVAL, "reserved must be 0");
  if (p.n_balls < 0 || p.n_balls > kMaxBalls) return set_error(GBRI_EINVAL, "n_balls must be in [0, 64]");
  if (p.n_balls >= 2 && p.algo != GBRI_ALGO_FISTA && M > 0) {
    S->nb = p.n_balls;
    GBRI_TRY(setup_balls(S, st));
  }
  if (p.algo != GBRI_ALGO_FISTA && !(p.eps > 0)) return set_error(GBRI_EINVAL, "eps must be > 0");
  if (p.op_norm_sq <= 0) {
    int32_t it = 0;
    GBRI_TRY(gbri_op_norm(P, 200, 1e-8, p.seed, &p.op_norm_sq, &it, st));
  }
  if (p.tau <= 0) p.tau = 0.49;
  if (p.sigma1 <= 0) p.sigma1 = 1.0;
  if (p.sigma2 <= 0) p.sigma2 = 1.0 / p.op_norm_sq;
  if (p.theta < 0) p.theta = 1.0;
  if (p.rho <= 0) p.rho = 1.0 / p.op_norm_sq;
  if (p.varrho <= 0) p.varrho = 1.0;
  if (p.eta <= 0) p.eta = 1.0;
  if (p.dualfb_iters <= 0) p.dualfb_iters = 1;
  if (p.check_every <= 0) p.check_every = 10;
  if (p.gamma <= 0) {
    GBRI_TRY(S->prec == GBRI_F64 ? default_gamma<double>(S, st, &p.gamma) : default_gamma<float>(S, st, &p.gamma));
    if (p.algo == GBRI_ALGO_FISTA) p.gamma *= p.op_norm_sq;  // 1e-3 max|Psi^dagger Phi^dagger y|
  }
  // x = 0, xhat = 0, duals = 0, c = 0, FISTA theta = 1
  GBRI_CHECK_CUDA(cudaMemsetAsync(S->z1, 0, rb * N * nw, st));
  GBRI_CHECK_CUDA(cudaMemsetAsync(S->psiz, 0, rb * N, st));
  GBRI_CHECK_CUDA(cudaMemsetAsync(S->sc, 0, sizeof(double) * SC_N, st));
  const double one = 1.0;
  GBRI_CHECK_CUDA(cudaMemcpyAsync(S->sc + SC_THETA, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  GBRI_CHECK_CUDA(cudaMemcpyAsync(S->sc + SC_ONE, &one, sizeof(double), cudaMemcpyHostToDevice, st));
  if (S->nb) GBRI_CHECK_CUDA(cudaMemsetAsync(S->bsc, 0, sizeof(double) * S->nb, st));  // c_j = 0 before the first step
  GBRI_CHECK_CUDA(cudaStreamSynchronize(st));  // the host scalar goes out of scope
  return GBRI_OK;
}

}  // namespace

namespace gbri {

int32_t solver_iteration_graph(gbri_solver* s) {
  if (s->graph_exec) return GBRI_OK;
  GBRI_CHECK(!profiling_enabled(), GBRI_EINVAL, "batched graphs cannot run while kernel timing is on");
  return capture_iteration(s);
}
cudaGraph_t solver_graph(gbri_solver* s) { return s->graph; }
int64_t solver_graph_version(const gbri_solver* s) { return s->graph_version; }
int64_t solver_launches_per_iteration(gbri_solver* s) { return s->launches_per_iter; }
const gbri_plan* solver_plan(const gbri_solver* s) { return s->plan; }
const gbri_wavelet* solver_wavelet(const gbri_solver* s) { return s->wav; }
void solver_add_iterations(gbri_solver* s, int n) { s->iters += n; }

bool solver_fused_eligible(const gbri_solver* s) {
  const gbri_plan* P = s->plan;
  return s->prec == GBRI_F32 && s->p.algo == GBRI_ALGO_PD && s->nb == 0 && P->step_layout && !P->det &&
         fused_pd_applies(P) && !profiling_enabled();
}

int32_t solver_phase(gbri_solver* s, int phase, cudaStream_t st) {
  GBRI_CHECK(solver_fused_eligible(s), GBRI_EINVAL, "solver cannot split its iteration around a shared pass");
  return pd_iteration<float>(s, st, phase);
}

cudaStream_t solver_stream(gbri_solver* s) {
  if (!s->cap_stream && cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
    return nullptr;
  return s->cap_stream;
}

void solver_fused_member(const gbri_solver* s, FusedMember* m) {
  const gbri_plan* P = s->plan;
  m->meta = P->meta;
  m->steps = P->steps;
  m->gtiles = P->gtiles;
  m->spec = P->as<const float2>(P->spec);
  m->grid = P->as<float2>(P->grid);
  m->u = static_cast<float2*>(s->u);
  m->y = static_cast<const float2*>(s->yp);
  m->c = s->sc + SC_C;
  m->dist = s->sc + SC_DIST;
  m->eps = s->p.eps;
  m->sigma2d = s->p.sigma2;
  m->sigma2 = (float)s->p.sigma2;
  m->K = P->K;
  m->nT = P->nT;
  m->log2S = P->log2S;
  m->item0 = 0;
  m->M = P->M;
  m->dbg = P->dbg;
}

}  // namespace gbri

extern "C" {

int32_t gbri_solver_capture(gbri_solver* s) {
  GBRI_CHECK(s, GBRI_EINVAL, "null solver");
  return solver_iteration_graph(s);
}

int32_t gbri_solver_create(gbri_solver** out, gbri_plan* plan, gbri_wavelet* wav, const void* d_y,
                           const gbri_solve_params* params, uint32_t flags, void* stream) {
  GBRI_CHECK(out && plan && wav && params && (d_y || plan->M == 0), GBRI_EINVAL, "null argument");
  *out = nullptr;
  GBRI_CHECK(wav->n == plan->n_side, GBRI_EINVAL, "wavelet and plan image sizes differ");
  GBRI_CHECK(wav->prec == plan->prec, GBRI_EINVAL, "wavelet and plan precisions differ");
  GBRI_CHECK(params->algo == GBRI_ALGO_PD || params->algo == GBRI_ALGO_ADMM || params->algo == GBRI_ALGO_FISTA,
             GBRI_EINVAL, "unknown algo");
  gbri_solver* S = new (std::nothrow) gbri_solver();
  GBRI_CHECK(S, GBRI_ENOMEM, "host allocation");
  S->plan = plan;
  S->wav = wav;
  S->prec = plan->prec;
  S->p = *params;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t r = create_solver(S, d_y, flags, st);
  if (r != GBRI_OK) {
    cudaStreamSynchronize(st);
    free_solver(S);
    return r;
  }
  *out = S;
  return GBRI_OK;
}

int32_t gbri_solver_destroy(gbri_solver* S) {
  if (S) cudaDeviceSynchronize();
  free_solver(S);
  return GBRI_OK;
}

int32_t gbri_solver_step(gbri_solver* S, int32_t n_iter, void* stream) {
  GBRI_CHECK(S && n_iter >= 0, GBRI_EINVAL, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (n_iter == 0) return GBRI_OK;
  if (use_graphs() && !profiling_enabled() && !S->graph_failed) {
    if (!S->graph_exec) {
      const int32_t r = capture_iteration(S);
      if (r != GBRI_OK) S->graph_failed = true;  // fall back to direct launches
    }
    if (S->graph_exec) {
      for (int k = 0; k < n_iter; ++k) {
        GBRI_CHECK_CUDA(cudaGraphLaunch(S->graph_exec, st));
        ++S->iters;
      }
      add_launches(S->launches_per_iter * n_iter);
      return GBRI_OK;
    }
  }
  for (int k = 0; k < n_iter; ++k) {
    GBRI_TRY(iteration(S, st));
    ++S->iters;
  }
  return GBRI_OK;
}

int32_t gbri_solver_reweight(gbri_solver* S, double delta, void* stream) {
  GBRI_CHECK(S && delta > 0, GBRI_EINVAL, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t N = (int64_t)S->plan->n_side * S->plan->n_side;
  const int64_t tot = N * S->wav->nw;
  if (!S->wts) {
    GBRI_TRY(zalloc_bytes(&S->wts, (size_t)tot * real_bytes(S->prec), st));
    // the captured iteration holds the (null) weights pointer: capture again on the next step
    if (S->graph_exec) cudaGraphExecDestroy(S->graph_exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    S->graph_exec = nullptr;
    S->graph = nullptr;
    ++S->graph_version;
  }
  const int b = img_blocks(tot);
  if (S->prec == GBRI_F64) {
    GBRI_TRY(psi_adjoint_apply<double>(S->wav, vec<double>(S->x), vec<double>(S->wts), DualEpi{0, 0.0, 0.0, 0.0, 0.0},
                                       st));
    launch_begin(GBRI_K_OTHER, st);
    k_sara_weights<double><<<b, 256, 0, st>>>(vec<double>(S->wts), tot, delta);
  } else {
    GBRI_TRY(psi_adjoint_apply<float>(S->wav, vec<float>(S->x), vec<float>(S->wts), DualEpi{0, 0.0, 0.0, 0.0, 0.0},
                                      st));
    launch_begin(GBRI_K_OTHER, st);
    k_sara_weights<float><<<b, 256, 0, st>>>(vec<float>(S->wts), tot, (float)delta);
  }
  return launch_end(GBRI_K_OTHER, st);
}

int32_t gbri_solver_get_x(gbri_solver* S, void* d_x, void* stream) {
  GBRI_CHECK(S && d_x, GBRI_EINVAL, "null argument");
  const int64_t N = (int64_t)S->plan->n_side * S->plan->n_side;
  GBRI_CHECK_CUDA(cudaMemcpyAsync(d_x, S->x, real_bytes(S->prec) * N, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream));
  return GBRI_OK;
}

int32_t gbri_solver_status(gbri_solver* S, int32_t* iters, double* rel_change, void* stream) {
  GBRI_CHECK(S, GBRI_EINVAL, "null solver");
  double rel = INFINITY;
  if (S->iters > 0) {
    cudaStream_t st = (cudaStream_t)stream;
    GBRI_CHECK_CUDA(cudaMemcpyAsync(&rel, S->sc + SC_REL, sizeof(double), cudaMemcpyDeviceToHost, st));
    GBRI_CHECK_CUDA(cudaStreamSynchronize(st));
  }
  if (iters) *iters = S->iters;
  if (rel_change) *rel_change = rel;
  return GBRI_OK;
}

int32_t gbri_solver_report(gbri_solver* S, gbri_solve_report* r, void* stream) {
  GBRI_CHECK(S && r, GBRI_EINVAL, "null argument");
  cudaStream_t st = (cudaStream_t)stream;
  GBRI_TRY(S->prec == GBRI_F64 ? residual<double>(S, st) : residual<float>(S, st));
  double sc[SC_N];
  GBRI_CHECK_CUDA(cudaMemcpyAsync(sc, S->sc, sizeof(sc), cudaMemcpyDeviceToHost, st));
  GBRI_CHECK_CUDA(cudaStreamSynchronize(st));
  r->iters = S->iters;
  r->status = GBRI_OK;
  r->rel_change = S->iters > 0 ? sc[SC_REL] : INFINITY;
  r->residual_norm = sc[SC_RES];
  r->op_norm_sq = S->p.op_norm_sq;
  r->gamma = S->p.gamma;
  r->ms_total = S->ms_total;
  return GBRI_OK;
}

int32_t gbri_solve(gbri_plan* plan, gbri_wavelet* wav, const void* d_y, const gbri_solve_params* params,
                   void* d_x_out, gbri_solve_report* report, uint32_t flags, void* stream) {
  GBRI_CHECK(d_x_out, GBRI_EINVAL, "null x");
  gbri_solver* S = nullptr;
  GBRI_TRY(gbri_solver_create(&S, plan, wav, d_y, params, flags, stream));
  cudaStream_t st = (cudaStream_t)stream;
  // wall time of the solve for the report (best effort: without events it reads 0)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  if (timed) cudaEventRecord(e0, st);
  int32_t rc = GBRI_OK;
  bool converged = false;
  const int every = S->p.check_every;
  while (S->iters < S->p.max_iter) {
    const int k = std::min(every, S->p.max_iter - S->iters);
    rc = gbri_solver_step(S, k, stream);
    if (rc != GBRI_OK) break;
    if (S->p.rel_tol > 0) {
      double rel = 0;
      if (cudaMemcpyAsync(&rel, S->sc + SC_REL, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) {
        rc = set_error(GBRI_ECUDA, "convergence read");
        break;
      }
      if (rel < S->p.rel_tol) {
        converged = true;
        break;
      }
    }
  }
  if (timed) cudaEventRecord(e1, st);
  if (rc == GBRI_OK) rc = gbri_solver_get_x(S, d_x_out, stream);
  if (rc == GBRI_OK) {
    float ms = 0.f;
    if (timed && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
      ms = 0.f;
    S->ms_total = ms;
    gbri_solve_report r{};
    rc = gbri_solver_report(S, &r, stream);
    if (rc == GBRI_OK) {
      r.status = (S->p.rel_tol > 0 && !converged) ? GBRI_ENOTCONV : GBRI_OK;
      if (report) *report = r;
      rc = r.status;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  gbri_solver_destroy(S);
  return rc;
}

}  // extern "C"
