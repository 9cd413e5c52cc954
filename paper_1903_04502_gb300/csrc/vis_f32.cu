// FP32 instantiations of the visibility kernels (FP32 bulk, FP64 global sums), including
// the polynomial-tap kernels of vis_fast.cuh.
#include "vis_fast.cuh"
#include "vis_kernels.cuh"
#include "vis_steps.cuh"

GBRI_INSTANTIATE_VIS(float)

namespace gbri {

template <class Epi>
int32_t launch_degrid_fast(gbri_plan* p, Epi epi, cudaStream_t s) {
  launch_begin(GBRI_K_DEGRID, s);
  const VisGeom geo = vis_geom(p);
  const float2* g = p->as<const float2>(p->spec);
  const size_t sm = degrid_smem(p);
  if (p->J == 4) k_degrid_fast<4, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi, p->work);
  else k_degrid_fast<6, Epi><<<p->degrid_blocks, kThreads, sm, s>>>(geo, g, epi, p->work);
  return launch_end(GBRI_K_DEGRID, s);
}

template <class Src>
int32_t launch_grid_fast(gbri_plan* p, Src src, cudaStream_t s) {
  launch_begin(GBRI_K_GRID, s);
  const size_t sm = grid_smem(p);
  const VisGeom geo = vis_geom(p);
  float2* g = p->as<float2>(p->grid);
  if (p->step_layout)
    k_steps<kStepGrid, Src><<<p->grid_blocks, kThreads, step_smem<kStepGrid, Src>(), s>>>(geo, nullptr, g, src,
                                                                                         p->work + 2);
  else if (p->J == 4) k_grid_fast<4, Src><<<p->grid_blocks, kThreads, sm, s>>>(geo, g, src, p->work + 2);
  else k_grid_fast<6, Src><<<p->grid_blocks, kThreads, sm, s>>>(geo, g, src, p->work + 2);
  return launch_end(GBRI_K_GRID, s);
}

#define GBRI_FAST_DG(E) template int32_t launch_degrid_fast<E<float>>(gbri_plan*, E<float>, cudaStream_t);
#define GBRI_FAST_GR(S) template int32_t launch_grid_fast<S<float>>(gbri_plan*, S<float>, cudaStream_t);
GBRI_FAST_DG(EpiStorePlan) GBRI_FAST_DG(EpiStoreRaw) GBRI_FAST_DG(EpiPD1) GBRI_FAST_DG(EpiADMM1)
GBRI_FAST_DG(EpiResid) GBRI_FAST_DG(EpiPD1L) GBRI_FAST_DG(EpiADMM1L)
GBRI_FAST_GR(SrcScaledL) GBRI_FAST_GR(SrcADMM2L) GBRI_FAST_GR(SrcPlan) GBRI_FAST_GR(SrcRaw) GBRI_FAST_GR(SrcADMM2)
#undef GBRI_FAST_DG
#undef GBRI_FAST_GR

cudaError_t prepare_fast_kernels() {
  const int lim = 220 * 1024;
  cudaError_t e = cudaSuccess;
#define GBRI_ATTR(kern) if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
#define GBRI_ATTR_DG(E) GBRI_ATTR((k_degrid_fast<4, E<float>>)); GBRI_ATTR((k_degrid_fast<6, E<float>>))
#define GBRI_ATTR_GR(S) GBRI_ATTR((k_grid_fast<4, S<float>>)); GBRI_ATTR((k_grid_fast<6, S<float>>))
  GBRI_ATTR_DG(EpiStorePlan); GBRI_ATTR_DG(EpiStoreRaw); GBRI_ATTR_DG(EpiPD1); GBRI_ATTR_DG(EpiADMM1);
  GBRI_ATTR_DG(EpiResid); GBRI_ATTR_DG(EpiPD1L); GBRI_ATTR_DG(EpiADMM1L);
  GBRI_ATTR_GR(SrcScaledL); GBRI_ATTR_GR(SrcADMM2L); GBRI_ATTR_GR(SrcPlan); GBRI_ATTR_GR(SrcRaw); GBRI_ATTR_GR(SrcADMM2);
  GBRI_ATTR((k_degrid_grid_fast<4, EpiPD1<float>>));
  GBRI_ATTR((k_degrid_grid_fast<4, EpiResid<float>>));
  GBRI_ATTR((k_steps<kStepGrid, SrcScaledL<float>>)); GBRI_ATTR((k_steps<kStepGrid, SrcADMM2L<float>>));
  GBRI_ATTR((k_steps<kStepGrid, SrcPlan<float>>)); GBRI_ATTR((k_steps<kStepGrid, SrcRaw<float>>));
  GBRI_ATTR((k_steps<kStepGrid, SrcADMM2<float>>));
  GBRI_ATTR((k_steps<kStepFused, EpiPD1<float>>)); GBRI_ATTR((k_steps<kStepFused, EpiResid<float>>));
  GBRI_ATTR(k_steps_multi);
#undef GBRI_ATTR_DG
#undef GBRI_ATTR_GR
#undef GBRI_ATTR
  return e;
}

int32_t launch_fused_multi(const FusedMember* d_mem, int n_mem, int n_items, double* d_sums, const PolyTaps& poly,
                           unsigned int* d_ctr, cudaStream_t s) {
  GBRI_CHECK(n_mem >= 1 && n_mem <= kMaxFusedMembers, GBRI_EINVAL, "fused pass: 1 to 256 members");
  if (n_items == 0) return GBRI_OK;
  // two blocks per SM, as the single-problem pass
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n_items, kThreads / 32), num_sms() * 2));
  launch_begin(GBRI_K_DEGRID_GRID, s);
  k_steps_multi<<<blocks, kThreads, steps_multi_smem(), s>>>(d_mem, n_mem, n_items, d_sums, poly, d_ctr);
  return launch_end(GBRI_K_DEGRID_GRID, s);
}

template <class Epi>
int32_t degrid_grid(gbri_plan* p, Epi epi, cudaStream_t s, bool zeroed) {
  float2* g = p->as<float2>(p->grid);
  // deterministic plans: the item windows go to slots and the fixed-order pass writes every cell
  if (!zeroed && !p->det) GBRI_CHECK_CUDA(cudaMemsetAsync(g, 0, sizeof(float2) * (size_t)p->K * p->K, s));
  // two blocks per SM (a window and an accumulator per warp); each block writes one
  // partial of the epilogue's sum of squares
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(p->n_gtiles, kThreads / 32), (int64_t)num_sms() * 2));
  launch_begin(GBRI_K_DEGRID_GRID, s);
  const size_t sm = degrid_grid_smem(p);
  const VisGeom geo = vis_geom(p);
  const float2* spec = p->as<const float2>(p->spec);
  if (p->step_layout)
    k_steps<kStepFused, Epi><<<blocks, kThreads, step_smem<kStepFused, Epi>(), s>>>(geo, spec, g, epi, p->work + 4);
  else if (p->tap_mode == kTapPoly)
    k_degrid_grid_fast<4, Epi><<<blocks, kThreads, sm, s>>>(geo, spec, g, epi, p->work + 4);
  else if (p->tap_mode == kTapFO) k_degrid_grid<4, kTapFO, Epi><<<blocks, kThreads, sm, s>>>(geo, spec, g, epi);
  else k_degrid_grid<4, kTapTable, Epi><<<blocks, kThreads, sm, s>>>(geo, spec, g, epi);
  GBRI_TRY(launch_end(GBRI_K_DEGRID_GRID, s));
  return p->det ? launch_grid_reduce<float>(p, s) : GBRI_OK;
}

int32_t launch_degrid_grid(gbri_plan* p, EpiPD1<float> epi, cudaStream_t s, bool zeroed) {
  return degrid_grid(p, epi, s, zeroed);
}
int32_t launch_degrid_grid(gbri_plan* p, EpiResid<float> epi, cudaStream_t s, bool zeroed) {
  return degrid_grid(p, epi, s, zeroed);
}

}  // namespace gbri
