// FP32 instantiations of the visibility kernels (FP32 bulk, FP64 global sums).
#include "vis_kernels.cuh"

GBRI_INSTANTIATE_VIS(float)

namespace gbri {

template <class Epi>
int32_t degrid_grid(gbri_plan* p, Epi epi, cudaStream_t s, bool zeroed) {
  float2* g = p->as<float2>(p->grid);
  if (!zeroed) GBRI_CHECK_CUDA(cudaMemsetAsync(g, 0, sizeof(float2) * (size_t)p->K * p->K, s));
  // two blocks per SM (a window and an accumulator per warp); each block writes one
  // partial of the epilogue's sum of squares
  const int blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>(ceil_div(p->n_gtiles, kThreads / 32), (int64_t)num_sms() * 2));
  launch_begin(GBRI_K_DEGRID_GRID, s);
  if (p->frac)
    k_degrid_grid<4, true, Epi><<<blocks, kThreads, degrid_grid_smem(p), s>>>(vis_geom(p), p->as<const float2>(p->spec),
                                                                             g, epi);
  else
    k_degrid_grid<4, false, Epi><<<blocks, kThreads, degrid_grid_smem(p), s>>>(vis_geom(p),
                                                                              p->as<const float2>(p->spec), g, epi);
  return launch_end(GBRI_K_DEGRID_GRID, s);
}

int32_t launch_degrid_grid(gbri_plan* p, EpiPD1<float> epi, cudaStream_t s, bool zeroed) {
  return degrid_grid(p, epi, s, zeroed);
}
int32_t launch_degrid_grid(gbri_plan* p, EpiResid<float> epi, cudaStream_t s, bool zeroed) {
  return degrid_grid(p, epi, s, zeroed);
}

}  // namespace gbri
