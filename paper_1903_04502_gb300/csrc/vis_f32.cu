// FP32 instantiations of the visibility kernels (FP32 bulk, FP64 global sums).
#include "vis_kernels.cuh"

GBRI_INSTANTIATE_VIS(float)
