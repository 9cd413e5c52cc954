// FP64 instantiations of the visibility kernels (the plain FP64 path).
#include "vis_kernels.cuh"

GBRI_INSTANTIATE_VIS(double)
