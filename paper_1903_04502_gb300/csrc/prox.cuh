// Proximal-operator helpers shared by the C entry points and the solvers.
#pragma once

#include "common.cuh"

namespace gbri {

// Blocks used by the l2-ball reduction for M visibilities (= partials needed).
int l2ball_blocks(int64_t M);

// Projection onto the l2 ball of radius eps around d_center with caller-provided
// scratch for the FP64 block partials (n_partials >= l2ball_blocks(M) uses all of them).
// R is the real type of the complex vectors (float: complex64, double: complex128).
template <class R>
int32_t proj_l2ball_with_scratch(const R* d_z, const R* d_center, R* d_out, int64_t M, double eps,
                                 double* d_norm_out, double* partials, int n_partials, cudaStream_t s);

}  // namespace gbri
