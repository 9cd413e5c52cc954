// Solver internals shared with the batch executor.
#pragma once

#include "common.cuh"
#include "nufft.cuh"

namespace gbri {

// Captures the solver's iteration as a CUDA graph if it has not been captured yet.
int32_t solver_iteration_graph(gbri_solver* s);
cudaGraph_t solver_graph(gbri_solver* s);
// Incremented whenever the solver's captured iteration is dropped (a batch holding a copy
// rebuilds its graph).
int64_t solver_graph_version(const gbri_solver* s);
int64_t solver_launches_per_iteration(gbri_solver* s);
const gbri_plan* solver_plan(const gbri_solver* s);
const gbri_wavelet* solver_wavelet(const gbri_solver* s);
// Account for iterations run by a batch replay.
void solver_add_iterations(gbri_solver* s, int n);
// A primal-dual solver with a global l2 ball on an FP32 step-layout plan (not deterministic):
// its fused degridding + gridding pass can run inside a batch's pass over several problems.
bool solver_fused_eligible(const gbri_solver* s);
// Enqueues phase 1 (up to the forward FFT, then a wait for the zeroed grid) or phase 2 (from
// the inverse FFT on) of such a solver's iteration on st; the shared pass goes between.
int32_t solver_phase(gbri_solver* s, int phase, cudaStream_t st);
// The solver's private stream (created on first use; null if that fails).
cudaStream_t solver_stream(gbri_solver* s);
// Its entry of the shared pass (item0 left 0).
void solver_fused_member(const gbri_solver* s, FusedMember* m);

}  // namespace gbri
