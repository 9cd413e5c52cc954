// Solver internals shared with the batch executor.
#pragma once

#include "common.cuh"

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

}  // namespace gbri
