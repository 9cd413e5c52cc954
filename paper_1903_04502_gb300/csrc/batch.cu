// Batched execution of many resident solvers: one CUDA graph whose branches are the
// members' captured iterations (independent problems, no dependencies between
// branches), launched once per batch iteration.  Problems of different image size,
// visibility count and kernel support run side by side on the device; membership
// can change between steps (continuous batching), which rebuilds the graph.
#include <algorithm>
#include <new>
#include <vector>

#include "solver.cuh"

struct gbri_batch {
  std::vector<gbri_solver*> members;
  std::vector<int64_t> versions;  // members' graph versions at the last rebuild
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  int64_t launches_per_iter = 0;
};

namespace {

void drop_graph(gbri_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->dirty = true;
}

int32_t rebuild(gbri_batch* b) {
  drop_graph(b);
  int64_t launches = 0;
  for (gbri_solver* s : b->members) {
    GBRI_TRY(gbri::solver_iteration_graph(s));
    launches += gbri::solver_launches_per_iteration(s);
  }
  GBRI_CHECK_CUDA(cudaGraphCreate(&b->graph, 0));
  for (gbri_solver* s : b->members) {
    cudaGraphNode_t node;
    GBRI_CHECK_CUDA(cudaGraphAddChildGraphNode(&node, b->graph, nullptr, 0, gbri::solver_graph(s)));
  }
  const cudaError_t e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return gbri::cuda_error(e, "cudaGraphInstantiate(batch)");
  }
  b->launches_per_iter = launches;
  b->versions.clear();
  for (gbri_solver* s : b->members) b->versions.push_back(gbri::solver_graph_version(s));
  b->dirty = false;
  return GBRI_OK;
}

}  // namespace

using namespace gbri;

extern "C" {

int32_t gbri_batch_create(gbri_batch** out) {
  GBRI_CHECK(out, GBRI_EINVAL, "null argument");
  *out = new (std::nothrow) gbri_batch();
  GBRI_CHECK(*out, GBRI_ENOMEM, "host allocation");
  return GBRI_OK;
}

int32_t gbri_batch_destroy(gbri_batch* b) {
  if (!b) return GBRI_OK;
  cudaDeviceSynchronize();
  drop_graph(b);
  delete b;
  return GBRI_OK;
}

int32_t gbri_batch_add(gbri_batch* b, gbri_solver* s) {
  GBRI_CHECK(b && s, GBRI_EINVAL, "null argument");
  for (gbri_solver* o : b->members) {
    GBRI_CHECK(o != s, GBRI_EINVAL, "solver is already in the batch");
    GBRI_CHECK(solver_plan(o) != solver_plan(s), GBRI_EINVAL, "two batch members share one plan");
    GBRI_CHECK(solver_wavelet(o) != solver_wavelet(s), GBRI_EINVAL, "two batch members share one wavelet object");
  }
  b->members.push_back(s);
  b->dirty = true;
  return GBRI_OK;
}

int32_t gbri_batch_remove(gbri_batch* b, gbri_solver* s) {
  GBRI_CHECK(b && s, GBRI_EINVAL, "null argument");
  auto it = std::find(b->members.begin(), b->members.end(), s);
  GBRI_CHECK(it != b->members.end(), GBRI_EINVAL, "solver is not in the batch");
  b->members.erase(it);
  b->dirty = true;
  return GBRI_OK;
}

int32_t gbri_batch_size(const gbri_batch* b) { return b ? (int32_t)b->members.size() : 0; }

int32_t gbri_batch_step(gbri_batch* b, int32_t n_iter, void* stream) {
  GBRI_CHECK(b && n_iter >= 0, GBRI_EINVAL, "bad argument");
  if (b->members.empty() || n_iter == 0) return GBRI_OK;
  for (size_t i = 0; !b->dirty && i < b->members.size(); ++i)
    if (i >= b->versions.size() || b->versions[i] != solver_graph_version(b->members[i])) b->dirty = true;
  if (b->dirty) GBRI_TRY(rebuild(b));
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < n_iter; ++k) GBRI_CHECK_CUDA(cudaGraphLaunch(b->exec, st));
  for (gbri_solver* s : b->members) solver_add_iterations(s, n_iter);
  add_launches(b->launches_per_iter * n_iter);
  return GBRI_OK;
}

}  // extern "C"
