// Batched execution of many resident solvers: one CUDA graph launched once per batch
// iteration.  Problems of different image size, visibility count and kernel support run
// side by side on the device; membership can change between steps (continuous batching),
// which rebuilds the graph.
//
// Members that are primal-dual solvers with a global l2 ball on FP32 step-layout plans
// sharing one kernel polynomial (solver_fused_eligible) share one launch of the fused
// degridding + gridding pass (k_steps_multi, a work list over all of their gridding items):
// each such member's iteration is enqueued in two phases on its own stream, the first up to
// its forward FFT, the second from its inverse FFT on, and the shared pass runs between
// them.  Every other member is a branch holding its own captured iteration.
#include <algorithm>
#include <cstring>
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
  // the shared pass
  bool shared_pass = true;             // gbri_batch_set_shared_pass
  int n_fused = 0;                     // members in it at the last rebuild
  cudaStream_t stream = nullptr;       // capture stream of the phased members
  std::vector<cudaEvent_t> events;     // fork / join events of that capture
  gbri::FusedMember* d_members = nullptr;
  double* d_sums = nullptr;
  unsigned int* d_ctr = nullptr;
  int member_cap = 0;
};

namespace {

using gbri::FusedMember;

void drop_graph(gbri_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->dirty = true;
}

void free_shared(gbri_batch* b) {
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  b->events.clear();
  cudaFree(b->d_members);
  cudaFree(b->d_sums);
  cudaFree(b->d_ctr);
  b->d_members = nullptr;
  b->d_sums = nullptr;
  b->d_ctr = nullptr;
  b->member_cap = 0;
}

// Device table, sums and counter for n members (kept across rebuilds while large enough).
int32_t reserve_shared(gbri_batch* b, int n) {
  if (n <= b->member_cap) return GBRI_OK;
  cudaFree(b->d_members);
  cudaFree(b->d_sums);
  cudaFree(b->d_ctr);
  b->d_members = nullptr;
  b->d_sums = nullptr;
  b->d_ctr = nullptr;
  b->member_cap = 0;
  if (cudaMalloc(&b->d_members, sizeof(FusedMember) * n) != cudaSuccess ||
      cudaMalloc(&b->d_sums, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&b->d_ctr, sizeof(unsigned int) * 2) != cudaSuccess)
    return gbri::set_error(GBRI_ENOMEM, "cudaMalloc (batch shared pass)");
  GBRI_CHECK_CUDA(cudaMemset(b->d_sums, 0, sizeof(double) * n));
  GBRI_CHECK_CUDA(cudaMemset(b->d_ctr, 0, sizeof(unsigned int) * 2));
  b->member_cap = n;
  return GBRI_OK;
}

int32_t new_event(gbri_batch* b, cudaEvent_t* e) {
  GBRI_CHECK_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  b->events.push_back(*e);
  return GBRI_OK;
}

// Captures the phased members' iterations around one shared pass into a graph.
int32_t capture_shared(gbri_batch* b, const std::vector<gbri_solver*>& fm, cudaGraph_t* out) {
  const int n = (int)fm.size();
  std::vector<FusedMember> tab(n);
  int items = 0;
  for (int k = 0; k < n; ++k) {
    gbri::solver_fused_member(fm[k], &tab[k]);
    tab[k].item0 = items;
    items += (int)gbri::solver_plan(fm[k])->n_gtiles;
  }
  GBRI_TRY(reserve_shared(b, n));
  GBRI_CHECK_CUDA(cudaMemcpy(b->d_members, tab.data(), sizeof(FusedMember) * n, cudaMemcpyHostToDevice));
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  b->events.clear();
  if (!b->stream) GBRI_CHECK_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
  std::vector<cudaStream_t> ms(n);
  for (int k = 0; k < n; ++k) {
    ms[k] = gbri::solver_stream(fm[k]);
    GBRI_CHECK(ms[k], GBRI_ECUDA, "solver stream");
  }
  cudaEvent_t e0 = nullptr, emid = nullptr;
  GBRI_TRY(new_event(b, &e0));
  GBRI_TRY(new_event(b, &emid));
  std::vector<cudaEvent_t> pre(n), post(n);
  for (int k = 0; k < n; ++k) {
    GBRI_TRY(new_event(b, &pre[k]));
    GBRI_TRY(new_event(b, &post[k]));
  }
  GBRI_CHECK_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  int32_t st = GBRI_OK;
  auto ok = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && st == GBRI_OK) st = gbri::cuda_error(e, what);
    return st == GBRI_OK;
  };
  if (ok(cudaEventRecord(e0, b->stream), "cudaEventRecord (batch fork)")) {
    for (int k = 0; k < n && st == GBRI_OK; ++k) {
      if (!ok(cudaStreamWaitEvent(ms[k], e0, 0), "cudaStreamWaitEvent (batch fork)")) break;
      st = gbri::solver_phase(fm[k], 1, ms[k]);
      if (st != GBRI_OK) break;
      if (!ok(cudaEventRecord(pre[k], ms[k]), "cudaEventRecord (phase 1)")) break;
      ok(cudaStreamWaitEvent(b->stream, pre[k], 0), "cudaStreamWaitEvent (phase 1)");
    }
  }
  if (st == GBRI_OK) {
    gbri::PolyTaps poly{};
    std::memcpy(&poly, &gbri::solver_plan(fm[0])->poly, sizeof(poly));
    st = gbri::launch_fused_multi(b->d_members, n, items, b->d_sums, poly, b->d_ctr, b->stream);
  }
  if (st == GBRI_OK && ok(cudaEventRecord(emid, b->stream), "cudaEventRecord (shared pass)")) {
    for (int k = 0; k < n && st == GBRI_OK; ++k) {
      if (!ok(cudaStreamWaitEvent(ms[k], emid, 0), "cudaStreamWaitEvent (shared pass)")) break;
      st = gbri::solver_phase(fm[k], 2, ms[k]);
      if (st != GBRI_OK) break;
      if (!ok(cudaEventRecord(post[k], ms[k]), "cudaEventRecord (phase 2)")) break;
      ok(cudaStreamWaitEvent(b->stream, post[k], 0), "cudaStreamWaitEvent (phase 2)");
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (st != GBRI_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return gbri::cuda_error(e, "cudaStreamEndCapture (batch)");
  *out = g;
  return GBRI_OK;
}

// Members for the shared pass: eligible ones with the first eligible member's kernel
// polynomial, at most kMaxFusedMembers, heaviest first (their items are taken in that
// order); none unless at least two qualify.
std::vector<gbri_solver*> shared_members(const gbri_batch* b) {
  std::vector<gbri_solver*> fm;
  if (!b->shared_pass) return fm;
  const gbri_plan* first = nullptr;
  for (gbri_solver* s : b->members) {
    if (!gbri::solver_fused_eligible(s)) continue;
    const gbri_plan* P = gbri::solver_plan(s);
    if (!first) first = P;
    else if (std::memcmp(&first->poly, &P->poly, sizeof(P->poly)) != 0) continue;
    if ((int)fm.size() < gbri::kMaxFusedMembers) fm.push_back(s);
  }
  if (fm.size() < 2) fm.clear();
  std::stable_sort(fm.begin(), fm.end(), [](gbri_solver* a, gbri_solver* c) {
    return gbri::solver_plan(a)->M > gbri::solver_plan(c)->M;
  });
  return fm;
}

int32_t rebuild(gbri_batch* b) {
  drop_graph(b);
  const std::vector<gbri_solver*> fm = shared_members(b);
  int64_t launches = 0;
  for (gbri_solver* s : b->members) {
    if (std::find(fm.begin(), fm.end(), s) != fm.end()) continue;
    GBRI_TRY(gbri::solver_iteration_graph(s));
    launches += gbri::solver_launches_per_iteration(s);
  }
  GBRI_CHECK_CUDA(cudaGraphCreate(&b->graph, 0));
  if (!fm.empty()) {
    cudaGraph_t g = nullptr;
    const int64_t before = gbri::launch_counter();
    const int32_t st = capture_shared(b, fm, &g);
    const int64_t captured = gbri::launch_counter() - before;
    gbri::add_launches(-captured);  // capturing launches nothing
    if (st != GBRI_OK) {
      drop_graph(b);
      return st;
    }
    cudaGraphNode_t node;
    const cudaError_t e = cudaGraphAddChildGraphNode(&node, b->graph, nullptr, 0, g);
    cudaGraphDestroy(g);  // the child node holds a copy
    if (e != cudaSuccess) {
      drop_graph(b);
      return gbri::cuda_error(e, "cudaGraphAddChildGraphNode (shared pass)");
    }
    launches += captured;
  }
  for (gbri_solver* s : b->members) {
    if (std::find(fm.begin(), fm.end(), s) != fm.end()) continue;
    cudaGraphNode_t node;
    GBRI_CHECK_CUDA(cudaGraphAddChildGraphNode(&node, b->graph, nullptr, 0, gbri::solver_graph(s)));
  }
  const cudaError_t e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(b);
    return gbri::cuda_error(e, "cudaGraphInstantiate(batch)");
  }
  b->n_fused = (int)fm.size();
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
  free_shared(b);
  if (b->stream) cudaStreamDestroy(b->stream);
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

int32_t gbri_batch_set_shared_pass(gbri_batch* b, int32_t enable) {
  GBRI_CHECK(b && (enable == 0 || enable == 1), GBRI_EINVAL, "bad argument");
  if (b->shared_pass != (enable == 1)) {
    b->shared_pass = enable == 1;
    b->dirty = true;
  }
  return GBRI_OK;
}

int32_t gbri_batch_shared_members(const gbri_batch* b) { return b ? b->n_fused : 0; }

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
