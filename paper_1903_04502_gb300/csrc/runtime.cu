// Library runtime: thread-local error messages, the launch counter and the
// optional per-kernel-kind CUDA-event timing used by the benchmark.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gbri {

namespace {
thread_local std::string g_err;

std::mutex g_prof_mu;
int32_t g_prof_cap = 0;
struct KindEvents {
  std::vector<cudaEvent_t> start, stop;
  int64_t used = 0;    // pairs recorded (ring of size cap)
  int64_t total = 0;   // launches seen
};
KindEvents g_kinds[GBRI_K_COUNT];
int64_t g_launches = 0;

void free_events_locked() {
  for (auto& k : g_kinds) {
    for (auto e : k.start) cudaEventDestroy(e);
    for (auto e : k.stop) cudaEventDestroy(e);
    k.start.clear();
    k.stop.clear();
    k.used = k.total = 0;
  }
}
}  // namespace

int32_t set_error(int32_t code, const std::string& msg) {
  g_err = msg;
  return code;
}

int32_t cuda_error(cudaError_t e, const char* what) {
  return set_error(GBRI_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

void launch_begin(int kind, cudaStream_t s, bool own) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (own) ++g_launches;
  if (g_prof_cap > 0) {
    KindEvents& k = g_kinds[kind];
    int64_t slot = k.total % g_prof_cap;
    cudaEventRecord(k.start[slot], s);
  }
}

int32_t launch_end(int kind, cudaStream_t s) {
  cudaError_t e = cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (g_prof_cap > 0) {
      KindEvents& k = g_kinds[kind];
      int64_t slot = k.total % g_prof_cap;
      cudaEventRecord(k.stop[slot], s);
      ++k.total;
      if (k.used < g_prof_cap) ++k.used;
    }
  }
  if (e != cudaSuccess) return cuda_error(e, "kernel launch");
  return GBRI_OK;
}

bool profiling_enabled() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_prof_cap > 0;
}

void add_launches(int64_t n) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_launches += n;
}

int64_t launch_counter() {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

namespace {
std::atomic<int64_t> g_alloc_countdown{0};
}

bool alloc_fault_injected() {
  int64_t v = g_alloc_countdown.load(std::memory_order_relaxed);
  while (v > 0) {
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1, std::memory_order_relaxed)) return v == 1;
  }
  return false;
}

int num_sms() {
  // cached per device ordinal: a host may hold GPUs with different SM counts
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  if (dev >= kMaxDev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

}  // namespace gbri

using namespace gbri;

extern "C" {

const char* gbri_last_error(void) { return g_err.c_str(); }

const char* gbri_version(void) { return "gbri 0.1 (sm_103a)"; }

int32_t gbri_profile_enable(int32_t capacity) {
  if (capacity < 0) return set_error(GBRI_EINVAL, "profile capacity < 0");
  cudaDeviceSynchronize();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  free_events_locked();
  g_prof_cap = 0;
  g_launches = 0;
  for (auto& k : g_kinds) {  // events are created up front so that timing adds no host work per launch
    k.start.resize(capacity);
    k.stop.resize(capacity);
    for (int32_t i = 0; i < capacity; ++i) {
      if (cudaEventCreate(&k.start[i]) != cudaSuccess || cudaEventCreate(&k.stop[i]) != cudaSuccess) {
        free_events_locked();
        return set_error(GBRI_ECUDA, "cudaEventCreate");
      }
    }
  }
  g_prof_cap = capacity;
  return GBRI_OK;
}

int32_t gbri_profile_read(int32_t kind, double* total_ms, int64_t* launches) {
  if (kind < 0 || kind >= GBRI_K_COUNT) return set_error(GBRI_EINVAL, "bad kernel kind");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_error(e, "cudaDeviceSynchronize");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  KindEvents& k = g_kinds[kind];
  double tot = 0.0;
  for (int64_t i = 0; i < k.used; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, k.start[i], k.stop[i]);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventElapsedTime");
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = k.used;
  return GBRI_OK;
}

int32_t gbri_debug_inject_alloc_failure(int32_t after_n) {
  if (after_n < 0) return set_error(GBRI_EINVAL, "after_n < 0");
  g_alloc_countdown.store(after_n, std::memory_order_relaxed);
  return GBRI_OK;
}

int64_t gbri_launch_count(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  return g_launches;
}

void gbri_launch_count_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_launches = 0;
}

}  // extern "C"
