// Kernel-class timing with CUDA events and the launch counter.
//
// Measurement support only: when enabled, each timed launch (or launch group, for
// the Gram's two kernels) is bracketed by two events recorded on the stream that
// runs it, so the elapsed times are device times of that stream.  Events are taken
// from a pool; prof_flush() waits for the recorded events and folds them into the
// per-class totals.
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace bmg {
namespace {

struct Pending {
  int cls;
  cudaEvent_t e0, e1;
  double bytes, flops;
};

struct Totals {
  double ms = 0.0, bytes = 0.0, flops = 0.0;
  long long launches = 0;
};

// Pools and totals are shared (guarded by mu); the open bracket of a launch belongs
// to the host thread that issued it, so concurrent solves on several threads (the
// batched entry point) time their own launches.
struct Profiler {
  std::mutex mu;
  std::atomic<bool> enabled{false};
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  Totals tot[KC_COUNT];

  cudaEvent_t get() {  // with mu held
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    check_cuda(cudaEventCreate(&e), "cudaEventCreate");
    return e;
  }
};

Profiler& prof() {
  static Profiler p;
  return p;
}

std::atomic<long long> g_launches{0};
thread_local cudaEvent_t t_open = nullptr;
thread_local int t_open_cls = -1;

const char* kNames[KC_COUNT] = {"spmm_am", "smooth_sweep", "residual", "transfer",
                                "gram", "dense_eig", "expand", "small"};
}  // namespace

long long launch_count() { return g_launches.load(); }
bool prof_enabled() { return prof().enabled; }
void count_launch() { g_launches.fetch_add(1); }
void count_launches(long long n) { g_launches.fetch_add(n); }

void prof_begin(int cls, cudaStream_t s) {
  Profiler& p = prof();
  if (!p.enabled) return;
  {
    std::lock_guard<std::mutex> lock(p.mu);
    t_open = p.get();
  }
  t_open_cls = cls;
  check_cuda(cudaEventRecord(t_open, s), "cudaEventRecord");
}

void prof_end(int cls, cudaStream_t s, double bytes, double flops) {
  Profiler& p = prof();
  if (!p.enabled || !t_open || t_open_cls != cls) return;
  cudaEvent_t e1;
  {
    std::lock_guard<std::mutex> lock(p.mu);
    e1 = p.get();
  }
  check_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
  {
    std::lock_guard<std::mutex> lock(p.mu);
    p.pending.push_back({cls, t_open, e1, bytes, flops});
  }
  t_open = nullptr;
  t_open_cls = -1;
}

void prof_flush() {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lock(p.mu);
  for (const Pending& q : p.pending) {
    check_cuda(cudaEventSynchronize(q.e1), "cudaEventSynchronize");
    float ms = 0.f;
    check_cuda(cudaEventElapsedTime(&ms, q.e0, q.e1), "cudaEventElapsedTime");
    Totals& t = p.tot[q.cls];
    t.ms += ms;
    t.bytes += q.bytes;
    t.flops += q.flops;
    t.launches += 1;
    p.pool.push_back(q.e0);
    p.pool.push_back(q.e1);
  }
  p.pending.clear();
}

}  // namespace bmg

using namespace bmg;

extern "C" bmg_status bmg_profile_enable(int enable) {
  try {
    Profiler& p = prof();
    prof_flush();
    p.enabled = enable != 0;
    return BMG_OK;
  } catch (...) {
    set_error("profiler: CUDA event failure");
    return BMG_ERR_CUDA;
  }
}

extern "C" bmg_status bmg_profile_reset(void) {
  try {
    Profiler& p = prof();
    prof_flush();
    std::lock_guard<std::mutex> lock(p.mu);
    for (auto& t : p.tot) t = Totals();
    return BMG_OK;
  } catch (...) {
    set_error("profiler: CUDA event failure");
    return BMG_ERR_CUDA;
  }
}

extern "C" bmg_status bmg_profile_read(int cls, double* total_ms, long long* launches, double* bytes,
                                       double* flops) {
  if (cls < 0 || cls >= KC_COUNT) {
    set_error("profiler: class out of range");
    return BMG_ERR_INVALID_ARG;
  }
  try {
    prof_flush();
  } catch (...) {
    set_error("profiler: CUDA event failure");
    return BMG_ERR_CUDA;
  }
  const Totals& t = prof().tot[cls];
  if (total_ms) *total_ms = t.ms;
  if (launches) *launches = t.launches;
  if (bytes) *bytes = t.bytes;
  if (flops) *flops = t.flops;
  return BMG_OK;
}

extern "C" const char* bmg_kernel_class_name(int cls) {
  return (cls >= 0 && cls < KC_COUNT) ? kNames[cls] : "";
}

extern "C" long long bmg_launch_count(void) { return launch_count(); }
