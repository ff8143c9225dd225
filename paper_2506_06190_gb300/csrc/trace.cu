// Launch counting and optional per-launch CUDA-event timing (tracing for benchmarks).
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace natbem {

namespace {
std::atomic<int64_t> g_launches{0};
thread_local int64_t t_launches = 0;  // this thread's launches (graph capture is per thread)
std::atomic<int> g_trace{0};
std::mutex g_mu;
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
std::vector<std::string> g_select;  // empty: trace every kernel

bool selected(const char* name) {
  if (g_select.empty()) return true;
  for (const auto& s : g_select)
    if (std::string(name).find(s) != std::string::npos) return true;
  return false;
}

cudaEvent_t get_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

TraceScope::TraceScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
  if (g_trace.load(std::memory_order_relaxed)) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!selected(name)) return;
    a_ = get_event();
    b_ = get_event();
    cudaEventRecord((cudaEvent_t)a_, s_);
  }
}

TraceScope::~TraceScope() {
  if (a_) {
    cudaEventRecord((cudaEvent_t)b_, s_);
    std::lock_guard<std::mutex> lk(g_mu);
    g_recs.push_back({name_, (cudaEvent_t)a_, (cudaEvent_t)b_});
  }
}

bool tracing_enabled() { return g_trace.load(std::memory_order_relaxed) != 0; }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }
int64_t thread_launch_count() { return t_launches; }
void add_launches(int64_t n) {
  g_launches.fetch_add(n, std::memory_order_relaxed);
  t_launches += n;
}

}  // namespace natbem

using namespace natbem;

extern "C" {

void nat_bem_trace_enable(int32_t enable) { g_trace.store(enable ? 1 : 0); }

void nat_bem_trace_select(const char* names) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_select.clear();
  if (!names) return;
  std::string all(names), cur;
  for (char ch : all) {
    if (ch == ',') {
      if (!cur.empty()) g_select.push_back(cur);
      cur.clear();
    } else {
      cur.push_back(ch);
    }
  }
  if (!cur.empty()) g_select.push_back(cur);
}

void nat_bem_trace_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    cudaEventSynchronize(r.b);
    g_free.push_back(r.a);
    g_free.push_back(r.b);
  }
  g_recs.clear();
  g_launches.store(0);
}

int64_t nat_bem_trace_launches(void) { return g_launches.load(); }

nat_bem_status nat_bem_trace_kernel(const char* name, double* total_ms, int64_t* launches) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_mu);
  double t = 0.0;
  int64_t c = 0;
  const std::string want = name ? name : "";
  for (auto& r : g_recs) {
    if (!want.empty() && std::string(r.name).find(want) == std::string::npos) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      set_error(std::string("trace: ") + cudaGetErrorString(e));
      return NAT_BEM_ECUDA;
    }
    t += ms;
    ++c;
  }
  if (total_ms) *total_ms = t;
  if (launches) *launches = c;
  return NAT_BEM_OK;
}

nat_bem_status nat_bem_trace_durations(const char* name, float* out_ms, int64_t cap, int64_t* count) {
  clear_error();
  if (!name || (cap > 0 && !out_ms) || cap < 0) {
    set_error("nat_bem_trace_durations: bad arguments");
    return NAT_BEM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int64_t c = 0;
  for (auto& r : g_recs) {
    if (std::string(r.name) != name) continue;
    cudaError_t e = cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      set_error(std::string("trace: ") + cudaGetErrorString(e));
      return NAT_BEM_ECUDA;
    }
    if (c < cap) out_ms[c] = ms;
    ++c;
  }
  if (count) *count = c;
  return NAT_BEM_OK;
}

}  // extern "C"
