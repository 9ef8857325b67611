// Launch accounting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through LaunchScope: it counts the
// launch and, while profiling is enabled, records a pair of CUDA events
// around it on the launching stream.  aml_profile_read() waits for the
// recorded events and accumulates elapsed time per kernel name.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "aml_internal.cuh"
#include "profile.cuh"

namespace aml {

namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_enabled{false};
std::mutex g_mu;
struct Pending {
  const char* name;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
struct Stat {
  long long launches = 0;
  double ms = 0.0;
};
std::map<std::string, Stat> g_stats;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  AML_CUDA(cudaEventCreate(&e));
  return e;
}
}  // namespace

LaunchScope::LaunchScope(const char* name, cudaStream_t s) : name_(name), s_(s) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (g_enabled.load(std::memory_order_relaxed)) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cs);
    if (cs != cudaStreamCaptureStatusNone) return;  // no timing inside graph capture
    std::lock_guard<std::mutex> lk(g_mu);
    a_ = get_event();
    b_ = get_event();
    AML_CUDA(cudaEventRecord(a_, s));
    active_ = true;
  }
}

LaunchScope::~LaunchScope() {
  if (!active_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cudaEventRecord(b_, s_) == cudaSuccess) g_pending.push_back({name_, a_, b_});
}

bool profiling_enabled() { return g_enabled.load(std::memory_order_relaxed); }

long long launch_count() { return g_launches.load(); }

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace aml

using namespace aml;

extern "C" {

aml_status aml_launch_count(int64_t* out) {
  if (!out) {
    set_error("aml_launch_count: out is NULL");
    return AML_EINVAL;
  }
  *out = (int64_t)launch_count();
  return AML_OK;
}

aml_status aml_profile_enable(int32_t on) {
  g_enabled.store(on != 0);
  return AML_OK;
}

aml_status aml_profile_read(aml_kernel_stat* stats, int32_t cap, int32_t* n_out, int32_t reset) {
  try {
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Pending& p : g_pending) {
      AML_CUDA(cudaEventSynchronize(p.b));
      float ms = 0.f;
      AML_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
      Stat& st = g_stats[p.name];
      st.launches += 1;
      st.ms += ms;
      g_pool.push_back(p.a);
      g_pool.push_back(p.b);
    }
    g_pending.clear();
    int32_t n = 0;
    for (const auto& kv : g_stats) {
      if (stats && n < cap) {
        std::memset(&stats[n], 0, sizeof(aml_kernel_stat));
        std::strncpy(stats[n].name, kv.first.c_str(), sizeof(stats[n].name) - 1);
        stats[n].launches = kv.second.launches;
        stats[n].total_ms = kv.second.ms;
      }
      ++n;
    }
    if (n_out) *n_out = n;
    if (reset) g_stats.clear();
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_profile_read: ") + f.msg);
    return f.status;
  }
}

}  // extern "C"
