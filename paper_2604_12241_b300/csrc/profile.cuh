// Launch accounting / CUDA-event timing scope (see profile.cu).
#pragma once

#include "aml_internal.cuh"

namespace aml {

class LaunchScope {
 public:
  LaunchScope(const char* name, cudaStream_t s);
  ~LaunchScope();
  LaunchScope(const LaunchScope&) = delete;
  LaunchScope& operator=(const LaunchScope&) = delete;

 private:
  const char* name_;
  cudaStream_t s_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
  bool active_ = false;
};

long long launch_count();
bool profiling_enabled();  // aml_profile_enable is on
void add_launches(long long n);  // kernels launched through a replayed CUDA graph

}  // namespace aml

// Launch a kernel through the accounting scope and check the launch.
#define AML_LAUNCH(name, stream, ...)               \
  do {                                              \
    ::aml::LaunchScope _aml_ls((name), (stream));   \
    __VA_ARGS__;                                    \
    AML_CUDA(cudaGetLastError());                   \
  } while (0)
