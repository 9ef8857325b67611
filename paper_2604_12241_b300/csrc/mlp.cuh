// Cost-model perceptron (see mlp.cu): layout and entry points.
#pragma once

#include "aml_internal.cuh"

namespace aml {

constexpr int MLP_IN = 16;
constexpr int MLP_H = 64;
constexpr int MLP_W1 = 0;                       // [64][16]
constexpr int MLP_B1 = MLP_W1 + MLP_H * MLP_IN;  // [64]
constexpr int MLP_W2 = MLP_B1 + MLP_H;           // [64][64]
constexpr int MLP_B2 = MLP_W2 + MLP_H * MLP_H;   // [64]
constexpr int MLP_W3 = MLP_B2 + MLP_H;           // [64]
constexpr int MLP_B3 = MLP_W3 + MLP_H;           // [1]
constexpr int MLP_NPARAM = MLP_B3 + 1;           // 5313

// Device model for inference: parameters plus input / label normalization.
struct MlpDevice {
  const float* params;   // fp32 master parameters (rounded to bf16 on load)
  float mean[MLP_IN];
  float inv_std[MLP_IN];
  float y_mean, y_std;
};

inline MlpDevice device_of(const CostModel& c) {
  MlpDevice M;
  M.params = c.params;
  for (int k = 0; k < MLP_IN; ++k) {
    M.mean[k] = c.mean[k];
    M.inv_std[k] = c.inv_std[k];
  }
  M.y_mean = c.y_mean;
  M.y_std = c.y_std;
  return M;
}

size_t mlp_grad_smem();
// grad = d(scale * sum_i (f(x_i) - y_i)^2)/d params; loss_sum = sum of squares
void mlp_grad(const float* params, const float* x, const float* y, int64_t n, float scale,
              float* grad, float* loss_sum, cudaStream_t s);
void mlp_adam(float* p, const float* g, float* m, float* v, int n, int step, float lr, float b1,
              float b2, float eps, cudaStream_t s);
// rows [0, min(n, *n_dev)) when n_dev is given, else [0, n)
void mlp_infer(const MlpDevice& M, const float* feat, int64_t n, float* out, cudaStream_t s,
               const int32_t* n_dev = nullptr);

}  // namespace aml
