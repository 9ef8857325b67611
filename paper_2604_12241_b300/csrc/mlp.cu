// Cost model: a 16 -> 64 -> 64 -> 1 ReLU perceptron that predicts the log of
// an anchor edge's cycle-search cost (clock64 cycles) from 16 cheap features.
//
// Parameters (fp32 master copy, trained with Adam), in this order:
//   W1 [64][16], b1 [64], W2 [64][64], b2 [64], w3 [64], b3 [1]   (5313 floats)
// The forward pass uses the weights rounded to bf16 and accumulates in fp32:
//   inference on tensor cores (mma.sync m16n8k16, bf16 x bf16 -> fp32), 16
//   items per warp, activations rounded to bf16 between layers;
//   training on CUDA cores in fp32 with the same bf16-rounded weights.
// Loss: mean squared error of the prediction against the (normalized) label.
#include <cuda_bf16.h>

#include <cstring>

#include "aml_internal.cuh"
#include "mlp.cuh"
#include "profile.cuh"

namespace aml {

// ------------------------------------------------------------- training

constexpr int TR_TILE = 64;      // samples per tile (one per thread of a 64-thread group)
constexpr int TR_THREADS = 128;  // threads per block
constexpr int XS = MLP_IN + 1;   // padded row strides of the per-sample tiles
constexpr int HS = MLP_H + 1;

__device__ __forceinline__ float bf16r(float x) {
  return __bfloat162float(__float2bfloat16(x));
}

// Per-sample forward/backward of a tile of samples into shared memory, then
// the parameter gradients as dot products over the tile's samples.  Block b
// takes tiles b, b + grid, ... and writes its partial sums to part[b] (the
// MLP_NPARAM gradient entries, then its squared error); k_mlp_reduce adds
// the blocks' partials in block order, so a gradient is the same bit for
// bit on every run (no floating-point atomics).
__global__ void __launch_bounds__(TR_THREADS) k_mlp_grad(const float* __restrict__ params,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ y, int64_t n,
                                                         float scale, float* __restrict__ part) {
  extern __shared__ float sm[];
  float* w = sm;                              // bf16-rounded parameters [MLP_NPARAM]
  float* sx = w + MLP_NPARAM;                 // [TR_TILE][XS]
  float* sh1 = sx + TR_TILE * XS;             // [TR_TILE][HS] activations
  float* sd1 = sh1 + TR_TILE * HS;            // [TR_TILE][HS] d(pre-activation 1)
  float* sh2 = sd1 + TR_TILE * HS;            // [TR_TILE][HS]
  float* sd2 = sh2 + TR_TILE * HS;            // [TR_TILE][HS] d(pre-activation 2)
  float* sdy = sd2 + TR_TILE * HS;            // [TR_TILE]
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) {
    const bool bias = (i >= MLP_B1 && i < MLP_B1 + MLP_H) || (i >= MLP_B2 && i < MLP_B2 + MLP_H) ||
                      i == MLP_B3;
    w[i] = bias ? params[i] : bf16r(params[i]);
  }
  // register accumulators: thread t owns parameters t, t+T, t+2T, ...
  constexpr int PER = (MLP_NPARAM + TR_THREADS - 1) / TR_THREADS;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  float my_loss = 0.f;
  __syncthreads();
  const int64_t n_tiles = (n + TR_TILE - 1) / TR_TILE;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t s0 = tile * TR_TILE;
    const int ts = threadIdx.x;
    if (ts < TR_TILE) {
      const int64_t s = s0 + ts;
      const bool valid = s < n;
      float xi[MLP_IN];
#pragma unroll
      for (int k = 0; k < MLP_IN; ++k) {
        xi[k] = valid ? x[s * MLP_IN + k] : 0.f;
        sx[ts * XS + k] = xi[k];
      }
      for (int j = 0; j < MLP_H; ++j) {
        float a = w[MLP_B1 + j];
#pragma unroll
        for (int k = 0; k < MLP_IN; ++k) a += w[MLP_W1 + j * MLP_IN + k] * xi[k];
        sh1[ts * HS + j] = a > 0.f ? a : 0.f;
      }
      float out = w[MLP_B3];
      for (int j = 0; j < MLP_H; ++j) {
        float a = w[MLP_B2 + j];
        for (int i = 0; i < MLP_H; ++i) a += w[MLP_W2 + j * MLP_H + i] * sh1[ts * HS + i];
        const float h = a > 0.f ? a : 0.f;
        sh2[ts * HS + j] = h;
        out += w[MLP_W3 + j] * h;
      }
      const float diff = valid ? out - y[s] : 0.f;
      my_loss += diff * diff;
      const float dy = scale * 2.f * diff;   // d(scale * sum diff^2)/d out
      sdy[ts] = dy;
      for (int j = 0; j < MLP_H; ++j)
        sd2[ts * HS + j] = sh2[ts * HS + j] > 0.f ? dy * w[MLP_W3 + j] : 0.f;
      for (int i = 0; i < MLP_H; ++i) {
        float a = 0.f;
        for (int j = 0; j < MLP_H; ++j) a += sd2[ts * HS + j] * w[MLP_W2 + j * MLP_H + i];
        sd1[ts * HS + i] = sh1[ts * HS + i] > 0.f ? a : 0.f;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int p = threadIdx.x + k * TR_THREADS;
      if (p >= MLP_NPARAM) break;
      float g = 0.f;
      if (p < MLP_B1) {                       // W1[j][i]
        const int j = p / MLP_IN, i = p % MLP_IN;
        for (int s = 0; s < TR_TILE; ++s) g += sd1[s * HS + j] * sx[s * XS + i];
      } else if (p < MLP_W2) {                // b1[j]
        const int j = p - MLP_B1;
        for (int s = 0; s < TR_TILE; ++s) g += sd1[s * HS + j];
      } else if (p < MLP_B2) {                // W2[j][i]
        const int q = p - MLP_W2, j = q / MLP_H, i = q % MLP_H;
        for (int s = 0; s < TR_TILE; ++s) g += sd2[s * HS + j] * sh1[s * HS + i];
      } else if (p < MLP_W3) {                // b2[j]
        const int j = p - MLP_B2;
        for (int s = 0; s < TR_TILE; ++s) g += sd2[s * HS + j];
      } else if (p < MLP_B3) {                // w3[j]
        const int j = p - MLP_W3;
        for (int s = 0; s < TR_TILE; ++s) g += sdy[s] * sh2[s * HS + j];
      } else {                                // b3
        for (int s = 0; s < TR_TILE; ++s) g += sdy[s];
      }
      acc[k] += g;
    }
    __syncthreads();
  }
  float* mine = part + (int64_t)blockIdx.x * (MLP_NPARAM + 1);
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int p = threadIdx.x + k * TR_THREADS;
    if (p < MLP_NPARAM) mine[p] = acc[k];
  }
  // the block's squared error, summed in thread order
  sx[threadIdx.x] = threadIdx.x < TR_TILE ? my_loss : 0.f;
  __syncthreads();
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int t = 0; t < TR_TILE; ++t) l += sx[t];
    mine[MLP_NPARAM] = l;
  }
}

// grad[p] = sum over blocks b (in order) of part[b][p]; loss likewise
__global__ void k_mlp_reduce(const float* __restrict__ part, int blocks,
                             float* __restrict__ grad, float* __restrict__ loss_sum) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > MLP_NPARAM) return;
  float s = 0.f;
  for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * (MLP_NPARAM + 1) + p];
  if (p < MLP_NPARAM) grad[p] = s;
  else *loss_sum = s;
}

// Adam (Kingma & Ba) on the fp32 master parameters.
__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g,
                           float* __restrict__ m, float* __restrict__ v, int n, float lr,
                           float b1, float b2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

size_t mlp_grad_smem() {
  return sizeof(float) * (MLP_NPARAM + TR_TILE * XS + 4 * TR_TILE * HS + TR_TILE);
}

void mlp_grad(const float* params, const float* x, const float* y, int64_t n, float scale,
              float* grad, float* loss_sum, cudaStream_t s) {
  static bool attr[64] = {false};
  int dev = 0;
  AML_CUDA(cudaGetDevice(&dev));
  if (dev >= 64 || !attr[dev]) {
    AML_CUDA(cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)mlp_grad_smem()));
    if (dev < 64) attr[dev] = true;
  }
  const int64_t tiles = (n + TR_TILE - 1) / TR_TILE;
  const unsigned blocks = (unsigned)std::min<int64_t>(std::max<int64_t>(tiles, 1), 296);
  DBuf<float> part((size_t)blocks * (MLP_NPARAM + 1), s);
  AML_LAUNCH("k_mlp_grad", s,
             k_mlp_grad<<<blocks, TR_THREADS, mlp_grad_smem(), s>>>(params, x, y, n, scale,
                                                                   part.p));
  AML_LAUNCH("k_mlp_reduce", s,
             k_mlp_reduce<<<grid_for(MLP_NPARAM + 1, 256), 256, 0, s>>>(part.p, (int)blocks, grad,
                                                                        loss_sum));
}

void mlp_adam(float* p, const float* g, float* m, float* v, int n, int step, float lr, float b1,
              float b2, float eps, cudaStream_t s) {
  const float bc1 = 1.f - powf(b1, (float)step);
  const float bc2 = 1.f - powf(b2, (float)step);
  AML_LAUNCH("k_mlp_adam", s,
             k_mlp_adam<<<grid_for(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, bc1,
                                                          bc2));
}

// ------------------------------------------------------------- inference
//
// One warp predicts 16 items per pass with bf16 mma.sync m16n8k16 (fp32
// accumulate).  Fragment layout of m16n8k16 (g = lane / 4, c = lane % 4):
// A (16 x 16, row-major): a0 = (g, 2c..2c+1), a1 = (g+8, 2c..), a2 = (g, 2c+8..),
// a3 = (g+8, 2c+8..); B (16 x 8, k x n): b0 = (k = 2c..2c+1, n = g),
// b1 = (k = 2c+8.., n = g); C (16 x 8): c0,c1 = (g, 2c..), c2,c3 = (g+8, 2c..).

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// feat: raw features [n][16]; the model's normalization is applied here.
// out: predicted label in the model's label units (de-normalized).
__global__ void __launch_bounds__(256) k_mlp_infer(MlpDevice M, const float* __restrict__ feat,
                                                   int64_t n_max, const int32_t* __restrict__ n_dev,
                                                   float* __restrict__ out) {
  const int64_t n = n_dev ? min(n_max, (int64_t)*n_dev) : n_max;
  __shared__ float s_w[MLP_NPARAM];
  for (int i = threadIdx.x; i < MLP_NPARAM; i += blockDim.x) s_w[i] = M.params[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, c = lane & 3;
  // B fragments of layer 1 (k = input feature, n = hidden unit) and layer 2
  uint32_t w1b[8][2], w2b[4][8][2];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int hn = nt * 8 + g;
    w1b[nt][0] =
        pack_bf16(s_w[MLP_W1 + hn * MLP_IN + 2 * c], s_w[MLP_W1 + hn * MLP_IN + 2 * c + 1]);
    w1b[nt][1] = pack_bf16(s_w[MLP_W1 + hn * MLP_IN + 2 * c + 8],
                           s_w[MLP_W1 + hn * MLP_IN + 2 * c + 9]);
  }
#pragma unroll
  for (int kt = 0; kt < 4; ++kt)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int hn = nt * 8 + g, k0 = kt * 16 + 2 * c;
      w2b[kt][nt][0] = pack_bf16(s_w[MLP_W2 + hn * MLP_H + k0], s_w[MLP_W2 + hn * MLP_H + k0 + 1]);
      w2b[kt][nt][1] =
          pack_bf16(s_w[MLP_W2 + hn * MLP_H + k0 + 8], s_w[MLP_W2 + hn * MLP_H + k0 + 9]);
    }
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t0 = warp * 16; t0 < n; t0 += n_warps * 16) {
    // A fragment of the 16 items' normalized features
    const int64_t r0 = t0 + g, r1 = t0 + g + 8;
    auto fv = [&](int64_t r, int k) -> float {
      return r < n ? (feat[r * MLP_IN + k] - M.mean[k]) * M.inv_std[k] : 0.f;
    };
    uint32_t a[4] = {pack_bf16(fv(r0, 2 * c), fv(r0, 2 * c + 1)),
                     pack_bf16(fv(r1, 2 * c), fv(r1, 2 * c + 1)),
                     pack_bf16(fv(r0, 2 * c + 8), fv(r0, 2 * c + 9)),
                     pack_bf16(fv(r1, 2 * c + 8), fv(r1, 2 * c + 9))};
    float h1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float bl = s_w[MLP_B1 + nt * 8 + 2 * c], bh = s_w[MLP_B1 + nt * 8 + 2 * c + 1];
      h1[nt][0] = bl;
      h1[nt][1] = bh;
      h1[nt][2] = bl;
      h1[nt][3] = bh;
      mma_bf16(h1[nt], a, w1b[nt][0], w1b[nt][1]);
#pragma unroll
      for (int q = 0; q < 4; ++q) h1[nt][q] = fmaxf(h1[nt][q], 0.f);
    }
    float h2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float bl = s_w[MLP_B2 + nt * 8 + 2 * c], bh = s_w[MLP_B2 + nt * 8 + 2 * c + 1];
      h2[nt][0] = bl;
      h2[nt][1] = bh;
      h2[nt][2] = bl;
      h2[nt][3] = bh;
    }
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
      // C fragments of hidden tiles 2kt, 2kt+1 are the A fragment of k-step kt
      const uint32_t a2[4] = {pack_bf16(h1[2 * kt][0], h1[2 * kt][1]),
                              pack_bf16(h1[2 * kt][2], h1[2 * kt][3]),
                              pack_bf16(h1[2 * kt + 1][0], h1[2 * kt + 1][1]),
                              pack_bf16(h1[2 * kt + 1][2], h1[2 * kt + 1][3])};
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) mma_bf16(h2[nt], a2, w2b[kt][nt][0], w2b[kt][nt][1]);
    }
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float wl = __bfloat162float(__float2bfloat16(s_w[MLP_W3 + nt * 8 + 2 * c]));
      const float wh = __bfloat162float(__float2bfloat16(s_w[MLP_W3 + nt * 8 + 2 * c + 1]));
      y0 += fmaxf(h2[nt][0], 0.f) * wl + fmaxf(h2[nt][1], 0.f) * wh;
      y1 += fmaxf(h2[nt][2], 0.f) * wl + fmaxf(h2[nt][3], 0.f) * wh;
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (c == 0) {
      if (r0 < n) out[r0] = (y0 + s_w[MLP_B3]) * M.y_std + M.y_mean;
      if (r1 < n) out[r1] = (y1 + s_w[MLP_B3]) * M.y_std + M.y_mean;
    }
  }
}

void mlp_infer(const MlpDevice& M, const float* feat, int64_t n, float* out, cudaStream_t s,
               const int32_t* n_dev) {
  if (n <= 0) return;
  const int64_t warps = (n + 15) / 16;
  const unsigned blocks = (unsigned)std::min<int64_t>((warps + 7) / 8, 148 * 8);
  AML_LAUNCH("k_mlp_infer", s, k_mlp_infer<<<blocks, 256, 0, s>>>(M, feat, n, n_dev, out));
}

}  // namespace aml

using namespace aml;

extern "C" {

aml_status aml_mlp_loss_grad(const float* params, const float* x, const float* y, int64_t n,
                             float* grad, float* loss) {
  try {
    AML_REQUIRE(params && x && y && grad && loss && n > 0, AML_EINVAL, "bad argument");
    cudaStream_t s = nullptr;
    DBuf<float> dp(MLP_NPARAM, s), dx((size_t)n * MLP_IN, s), dy((size_t)n, s),
        dg(MLP_NPARAM, s), dl(1, s);
    AML_CUDA(cudaMemcpyAsync(dp.p, params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dx.p, x, n * MLP_IN * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dy.p, y, n * 4, cudaMemcpyHostToDevice, s));
    mlp_grad(dp.p, dx.p, dy.p, n, 1.0f / (float)n, dg.p, dl.p, s);
    AML_CUDA(cudaMemcpyAsync(grad, dg.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaMemcpyAsync(loss, dl.p, 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaStreamSynchronize(s));
    *loss /= (float)n;
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_mlp_loss_grad: ") + f.msg);
    return f.status;
  }
}

aml_status aml_mlp_adam_step(float* params, const float* grad, float* m, float* v, int32_t step,
                             float lr, float beta1, float beta2, float eps) {
  try {
    AML_REQUIRE(params && grad && m && v && step >= 1, AML_EINVAL, "bad argument");
    cudaStream_t s = nullptr;
    DBuf<float> dp(MLP_NPARAM, s), dg(MLP_NPARAM, s), dm(MLP_NPARAM, s), dv(MLP_NPARAM, s);
    AML_CUDA(cudaMemcpyAsync(dp.p, params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dg.p, grad, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dm.p, m, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dv.p, v, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    mlp_adam(dp.p, dg.p, dm.p, dv.p, MLP_NPARAM, step, lr, beta1, beta2, eps, s);
    AML_CUDA(cudaMemcpyAsync(params, dp.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaMemcpyAsync(m, dm.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaMemcpyAsync(v, dv.p, MLP_NPARAM * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaStreamSynchronize(s));
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_mlp_adam_step: ") + f.msg);
    return f.status;
  }
}

aml_status aml_mlp_predict(const float* params, const float* norm, const float* feat, int64_t n,
                           float* out) {
  try {
    AML_REQUIRE(params && norm && feat && out && n > 0, AML_EINVAL, "bad argument");
    cudaStream_t s = nullptr;
    DBuf<float> dp(MLP_NPARAM, s), dx((size_t)n * MLP_IN, s), dout((size_t)n, s);
    AML_CUDA(cudaMemcpyAsync(dp.p, params, MLP_NPARAM * 4, cudaMemcpyHostToDevice, s));
    AML_CUDA(cudaMemcpyAsync(dx.p, feat, n * MLP_IN * 4, cudaMemcpyHostToDevice, s));
    MlpDevice M;
    M.params = dp.p;
    for (int k = 0; k < MLP_IN; ++k) {
      M.mean[k] = norm[k];
      M.inv_std[k] = norm[MLP_IN + k];
    }
    M.y_mean = norm[2 * MLP_IN];
    M.y_std = norm[2 * MLP_IN + 1];
    mlp_infer(M, dx.p, n, dout.p, s);
    AML_CUDA(cudaMemcpyAsync(out, dout.p, n * 4, cudaMemcpyDeviceToHost, s));
    AML_CUDA(cudaStreamSynchronize(s));
    return AML_OK;
  } catch (const Failure& f) {
    set_error(std::string("aml_mlp_predict: ") + f.msg);
    return f.status;
  }
}

}  // extern "C"
