// Rank predictor: a 3-layer MLP (F -> 64 -> 64 -> 1, tanh) trained on the
// GPU with the library's own forward, backward and Adam kernels (FP32).
// Parameter vector layout: W1 (64 x F, row-major), b1 (64), W2 (64 x 64,
// row-major), b2 (64), w3 (64), b3 (1).
#include "h2_common.cuh"
#include "h2_mlp.h"
#include "h2_prof.h"

namespace h2 {

namespace {

constexpr int NT = 256;
constexpr int WID = MLP_WIDTH;

struct Off {
  int W1, b1, W2, b2, w3, b3, P;
  __host__ __device__ explicit Off(int F) {
    W1 = 0;
    b1 = W1 + WID * F;
    W2 = b1 + WID;
    b2 = W2 + WID * WID;
    w3 = b2 + WID;
    b3 = w3 + WID;
    P = b3 + 1;
  }
};

// one thread per sample: activations stored for the backward pass; squared
// errors summed per block when targets are given
__global__ void __launch_bounds__(NT) mlp_forward_kernel(const float* __restrict__ prm, int F, const float* __restrict__ X,
                                                         int B, float* __restrict__ H1, float* __restrict__ H2,
                                                         float* __restrict__ Y, const float* __restrict__ T,
                                                         float* __restrict__ loss_part) {
  extern __shared__ float sp[];
  const Off o(F);
  for (int e = threadIdx.x; e < o.P; e += NT) sp[e] = prm[e];
  __shared__ float red[32];
  __syncthreads();
  const int s = blockIdx.x * NT + threadIdx.x;
  float err = 0.f;
  if (s < B) {
    const float* x = X + (long long)s * F;
    float h1[WID];
#pragma unroll 4
    for (int j = 0; j < WID; ++j) {
      float a = sp[o.b1 + j];
      for (int f = 0; f < F; ++f) a = fmaf(sp[o.W1 + j * F + f], x[f], a);
      h1[j] = tanhf(a);
      H1[(long long)s * WID + j] = h1[j];
    }
    float y = sp[o.b3];
    for (int j = 0; j < WID; ++j) {
      float a = sp[o.b2 + j];
#pragma unroll 8
      for (int i = 0; i < WID; ++i) a = fmaf(sp[o.W2 + j * WID + i], h1[i], a);
      float h = tanhf(a);
      H2[(long long)s * WID + j] = h;
      y = fmaf(sp[o.w3 + j], h, y);
    }
    Y[s] = y;
    if (T) {
      float d = y - T[s];
      err = d * d;
    }
  }
  if (loss_part) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 16; k > 0; k >>= 1) err += __shfl_down_sync(0xffffffffu, err, k);
    if (lane == 0) red[warp] = err;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < NT / 32; ++w) t += red[w];
      loss_part[blockIdx.x] = t;
    }
  }
}

// one thread per sample: gradient of mean((y - t)^2) accumulated into a
// per-block partial gradient in shared memory
__global__ void __launch_bounds__(NT) mlp_backward_kernel(const float* __restrict__ prm, int F, const float* __restrict__ X,
                                                          int B, const float* __restrict__ H1, const float* __restrict__ H2,
                                                          const float* __restrict__ Y, const float* __restrict__ T,
                                                          float* __restrict__ gpart) {
  extern __shared__ float sm[];
  const Off o(F);
  float* sp = sm;           // parameters
  float* sg = sm + o.P;     // gradient partial
  for (int e = threadIdx.x; e < o.P; e += NT) {
    sp[e] = prm[e];
    sg[e] = 0.f;
  }
  __syncthreads();
  const int s = blockIdx.x * NT + threadIdx.x;
  if (s < B) {
    const float* x = X + (long long)s * F;
    const float* h1 = H1 + (long long)s * WID;
    const float* h2 = H2 + (long long)s * WID;
    const float dy = 2.f * (Y[s] - T[s]) / (float)B;
    atomicAdd(&sg[o.b3], dy);
    float dh1[WID];
#pragma unroll
    for (int i = 0; i < WID; ++i) dh1[i] = 0.f;
    for (int j = 0; j < WID; ++j) {
      const float hj = h2[j];
      atomicAdd(&sg[o.w3 + j], dy * hj);
      const float d2 = dy * sp[o.w3 + j] * (1.f - hj * hj);
      atomicAdd(&sg[o.b2 + j], d2);
#pragma unroll 8
      for (int i = 0; i < WID; ++i) {
        atomicAdd(&sg[o.W2 + j * WID + i], d2 * h1[i]);
        dh1[i] = fmaf(sp[o.W2 + j * WID + i], d2, dh1[i]);
      }
    }
    for (int i = 0; i < WID; ++i) {
      const float d1 = dh1[i] * (1.f - h1[i] * h1[i]);
      atomicAdd(&sg[o.b1 + i], d1);
      for (int f = 0; f < F; ++f) atomicAdd(&sg[o.W1 + i * F + f], d1 * x[f]);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < o.P; e += NT) gpart[(long long)blockIdx.x * o.P + e] = sg[e];
}

// gradient = fixed-order sum of the block partials; optional Adam step
__global__ void mlp_reduce_adam_kernel(const float* __restrict__ gpart, int nblk, int P, float* __restrict__ grad,
                                       float* __restrict__ prm, float* __restrict__ m1, float* __restrict__ m2, float lr,
                                       float b1c, float b2c, int update) {
  const int e = blockIdx.x * NT + threadIdx.x;
  if (e >= P) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += gpart[(long long)b * P + e];
  grad[e] = g;
  if (update) {
    const float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    float a = beta1 * m1[e] + (1.f - beta1) * g;
    float v = beta2 * m2[e] + (1.f - beta2) * g * g;
    m1[e] = a;
    m2[e] = v;
    prm[e] -= lr * (a / b1c) / (sqrtf(v / b2c) + eps);
  }
}

}  // namespace

int mlp_param_count(int F) { return Off(F).P; }

void mlp_forward(const float* prm, int F, const float* X, int B, float* H1, float* H2, float* Y, const float* T,
                 float* loss_part, cudaStream_t s) {
  const int nblk = (B + NT - 1) / NT;
  const size_t smem = (size_t)Off(F).P * 4;
  ProfScope ps("mlp_forward", s);
  mlp_forward_kernel<<<nblk, NT, smem, s>>>(prm, F, X, B, H1, H2, Y, T, loss_part);
  H2_LAUNCH_CHECK();
}

void mlp_backward(const float* prm, int F, const float* X, int B, const float* H1, const float* H2, const float* Y,
                  const float* T, float* gpart, cudaStream_t s) {
  const int nblk = (B + NT - 1) / NT;
  const size_t smem = (size_t)Off(F).P * 8;
  static bool attr = false;
  if (!attr) {
    H2_CUDA(cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024));
    attr = true;
  }
  ProfScope ps("mlp_backward", s);
  mlp_backward_kernel<<<nblk, NT, smem, s>>>(prm, F, X, B, H1, H2, Y, T, gpart);
  H2_LAUNCH_CHECK();
}

void mlp_reduce_adam(const float* gpart, int nblk, int F, float* grad, float* prm, float* m1, float* m2, float lr,
                     int step, bool update, cudaStream_t s) {
  const int P = Off(F).P;
  const float b1c = 1.f - powf(0.9f, (float)step), b2c = 1.f - powf(0.999f, (float)step);
  ProfScope ps(update ? "mlp_adam" : "mlp_reduce", s);
  mlp_reduce_adam_kernel<<<(P + NT - 1) / NT, NT, 0, s>>>(gpart, nblk, P, grad, prm, m1, m2, lr, b1c, b2c,
                                                          update ? 1 : 0);
  H2_LAUNCH_CHECK();
}

}  // namespace h2
