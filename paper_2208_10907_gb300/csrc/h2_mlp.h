// Rank-predictor MLP: kernels (k_mlp.cu) and the host object behind the
// h2_mlp_* entry points.
#pragma once
#include <cuda_runtime.h>

#include <vector>

namespace h2 {

constexpr int MLP_WIDTH = 64;
constexpr int MLP_FEATURES = 8;

int mlp_param_count(int F);
void mlp_forward(const float* prm, int F, const float* X, int B, float* H1, float* H2, float* Y, const float* T,
                 float* loss_part, cudaStream_t s);
void mlp_backward(const float* prm, int F, const float* X, int B, const float* H1, const float* H2, const float* Y,
                  const float* T, float* gpart, cudaStream_t s);
void mlp_reduce_adam(const float* gpart, int nblk, int F, float* grad, float* prm, float* m1, float* m2, float lr,
                     int step, bool update, cudaStream_t s);

// Device state of one predictor.
struct Mlp {
  int F = MLP_FEATURES;
  int P = 0;
  int step = 0;
  float* prm = nullptr;   // parameters
  float* m1 = nullptr;    // Adam moments
  float* m2 = nullptr;
  float* grad = nullptr;
  cudaStream_t s = nullptr;
};

// Features of one box for the predictor (host side, also used when the
// factorization asks for predicted ranks).
void box_features(int n, const double* lo, const double* hi, int n_near, int n_far, int height, int n_samples,
                  float* out);

}  // namespace h2
