// C ABI of the rank-predictor MLP (create / train / forward / gradient).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/h2ulv.h"
#include "h2_common.cuh"
#include "h2_mlp.h"

namespace h2 {

void box_features(int n, const double* lo, const double* hi, int n_near, int n_far, int height, int n_samples,
                  float* out) {
  double e[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  std::sort(e, e + 3, [](double a, double b) { return a > b; });
  const double e0 = e[0] > 0 ? e[0] : 1.0;
  out[0] = (float)(n / 256.0);
  out[1] = (float)(e[1] / e0);
  out[2] = (float)(e[2] / e0);
  out[3] = (float)(height / 8.0);
  out[4] = (float)(n_near / 64.0);
  out[5] = (float)(n_far / 64.0);
  out[6] = (float)(std::log2(1.0 + n_samples) / 12.0);
  out[7] = (float)(std::log2(1.0 + (double)n) / 8.0);
}

}  // namespace h2

using namespace h2;

struct h2_mlp_ {
  Mlp m;
};

namespace {
thread_local std::string g_mlp_err;

bool is_dev(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class F> h2_status mlp_guard(F&& f) {
  try {
    f();
    return H2_OK;
  } catch (const StatusError& e) {
    g_mlp_err = e.what();
    return (h2_status)e.status;
  } catch (const std::exception& e) {
    g_mlp_err = e.what();
    return H2_ERR_DEVICE;
  }
}

// device copy of a caller array (host or device)
struct DevArr {
  float* p = nullptr;
  bool own = false;
  DevArr(const float* src, size_t n, cudaStream_t s) {
    if (is_dev(src)) {
      p = const_cast<float*>(src);
    } else {
      H2_CUDA(cudaMalloc(&p, std::max<size_t>(n, 1) * 4));
      own = true;
      H2_CUDA(cudaMemcpyAsync(p, src, n * 4, cudaMemcpyHostToDevice, s));
    }
  }
  ~DevArr() {
    if (own) cudaFree(p);
  }
};

struct Work {
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *gpart = nullptr, *loss = nullptr;
  Work(int B, int P, cudaStream_t) {
    const int nblk = (B + 255) / 256;
    H2_CUDA(cudaMalloc(&H1, (size_t)B * MLP_WIDTH * 4));
    H2_CUDA(cudaMalloc(&H2, (size_t)B * MLP_WIDTH * 4));
    H2_CUDA(cudaMalloc(&Y, (size_t)B * 4));
    H2_CUDA(cudaMalloc(&gpart, (size_t)nblk * P * 4));
    H2_CUDA(cudaMalloc(&loss, (size_t)nblk * 4));
  }
  ~Work() {
    cudaFree(H1);
    cudaFree(H2);
    cudaFree(Y);
    cudaFree(gpart);
    cudaFree(loss);
  }
};
}  // namespace

extern "C" {

int32_t h2_mlp_param_count(int32_t n_features) { return n_features > 0 ? mlp_param_count(n_features) : 0; }

h2_status h2_mlp_create(int32_t n_features, const float* init_params, void* stream, h2_mlp* out) {
  if (!out || !init_params || n_features != MLP_FEATURES) {
    g_mlp_err = "h2_mlp_create: n_features must be 8 and init_params non-null";
    return H2_ERR_ARG;
  }
  *out = nullptr;
  auto* M = new h2_mlp_();
  h2_status st = mlp_guard([&] {
    Mlp& m = M->m;
    m.F = n_features;
    m.P = mlp_param_count(m.F);
    m.s = (cudaStream_t)stream;
    H2_CUDA(cudaMalloc(&m.prm, (size_t)m.P * 4));
    H2_CUDA(cudaMalloc(&m.m1, (size_t)m.P * 4));
    H2_CUDA(cudaMalloc(&m.m2, (size_t)m.P * 4));
    H2_CUDA(cudaMalloc(&m.grad, (size_t)m.P * 4));
    H2_CUDA(cudaMemsetAsync(m.m1, 0, (size_t)m.P * 4, m.s));
    H2_CUDA(cudaMemsetAsync(m.m2, 0, (size_t)m.P * 4, m.s));
    H2_CUDA(cudaMemcpyAsync(m.prm, init_params, (size_t)m.P * 4,
                            is_dev(init_params) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m.s));
    H2_CUDA(cudaStreamSynchronize(m.s));
  });
  if (st != H2_OK) {
    h2_mlp_destroy(M);
    return st;
  }
  *out = M;
  return H2_OK;
}

h2_status h2_mlp_train(h2_mlp M, const float* X, const float* T, int32_t B, int32_t steps, float lr, float* loss_out) {
  if (!M || !X || !T || B < 1 || steps < 0) {
    g_mlp_err = "invalid h2_mlp_train arguments";
    return H2_ERR_ARG;
  }
  return mlp_guard([&] {
    Mlp& m = M->m;
    DevArr dx(X, (size_t)B * m.F, m.s), dt(T, (size_t)B, m.s);
    Work w(B, m.P, m.s);
    const int nblk = (B + 255) / 256;
    for (int k = 0; k < steps; ++k) {
      mlp_forward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, dt.p, w.loss, m.s);
      mlp_backward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, dt.p, w.gpart, m.s);
      ++m.step;
      mlp_reduce_adam(w.gpart, nblk, m.F, m.grad, m.prm, m.m1, m.m2, lr, m.step, true, m.s);
    }
    // final loss (mean squared error) with the trained parameters
    mlp_forward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, dt.p, w.loss, m.s);
    std::vector<float> lp(nblk);
    H2_CUDA(cudaMemcpyAsync(lp.data(), w.loss, nblk * 4, cudaMemcpyDeviceToHost, m.s));
    H2_CUDA(cudaStreamSynchronize(m.s));
    double t = 0;
    for (float v : lp) t += v;
    if (loss_out) *loss_out = (float)(t / B);
  });
}

h2_status h2_mlp_forward(h2_mlp M, const float* X, int32_t B, float* Y) {
  if (!M || !X || !Y || B < 1) {
    g_mlp_err = "invalid h2_mlp_forward arguments";
    return H2_ERR_ARG;
  }
  return mlp_guard([&] {
    Mlp& m = M->m;
    DevArr dx(X, (size_t)B * m.F, m.s);
    Work w(B, m.P, m.s);
    mlp_forward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, nullptr, nullptr, m.s);
    H2_CUDA(cudaMemcpyAsync(Y, w.Y, (size_t)B * 4, is_dev(Y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m.s));
    H2_CUDA(cudaStreamSynchronize(m.s));
  });
}

h2_status h2_mlp_gradient(h2_mlp M, const float* X, const float* T, int32_t B, float* grad, float* loss) {
  if (!M || !X || !T || !grad || B < 1) {
    g_mlp_err = "invalid h2_mlp_gradient arguments";
    return H2_ERR_ARG;
  }
  return mlp_guard([&] {
    Mlp& m = M->m;
    DevArr dx(X, (size_t)B * m.F, m.s), dt(T, (size_t)B, m.s);
    Work w(B, m.P, m.s);
    const int nblk = (B + 255) / 256;
    mlp_forward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, dt.p, w.loss, m.s);
    mlp_backward(m.prm, m.F, dx.p, B, w.H1, w.H2, w.Y, dt.p, w.gpart, m.s);
    mlp_reduce_adam(w.gpart, nblk, m.F, m.grad, m.prm, m.m1, m.m2, 0.f, 1, false, m.s);
    H2_CUDA(cudaMemcpyAsync(grad, m.grad, (size_t)m.P * 4,
                            is_dev(grad) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m.s));
    std::vector<float> lp(nblk);
    H2_CUDA(cudaMemcpyAsync(lp.data(), w.loss, nblk * 4, cudaMemcpyDeviceToHost, m.s));
    H2_CUDA(cudaStreamSynchronize(m.s));
    double t = 0;
    for (float v : lp) t += v;
    if (loss) *loss = (float)(t / B);
  });
}

h2_status h2_mlp_params(h2_mlp M, float* out) {
  if (!M || !out) {
    g_mlp_err = "invalid h2_mlp_params arguments";
    return H2_ERR_ARG;
  }
  return mlp_guard([&] {
    Mlp& m = M->m;
    H2_CUDA(cudaMemcpyAsync(out, m.prm, (size_t)m.P * 4, is_dev(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                            m.s));
    H2_CUDA(cudaStreamSynchronize(m.s));
  });
}

const char* h2_mlp_last_error(void) { return g_mlp_err.c_str(); }

void h2_mlp_destroy(h2_mlp M) {
  if (!M) return;
  Mlp& m = M->m;
  if (m.prm) cudaFree(m.prm);
  if (m.m1) cudaFree(m.m1);
  if (m.m2) cudaFree(m.m2);
  if (m.grad) cudaFree(m.grad);
  delete M;
}

}  // extern "C"
