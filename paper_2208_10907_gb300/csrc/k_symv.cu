// Near-field part of the H^2 matvec over symmetric block storage: each
// stored leaf block A_IJ (I <= J) is read from HBM once and yields both
// u = A_IJ x_J (for box I) and v = A_IJ^T x_I (for box J), written to
// per-pair partial buffers; a second kernel sums each box's partials in a
// fixed order (deterministic, no atomics).
#include "h2_common.cuh"
#include "h2_prof.h"

namespace h2 {

namespace {

constexpr int NT = 256;

template <typename T, int NR>
__global__ void __launch_bounds__(NT) symv_pairs_kernel(const SymPairTask* __restrict__ tasks, const T* __restrict__ x,
                                                        long long ldx, T* __restrict__ part) {
  const SymPairTask tk = tasks[blockIdx.x];
  const int nI = tk.nI, nJ = tk.nJ;
  const T* A = reinterpret_cast<const T*>(tk.A);
  __shared__ T xI[256][NR], xJ[256][NR];
  __shared__ T uacc[8][256][NR];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < 256 * NR; e += NT) {
    int i = e % 256, c = e / 256;
    xI[i][c] = i < nI ? x[tk.sI + i + c * ldx] : (T)0;
    xJ[i][c] = i < nJ ? x[tk.sJ + i + c * ldx] : (T)0;
  }
  __syncthreads();
  // warp w handles columns j = w, w + 8, ...; lane handles rows lane + 32 t
  T u[8][NR];
  T xi[8][NR];   // this lane's rows of x_I, kept in registers for every column
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int c = 0; c < NR; ++c) {
      u[t][c] = (T)0;
      xi[t][c] = xI[lane + 32 * t][c];
    }
  T* vout = reinterpret_cast<T*>(part) + tk.vo;
  // four columns per warp per pass: 32 independent loads per lane in flight
  for (int j0 = warp * 4; j0 < nJ; j0 += 32) {
    T a[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q;
      const T* col = A + (long long)min(j, nJ - 1) * tk.lda;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        int i = lane + 32 * t;
        a[q][t] = (i < nI && j < nJ) ? col[i] : (T)0;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int j = j0 + q;
      T v[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) v[c] = (T)0;
      T xj[NR];
#pragma unroll
      for (int c = 0; c < NR; ++c) xj[c] = (j < nJ) ? xJ[j][c] : (T)0;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
          v[c] = fma(a[q][t], xi[t][c], v[c]);
          u[t][c] = fma(a[q][t], xj[c], u[t][c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NR; ++c) {
        T s = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0 && j < nJ) vout[j + c * nJ] = s;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int c = 0; c < NR; ++c) uacc[warp][lane + 32 * t][c] = u[t][c];
  __syncthreads();
  T* uout = reinterpret_cast<T*>(part) + tk.uo;
  for (int e = tid; e < nI * NR; e += NT) {
    int i = e % nI, c = e / nI;
    T s = (T)0;
#pragma unroll
    for (int w = 0; w < 8; ++w) s += uacc[w][i][c];
    uout[i + c * nI] = s;
  }
}

// y(box) = sum of its partials in list order.
template <typename T>
__global__ void __launch_bounds__(NT) gather_parts_kernel(const GatherTask* __restrict__ tasks, const long long* __restrict__ offs,
                                                          const T* __restrict__ part, T* __restrict__ y, long long ldy,
                                                          int nrhs) {
  const GatherTask tk = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < tk.n * nrhs; e += NT) {
    int i = e % tk.n, c = e / tk.n;
    T s = (T)0;
    for (int q = tk.p0; q < tk.p0 + tk.np; ++q) s += part[offs[q] + i + (long long)c * tk.n];
    y[tk.s + i + c * ldy] = s;
  }
}

}  // namespace

void launch_symv_pairs(const SymPairTask* d, int ntasks, const double* x, int64_t ldx, double* part, int nrhs,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("symv_pairs_f64", s);
  if (nrhs == 1) symv_pairs_kernel<double, 1><<<ntasks, NT, 0, s>>>(d, x, ldx, part);
  else if (nrhs == 2) symv_pairs_kernel<double, 2><<<ntasks, NT, 0, s>>>(d, x, ldx, part);
  else throw StatusError(1, "symv_pairs: nrhs > 2");
  H2_LAUNCH_CHECK();
}

void launch_gather_parts(const GatherTask* d, int ntasks, const long long* offs, const double* part, double* y,
                         int64_t ldy, int nrhs, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("gather_parts_f64", s);
  gather_parts_kernel<double><<<ntasks, NT, 0, s>>>(d, offs, part, y, ldy, nrhs);
  H2_LAUNCH_CHECK();
}

}  // namespace h2
