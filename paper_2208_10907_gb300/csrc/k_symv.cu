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

// ---------------------------------------------------------------------------
// Single right-hand side: the same pass in double-float arithmetic.  Each
// FP64 block entry is split exactly by bit manipulation into a pair of FP32
// values (hi = leading 24 significand bits, lo = the next 23), x likewise,
// and every product a*x is formed as hi*hi (exact through an FMA residual)
// plus the two cross terms, accumulated in an unnormalised (hi, lo) FP32
// pair.  The relative error per product is about 2^-46; the work runs on the
// FP32 pipes, which on this GPU are 64 times faster than FP64, so the pass
// is bound by the HBM read of the blocks instead of by FP64 FMA throughput.
// ---------------------------------------------------------------------------
constexpr int DFQ = 2;   // columns per warp pass of the double-float kernel

__device__ __forceinline__ void df_split(double a, float& h, float& l) {
  const unsigned hi32 = (unsigned)__double2hiint(a), lo32 = (unsigned)__double2loint(a);
  const unsigned sign = hi32 & 0x80000000u;
  const int fe = (int)((hi32 >> 20) & 0x7FFu) - 896;           // FP32 biased exponent of a
  if (fe >= 24 && fe <= 254) {
    const unsigned mh = (__funnelshift_l(lo32, hi32, 3)) & 0x7FFFFFu;   // significand bits 51..29
    const unsigned ml = (lo32 >> 6) & 0x7FFFFFu;                       // significand bits 28..6
    h = __uint_as_float(sign | ((unsigned)fe << 23) | mh);
    const unsigned lb = sign | ((unsigned)(fe - 23) << 23);
    l = __fsub_rn(__uint_as_float(lb | ml), __uint_as_float(lb));
  } else if (((hi32 >> 20) & 0x7FFu) == 0u) {
    h = 0.f;                                                  // zero or FP64 subnormal
    l = 0.f;
  } else {                                                    // outside the pair's range: round
    h = __double2float_rn(a);
    l = __double2float_rn(a - (double)h);
  }
}

// (sh, sl) += (ah + al) * (xh + xl), dropping al*xl
__device__ __forceinline__ void df_fma(float ah, float al, float xh, float xl, float& sh, float& sl) {
  const float p = __fmul_rn(ah, xh);
  const float pe = fmaf(ah, xh, -p);
  const float c = fmaf(ah, xl, fmaf(al, xh, pe));
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sl = __fadd_rn(sl, __fadd_rn(e, c));
  sh = s;
}

// (sh, sl) += (oh, ol)
__device__ __forceinline__ void df_add(float oh, float ol, float& sh, float& sl) {
  const float s = __fadd_rn(sh, oh);
  const float bb = __fsub_rn(s, sh);
  const float e = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
  sl = __fadd_rn(sl, __fadd_rn(e, ol));
  sh = s;
}

__global__ void __launch_bounds__(NT, 3) symv_pairs_df_kernel(const SymPairTask* __restrict__ tasks,
                                                           const double* __restrict__ x, double* __restrict__ part) {
  const SymPairTask tk = tasks[blockIdx.x];
  const int nI = tk.nI, nJ = tk.nJ;
  const double* A = reinterpret_cast<const double*>(tk.A);
  __shared__ float xJh[256], xJl[256];
  __shared__ float2 uacc[8][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    float h, l;
    df_split(tid < nJ ? x[tk.sJ + tid] : 0.0, h, l);
    xJh[tid] = h;
    xJl[tid] = l;
  }
  float xih[8], xil[8], uh[8], ul[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    const int i = lane + 32 * t;
    df_split(i < nI ? x[tk.sI + i] : 0.0, xih[t], xil[t]);
    uh[t] = 0.f;
    ul[t] = 0.f;
  }
  __syncthreads();
  // partial results leave as unnormalised (hi, lo) FP32 pairs in the 8-byte
  // slots of the partial buffer; the gather adds them in FP64
  float2* vout = reinterpret_cast<float2*>(part) + tk.vo;
  // two columns per warp pass: few enough registers for three CTAs per SM
  for (int j0 = warp * DFQ; j0 < nJ; j0 += 8 * DFQ) {
    double a[DFQ][8];
#pragma unroll
    for (int q = 0; q < DFQ; ++q) {
      const int j = j0 + q;
      const double* col = A + (long long)min(j, nJ - 1) * tk.lda;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int i = lane + 32 * t;
        a[q][t] = (i < nI && j < nJ) ? col[i] : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < DFQ; ++q) {
      const int j = j0 + q;
      const float xjh = j < nJ ? xJh[j] : 0.f, xjl = j < nJ ? xJl[j] : 0.f;
      float vh = 0.f, vl = 0.f;
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        float ah, al;
        df_split(a[q][t], ah, al);
        df_fma(ah, al, xih[t], xil[t], vh, vl);
        df_fma(ah, al, xjh, xjl, uh[t], ul[t]);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, vh, o), ol = __shfl_down_sync(0xffffffffu, vl, o);
        df_add(oh, ol, vh, vl);
      }
      if (lane == 0 && j < nJ) vout[j] = make_float2(vh, vl);
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) uacc[warp][lane + 32 * t] = make_float2(uh[t], ul[t]);
  __syncthreads();
  float2* uout = reinterpret_cast<float2*>(part) + tk.uo;
  for (int i = tid; i < nI; i += NT) {
    float sh = uacc[0][i].x, sl = uacc[0][i].y;
#pragma unroll
    for (int w = 1; w < 8; ++w) df_add(uacc[w][i].x, uacc[w][i].y, sh, sl);
    uout[i] = make_float2(sh, sl);
  }
}

// y(box) = sum of its partials in list order (FP64 partials, or the
// double-float kernel's (hi, lo) FP32 pairs when DF is set).
template <typename T, bool DF>
__global__ void __launch_bounds__(NT) gather_parts_kernel(const GatherTask* __restrict__ tasks, const long long* __restrict__ offs,
                                                          const T* __restrict__ part, T* __restrict__ y, long long ldy,
                                                          int nrhs) {
  const GatherTask tk = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < tk.n * nrhs; e += NT) {
    int i = e % tk.n, c = e / tk.n;
    T s = (T)0;
    for (int q = tk.p0; q < tk.p0 + tk.np; ++q) {
      const long long o = offs[q] + i + (long long)c * tk.n;
      if (DF) {
        const float2 v = reinterpret_cast<const float2*>(part)[o];
        s += (T)v.x + (T)v.y;
      } else {
        s += part[o];
      }
    }
    y[tk.s + i + c * ldy] = s;
  }
}

}  // namespace

void launch_symv_pairs(const SymPairTask* d, int ntasks, const double* x, int64_t ldx, double* part, int nrhs,
                       cudaStream_t s) {
  if (ntasks <= 0) return;
  if (nrhs == 1) {
    ProfScope ps("symv_pairs_df", s);
    symv_pairs_df_kernel<<<ntasks, NT, 0, s>>>(d, x, part);
    H2_LAUNCH_CHECK();
    return;
  }
  ProfScope ps("symv_pairs_f64", s);
  if (nrhs == 2) symv_pairs_kernel<double, 2><<<ntasks, NT, 0, s>>>(d, x, ldx, part);
  else throw StatusError(1, "symv_pairs: nrhs > 2");
  H2_LAUNCH_CHECK();
}

void launch_gather_parts(const GatherTask* d, int ntasks, const long long* offs, const double* part, double* y,
                         int64_t ldy, int nrhs, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("gather_parts_f64", s);
  // one right-hand side: the partials come from the double-float kernel
  if (nrhs == 1) gather_parts_kernel<double, true><<<ntasks, NT, 0, s>>>(d, offs, part, y, ldy, nrhs);
  else gather_parts_kernel<double, false><<<ntasks, NT, 0, s>>>(d, offs, part, y, ldy, nrhs);
  H2_LAUNCH_CHECK();
}

}  // namespace h2
