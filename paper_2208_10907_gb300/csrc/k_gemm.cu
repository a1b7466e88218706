// Batched, segmented SIMT GEMM: C = alpha * sum_t op(A_t) op(B_t) + beta * Cin.
//
// Every task owns one output matrix; the terms of a task are summed in the
// CTA's registers (owner-computes, deterministic, no atomics).  This one
// kernel serves the fill-in Grams (sum over near boxes), the projections
// (eq. rs, eq. ss), the Schur updates, the near-field part of the H^2
// matvec and the solve sweeps.
#include "h2_common.cuh"
#include "h2_prof.h"

#include <map>
#include <string>

namespace h2 {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename T> __device__ __forceinline__ T ld_elem(const void* p, long long idx, bool f64in) {
  if (f64in) return (T)(reinterpret_cast<const double*>(p)[idx]);
  return reinterpret_cast<const T*>(p)[idx];
}

template <typename T, bool F64IN>
__global__ void __launch_bounds__(NT) gemm_kernel(const GemmTask* __restrict__ tasks,
                                                  const GemmTerm* __restrict__ terms) {
  const GemmTask tk = tasks[blockIdx.x];
  const int tiles_m = (tk.M + BM - 1) / BM;
  const int tiles_n = (tk.N + BN - 1) / BN;
  const int tile = blockIdx.y;
  if (tile >= tiles_m * tiles_n) return;
  const int i0 = (tile % tiles_m) * BM;
  const int j0 = (tile / tiles_m) * BN;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;

  for (int t = tk.t0; t < tk.t0 + tk.nt; ++t) {
    const GemmTerm tm = terms[t];
    const bool TRA = (tm.flags & 1) != 0, TRB = (tm.flags & 2) != 0;   // uniform per CTA
    for (int k0 = 0; k0 < tm.K; k0 += BK) {
      // ---- stage op(A) tile (BM x BK) as As[k][i]
      if (!TRA) {
        int i = tid % 64, kk = tid / 64;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int k = kk + 4 * q;
          int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < tk.M && gk < tm.K) ? ld_elem<T>(tm.A, (long long)gi + (long long)gk * tm.lda, F64IN) : (T)0;
        }
      } else {
        int k = tid % 16, ii = tid / 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int i = ii + 16 * q;
          int gi = i0 + i, gk = k0 + k;
          As[k][i] = (gi < tk.M && gk < tm.K) ? ld_elem<T>(tm.A, (long long)gk + (long long)gi * tm.lda, F64IN) : (T)0;
        }
      }
      // ---- stage op(B) tile (BK x BN) as Bs[k][j]
      if (!TRB) {
        int k = tid % 16, jj = tid / 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int j = jj + 16 * q;
          int gj = j0 + j, gk = k0 + k;
          Bs[k][j] = (gj < tk.N && gk < tm.K) ? ld_elem<T>(tm.B, (long long)gk + (long long)gj * tm.ldb, F64IN) : (T)0;
        }
      } else {
        int j = tid % 64, kk = tid / 64;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          int k = kk + 4 * q;
          int gj = j0 + j, gk = k0 + k;
          Bs[k][j] = (gj < tk.N && gk < tm.K) ? ld_elem<T>(tm.B, (long long)gj + (long long)gk * tm.ldb, F64IN) : (T)0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        T a[4], b[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          a[q] = As[k][ty + 16 * q];
          b[q] = Bs[k][tx + 16 * q];
        }
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[p][q] = fma(a[p], b[q], acc[p][q]);
      }
      __syncthreads();
    }
  }
  T* C = reinterpret_cast<T*>(tk.C);
  const T* Cin = reinterpret_cast<const T*>(tk.Cin);
  const T alpha = (T)tk.alpha, beta = (T)tk.beta;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int gi = i0 + ty + 16 * p;
    if (gi >= tk.M) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gj = j0 + tx + 16 * q;
      if (gj >= tk.N) continue;
      T v = alpha * acc[p][q];
      if (Cin != nullptr && tk.beta != 0.0) v += beta * Cin[gi + (long long)gj * tk.ldcin];
      C[gi + (long long)gj * tk.ldc] = v;
    }
  }
}


// ---------------------------------------------------------------------------
// Skinny products (N <= 8 columns: one right-hand side or a few): the 64-wide
// tile of the GEMM above would waste most of its FMAs, so each CTA streams a
// 256-row slice of op(A) once and keeps the N columns of op(B) in shared
// memory.  Non-transposed terms: one thread per row, coalesced along the
// column.  Transposed terms: one warp per row, lanes along the contiguous
// column, then a warp reduction.  This is bandwidth-bound by design.
// ---------------------------------------------------------------------------
constexpr int GV_ROWS = 256, GV_MAXN = 8;

template <typename T, int NR>
__device__ __forceinline__ void xload(T (&xv)[GV_MAXN], const T* B, long long k, long long ldb, bool trb, int n) {
#pragma unroll
  for (int c = 0; c < GV_MAXN; ++c)
    if (c < NR) xv[c] = (c < n) ? (trb ? B[c + k * ldb] : B[k + c * ldb]) : (T)0;
}

template <typename T, int NR>
__global__ void __launch_bounds__(NT) gemv_kernel(const GemmTask* __restrict__ tasks,
                                                  const GemmTerm* __restrict__ terms) {
  const GemmTask tk = tasks[blockIdx.x];
  const int i0 = blockIdx.y * GV_ROWS;
  if (i0 >= tk.M) return;
  const int rows = min(GV_ROWS, tk.M - i0);
  __shared__ T yacc[GV_ROWS][GV_MAXN + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  bool any_tra = false;
  for (int t = tk.t0; t < tk.t0 + tk.nt; ++t) any_tra |= (terms[t].flags & 1) != 0;
  if (any_tra) {
    for (int e = tid; e < GV_ROWS * (GV_MAXN + 1); e += NT) (&yacc[0][0])[e] = (T)0;
    __syncthreads();
  }
  T racc[GV_MAXN];
#pragma unroll
  for (int c = 0; c < GV_MAXN; ++c) racc[c] = (T)0;
  for (int t = tk.t0; t < tk.t0 + tk.nt; ++t) {
    const GemmTerm tm = terms[t];
    const bool TRA = (tm.flags & 1) != 0, TRB = (tm.flags & 2) != 0;
    const T* A = reinterpret_cast<const T*>(tm.A);
    const T* B = reinterpret_cast<const T*>(tm.B);
    if (!TRA) {
      // one thread per row; x(k, :) is the same address for every thread
      if (tid < rows) {
        const T* a = A + (i0 + tid);
        int k = 0;
        for (; k + 4 <= tm.K; k += 4) {
          T v0 = a[(long long)(k + 0) * tm.lda], v1 = a[(long long)(k + 1) * tm.lda];
          T v2 = a[(long long)(k + 2) * tm.lda], v3 = a[(long long)(k + 3) * tm.lda];
          T x0[GV_MAXN], x1[GV_MAXN], x2[GV_MAXN], x3[GV_MAXN];
          xload<T, NR>(x0, B, k + 0, tm.ldb, TRB, tk.N);
          xload<T, NR>(x1, B, k + 1, tm.ldb, TRB, tk.N);
          xload<T, NR>(x2, B, k + 2, tm.ldb, TRB, tk.N);
          xload<T, NR>(x3, B, k + 3, tm.ldb, TRB, tk.N);
#pragma unroll
          for (int c = 0; c < GV_MAXN; ++c)
            if (c < NR) racc[c] = fma(v3, x3[c], fma(v2, x2[c], fma(v1, x1[c], fma(v0, x0[c], racc[c]))));
        }
        for (; k < tm.K; ++k) {
          T v = a[(long long)k * tm.lda];
          T x0[GV_MAXN];
          xload<T, NR>(x0, B, k, tm.ldb, TRB, tk.N);
#pragma unroll
          for (int c = 0; c < GV_MAXN; ++c)
            if (c < NR) racc[c] = fma(v, x0[c], racc[c]);
        }
      }
    } else {
      // one warp per row: lanes along the contiguous column of the stored matrix
      for (int r = warp; r < rows; r += NT / 32) {
        const T* a = A + (long long)(i0 + r) * tm.lda;
        T acc[GV_MAXN];
#pragma unroll
        for (int c = 0; c < GV_MAXN; ++c) acc[c] = (T)0;
        // four strided elements per lane per pass: their loads are issued
        // together and feed independent accumulators
        T acc2[GV_MAXN];
#pragma unroll
        for (int c = 0; c < GV_MAXN; ++c) acc2[c] = (T)0;
        int k = lane;
        for (; k + 96 < tm.K; k += 128) {
          const T v0 = a[k], v1 = a[k + 32], v2 = a[k + 64], v3 = a[k + 96];
          T x0[GV_MAXN], x1[GV_MAXN], x2[GV_MAXN], x3[GV_MAXN];
          xload<T, NR>(x0, B, k, tm.ldb, TRB, tk.N);
          xload<T, NR>(x1, B, k + 32, tm.ldb, TRB, tk.N);
          xload<T, NR>(x2, B, k + 64, tm.ldb, TRB, tk.N);
          xload<T, NR>(x3, B, k + 96, tm.ldb, TRB, tk.N);
#pragma unroll
          for (int c = 0; c < GV_MAXN; ++c)
            if (c < NR) {
              acc[c] = fma(v0, x0[c], acc[c]);
              acc2[c] = fma(v1, x1[c], acc2[c]);
              acc[c] = fma(v2, x2[c], acc[c]);
              acc2[c] = fma(v3, x3[c], acc2[c]);
            }
        }
        for (; k < tm.K; k += 32) {
          T v = a[k];
          T x0[GV_MAXN];
          xload<T, NR>(x0, B, k, tm.ldb, TRB, tk.N);
#pragma unroll
          for (int c = 0; c < GV_MAXN; ++c)
            if (c < NR) acc[c] = fma(v, x0[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < GV_MAXN; ++c) acc[c] += acc2[c];
#pragma unroll
        for (int c = 0; c < GV_MAXN; ++c) {
          if (c < NR) {
            T v = acc[c];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) yacc[r][c] += v;
          }
        }
      }
    }
  }
  if (any_tra) __syncthreads();
  T* C = reinterpret_cast<T*>(tk.C);
  const T* Cin = reinterpret_cast<const T*>(tk.Cin);
  if (tid < rows) {
#pragma unroll
    for (int c = 0; c < GV_MAXN; ++c) {
      if (c < NR && c < tk.N) {
        T y = racc[c] + (any_tra ? yacc[tid][c] : (T)0);
        T v = (T)tk.alpha * y;
        if (Cin != nullptr && tk.beta != 0.0) v += (T)tk.beta * Cin[(i0 + tid) + (long long)c * tk.ldcin];
        C[(i0 + tid) + (long long)c * tk.ldc] = v;
      }
    }
  }
}

template <typename T>
void gemv_dispatch(int N, dim3 g, const GemmTask* d_tasks, const GemmTerm* d_terms, cudaStream_t s) {
  if (N <= 1) gemv_kernel<T, 1><<<g, NT, 0, s>>>(d_tasks, d_terms);
  else if (N <= 2) gemv_kernel<T, 2><<<g, NT, 0, s>>>(d_tasks, d_terms);
  else if (N <= 4) gemv_kernel<T, 4><<<g, NT, 0, s>>>(d_tasks, d_terms);
  else gemv_kernel<T, 8><<<g, NT, 0, s>>>(d_tasks, d_terms);
}

template <typename T, bool F64IN>
void dispatch(const GemmTask* d_tasks, const GemmTerm* d_terms, dim3 grid, cudaStream_t s) {
  gemm_kernel<T, F64IN><<<grid, NT, 0, s>>>(d_tasks, d_terms);
}

}  // namespace

void launch_gemm_tc(const GemmTask* d_tasks, const GemmTerm* d_terms, int ntasks, int maxM, int maxN,
                    cudaStream_t s);

// FP32-class products go to the tcgen05 split-3xTF32 kernel unless H2_TC=0
// (H2_TC=1 forces it); by default the autotuner below decides per shape.
static int tc_mode() {
  static int v = -2;
  if (v == -2) {
    const char* e = getenv("H2_TC");
    v = !e ? -1 : (e[0] == '0' ? 0 : 1);
  }
  return v;
}

// ---------------------------------------------------------------------------
// Autotuner: for each shape bucket (output rows, output columns, summed K of
// a task, each rounded up to a power of two) the tcgen05 kernel and the SIMT
// kernel are timed once on scratch data of that shape (512 tasks, random
// values, CUDA events) and the faster one is used for the rest of the
// process.  The decision is made the first time a bucket is seen.
// ---------------------------------------------------------------------------
namespace {
int pow2_bucket(int v) {
  int b = 16;
  while (b < v && b < (1 << 20)) b <<= 1;
  return b;
}

__global__ void fill_kernel(float* p, size_t n) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
    p[e] = (float)((e * 2654435761u) % 1000) * 1e-3f - 0.5f;
}

struct TuneKey {
  int m, n, k;
  bool operator<(const TuneKey& o) const {
    return m != o.m ? m < o.m : (n != o.n ? n < o.n : k < o.k);
  }
};
std::map<TuneKey, bool>& tune_table() {
  static std::map<TuneKey, bool> t;
  return t;
}
}  // namespace

static bool autotune_use_tc(int maxM, int maxN, int ksum, cudaStream_t s) {
  TuneKey key{pow2_bucket(maxM), pow2_bucket(maxN), pow2_bucket(ksum)};
  auto& tab = tune_table();
  auto it = tab.find(key);
  if (it != tab.end()) return it->second;
  const int M = key.m, N = key.n, K = std::min(key.k, 4096);
  const int T = std::max(32, std::min(512, 131072 / K));
  float *A = nullptr, *B = nullptr, *C = nullptr;
  GemmTask* dt = nullptr;
  GemmTerm* dm = nullptr;
  bool tc = true;
  cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr;
  size_t na = (size_t)T * M * K, nb = (size_t)T * K * N, nc = (size_t)T * M * N;
  if (cudaMalloc(&A, na * 4) == cudaSuccess && cudaMalloc(&B, nb * 4) == cudaSuccess &&
      cudaMalloc(&C, nc * 4) == cudaSuccess && cudaMalloc(&dt, T * sizeof(GemmTask)) == cudaSuccess &&
      cudaMalloc(&dm, T * sizeof(GemmTerm)) == cudaSuccess) {
    std::vector<GemmTask> ht(T);
    std::vector<GemmTerm> hm(T);
    for (int t = 0; t < T; ++t) {
      ht[t] = GemmTask{C + (size_t)t * M * N, nullptr, M, N, M, M, t, 1, 1.0, 0.0};
      hm[t] = GemmTerm{A + (size_t)t * M * K, B + (size_t)t * K * N, K, M, K, 0};
    }
    fill_kernel<<<1024, 256, 0, s>>>(A, na);
    fill_kernel<<<1024, 256, 0, s>>>(B, nb);
    cudaMemcpyAsync(dt, ht.data(), T * sizeof(GemmTask), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dm, hm.data(), T * sizeof(GemmTerm), cudaMemcpyHostToDevice, s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    launch_gemm_tc(dt, dm, T, M, N, s);   // warm both paths
    gemm_kernel<float, false><<<dim3(T, tiles), NT, 0, s>>>(dt, dm);
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch_gemm_tc(dt, dm, T, M, N, s);
    cudaEventRecord(e1, s);
    for (int r = 0; r < 3; ++r) gemm_kernel<float, false><<<dim3(T, tiles), NT, 0, s>>>(dt, dm);
    cudaEventRecord(e2, s);
    if (cudaEventSynchronize(e2) == cudaSuccess) {
      float ttc = 0, tsimt = 0;
      cudaEventElapsedTime(&ttc, e0, e1);
      cudaEventElapsedTime(&tsimt, e1, e2);
      tc = ttc <= tsimt;
    }
  }
  (void)cudaGetLastError();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e2) cudaEventDestroy(e2);
  cudaFree(A);
  cudaFree(B);
  cudaFree(C);
  cudaFree(dt);
  cudaFree(dm);
  tab[key] = tc;
  return tc;
}

std::string autotune_report() {
  std::string o = "[";
  bool first = true;
  for (auto& kv : tune_table()) {
    o += (first ? "" : ",") + std::string("{\"m\":") + std::to_string(kv.first.m) + ",\"n\":" +
         std::to_string(kv.first.n) + ",\"k\":" + std::to_string(kv.first.k) + ",\"kernel\":\"" +
         (kv.second ? "tcgen05" : "simt") + "\"}";
    first = false;
  }
  return o + "]";
}

void launch_gemm(Prec p, const GemmTask* d_tasks, const GemmTerm* d_terms,
                 int ntasks, int maxM, int maxN, cudaStream_t s, bool inputs_f64, int ksum) {
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) return;
  if (maxN <= GV_MAXN && !inputs_f64) {
    dim3 g(ntasks, (maxM + GV_ROWS - 1) / GV_ROWS);
    ProfScope ps(p == Prec::F64 ? "gemv_f64" : "gemv_f32", s);
    if (p == Prec::F64) gemv_dispatch<double>(maxN, g, d_tasks, d_terms, s);
    else gemv_dispatch<float>(maxN, g, d_tasks, d_terms, s);
    H2_LAUNCH_CHECK();
    return;
  }
  const int tm = tc_mode();
  bool use_tc = false;
  if (p == Prec::F32 && !inputs_f64 && maxM >= 32 && maxN >= 32 && tm != 0) {
    if (tm == 1 || ksum <= 0) use_tc = true;
    else {
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      cudaStreamIsCapturing(s, &cs);
      use_tc = (cs != cudaStreamCaptureStatusNone) ? true : autotune_use_tc(maxM, maxN, ksum, s);
    }
  }
  if (use_tc) {
    launch_gemm_tc(d_tasks, d_terms, ntasks, maxM, maxN, s);
    return;
  }
  int tiles = ((maxM + BM - 1) / BM) * ((maxN + BN - 1) / BN);
  dim3 grid(ntasks, tiles);
  ProfScope ps(p == Prec::F64 ? "gemm_f64" : "gemm_f32", s);
  if (p == Prec::F64) dispatch<double, false>(d_tasks, d_terms, grid, s);
  else if (inputs_f64) dispatch<float, true>(d_tasks, d_terms, grid, s);
  else dispatch<float, false>(d_tasks, d_terms, grid, s);
  H2_LAUNCH_CHECK();
}

}  // namespace h2
