// Batched small dense linear algebra, one CTA per box (n <= NMAX = 512).
//
// LU with partial pivoting (eq. lu), triangular solves (the eliminations of
// S^RS and S^SR and the solve sweeps), pivoted Cholesky of a Gram matrix
// (= column-pivoted QR of the block row, eq. u / eq. fillu), column-pivoted
// Householder QR, Householder QR with explicit Q (orthogonalised basis
// [U^R U^S]), the streamed fold of a far-field block row and the
// interpolation matrix of the ID.
#include "h2_common.cuh"
#include "h2_prof.h"

namespace h2 {

namespace {

constexpr int NT = 256;

template <typename T> __device__ __forceinline__ T tabs(T x) { return x < (T)0 ? -x : x; }

// Block-wide argmax of |val| with ties broken by the lowest index.
template <typename T>
__device__ void block_argmax(T val, int idx, T* s_val, int* s_idx, T& out_val, int& out_idx) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T v2 = __shfl_down_sync(0xffffffffu, val, o);
    int i2 = __shfl_down_sync(0xffffffffu, idx, o);
    if (v2 > val || (v2 == val && i2 < idx)) { val = v2; idx = i2; }
  }
  if (lane == 0) { s_val[warp] = val; s_idx[warp] = idx; }
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    val = lane < nw ? s_val[lane] : (T)-1;
    idx = lane < nw ? s_idx[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      T v2 = __shfl_down_sync(0xffffffffu, val, o);
      int i2 = __shfl_down_sync(0xffffffffu, idx, o);
      if (v2 > val || (v2 == val && i2 < idx)) { val = v2; idx = i2; }
    }
    if (lane == 0) { s_val[0] = val; s_idx[0] = idx; }
  }
  __syncthreads();
  out_val = s_val[0];
  out_idx = s_idx[0];
  __syncthreads();
}

template <typename T> __device__ T block_sum(T v, T* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) s[warp] = v;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    v = lane < nw ? s[lane] : (T)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) s[0] = v;
  }
  __syncthreads();
  T r = s[0];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// LU with partial pivoting of an m x nc panel (m >= nc), right-looking,
// column k and row k staged in shared memory.  Ties -> lowest row index.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) getrf_kernel(const LuTask* __restrict__ tasks) {
  const LuTask tk = tasks[blockIdx.x];
  T* A = reinterpret_cast<T*>(tk.A);
  const int m = tk.m, nc = tk.nc, lda = tk.lda;
  __shared__ T s_val[32];
  __shared__ int s_idx[32];
  extern __shared__ unsigned char smem_raw[];
  T* colk = reinterpret_cast<T*>(smem_raw);   // m
  T* rowk = colk + m;                          // nc
  bool singular = false;
  for (int k = 0; k < nc; ++k) {
    T best = (T)-1;
    int bi = 0x7fffffff;
    for (int i = k + threadIdx.x; i < m; i += NT) {
      T v = tabs(A[i + (long long)k * lda]);
      if (v > best || (v == best && i < bi)) { best = v; bi = i; }
    }
    T pv;
    int p;
    block_argmax(best, bi, s_val, s_idx, pv, p);
    if (tk.spd) p = k;       // symmetric positive definite: no pivoting
    if (p < k || p >= m) {   // every candidate was NaN: keep the row, flag the panel
      p = k;
      if (threadIdx.x == 0 && tk.info) atomicCAS(tk.info, 0, k + 1);
    }
    if (threadIdx.x == 0) tk.piv[k] = p;
    if (p != k) {
      for (int j = threadIdx.x; j < nc; j += NT) {
        T a = A[k + (long long)j * lda];
        A[k + (long long)j * lda] = A[p + (long long)j * lda];
        A[p + (long long)j * lda] = a;
      }
    }
    __syncthreads();
    T akk = A[k + (long long)k * lda];
    if (akk == (T)0 || akk != akk || (tk.spd && akk < (T)0)) {
      if (!singular && threadIdx.x == 0 && tk.info) atomicCAS(tk.info, 0, k + 1);
      singular = true;
      __syncthreads();
      continue;
    }
    T inv = (T)1 / akk;
    for (int i = k + 1 + threadIdx.x; i < m; i += NT) {
      T v = A[i + (long long)k * lda] * inv;
      A[i + (long long)k * lda] = v;
      colk[i] = v;
    }
    for (int j = k + 1 + threadIdx.x; j < nc; j += NT) rowk[j] = A[k + (long long)j * lda];
    __syncthreads();
    // trailing update, four columns at a time (their loads are issued
    // together, so the L2 latency is paid once per four), rows spread over
    // the threads
    int j = k + 1;
    for (; j + 3 < nc; j += 4) {
      const T r0 = rowk[j], r1 = rowk[j + 1], r2 = rowk[j + 2], r3 = rowk[j + 3];
      T* c0 = A + (long long)j * lda;
      T* c1 = c0 + lda;
      T* c2 = c1 + lda;
      T* c3 = c2 + lda;
      for (int i = k + 1 + threadIdx.x; i < m; i += NT) {
        const T ci = colk[i];
        const T v0 = c0[i], v1 = c1[i], v2 = c2[i], v3 = c3[i];
        c0[i] = v0 - ci * r0;
        c1[i] = v1 - ci * r1;
        c2[i] = v2 - ci * r2;
        c3[i] = v3 - ci * r3;
      }
    }
    for (; j < nc; ++j) {
      const T rj = rowk[j];
      T* col = A + (long long)j * lda;
      for (int i = k + 1 + threadIdx.x; i < m; i += NT) col[i] -= colk[i] * rj;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// The same LU, blocked (m <= NMAX): left-looking over panels of LW = 32
// columns held in shared memory.  A panel receives the row interchanges of
// the columns before it, then their updates 32 columns at a time (the unit
// lower triangle of the block, then the rows below it, whose L entries are
// read from global memory once per row), then is factored in shared memory;
// its interchanges are applied to the finished columns to its left.  Every
// entry receives the same updates in the same order and form (x - l*u) as in
// the unblocked kernel above, so the two give identical results; the
// trailing matrix is no longer read and written at every step.
// ---------------------------------------------------------------------------
constexpr int LW = 32, LWP = LW + 1;

template <typename T>
__global__ void __launch_bounds__(NT, 2) getrf_blocked_kernel(const LuTask* __restrict__ tasks) {
  const LuTask tk = tasks[blockIdx.x];
  T* A = reinterpret_cast<T*>(tk.A);
  const int m = tk.m, nc = tk.nc, lda = tk.lda;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ T s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv[NMAX];
  __shared__ unsigned char s_skip[NMAX];     // column k's pivot was zero / NaN: it updates nothing
  __shared__ T Ld[LW * LWP];                 // unit lower triangle of one finished 32-column block
  extern __shared__ unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);     // panel, m x LW, row-major with pitch LWP
  bool singular = false;
  for (int p0 = 0; p0 < nc; p0 += LW) {
    const int w = min(LW, nc - p0);
    for (int e = tid; e < m * w; e += NT) {
      const int i = e % m, c = e / m;
      P[i * LWP + c] = A[i + (long long)(p0 + c) * lda];
    }
    __syncthreads();
    // interchanges of the columns to the left, in order (one thread per column)
    if (tid < w) {
      for (int k = 0; k < p0; ++k) {
        const int p = s_piv[k];
        if (p != k) {
          const T a = P[k * LWP + tid];
          P[k * LWP + tid] = P[p * LWP + tid];
          P[p * LWP + tid] = a;
        }
      }
    }
    __syncthreads();
    for (int q = 0; q < p0; q += LW) {
      for (int e = tid; e < LW * LW; e += NT) {
        const int r = e % LW, k = e / LW;
        Ld[r * LWP + k] = A[(q + r) + (long long)(q + k) * lda];
      }
      __syncthreads();
      // rows q .. q+31: each warp solves whole columns, lanes = rows
      for (int c = warp; c < w; c += NT / 32) {
        for (int k = 0; k < LW - 1; ++k) {
          if (!s_skip[q + k] && lane > k)
            P[(q + lane) * LWP + c] = P[(q + lane) * LWP + c] - Ld[lane * LWP + k] * P[(q + k) * LWP + c];
          __syncwarp();
        }
      }
      __syncthreads();
      // rows below the block, each row in two halves of 16 columns
      const int nbelow = m - q - LW;
      for (int e = tid; e < 2 * nbelow; e += NT) {
        const int r = q + LW + e % nbelow, h = (e / nbelow) * (LW / 2);
        T lv[LW], acc[LW / 2];
#pragma unroll
        for (int k = 0; k < LW; ++k) lv[k] = A[r + (long long)(q + k) * lda];
#pragma unroll
        for (int c = 0; c < LW / 2; ++c) acc[c] = P[r * LWP + h + c];
#pragma unroll
        for (int k = 0; k < LW; ++k) {
          if (s_skip[q + k]) continue;
#pragma unroll
          for (int c = 0; c < LW / 2; ++c) acc[c] = acc[c] - lv[k] * P[(q + k) * LWP + h + c];
        }
#pragma unroll
        for (int c = 0; c < LW / 2; ++c) P[r * LWP + h + c] = acc[c];
      }
      __syncthreads();
    }
    // factor the panel in shared memory
    for (int c = 0; c < w; ++c) {
      const int k = p0 + c;
      T best = (T)-1;
      int bi = 0x7fffffff;
      for (int i = k + tid; i < m; i += NT) {
        const T v = tabs(P[i * LWP + c]);
        if (v > best || (v == best && i < bi)) { best = v; bi = i; }
      }
      T pv;
      int p;
      block_argmax(best, bi, s_val, s_idx, pv, p);
      if (tk.spd) p = k;
      if (p < k || p >= m) {
        p = k;
        if (tid == 0 && tk.info) atomicCAS(tk.info, 0, k + 1);
      }
      if (tid == 0) {
        s_piv[k] = p;
        tk.piv[k] = p;
      }
      if (p != k) {
        for (int j = tid; j < w; j += NT) {
          const T a = P[k * LWP + j];
          P[k * LWP + j] = P[p * LWP + j];
          P[p * LWP + j] = a;
        }
      }
      __syncthreads();
      const T akk = P[k * LWP + c];
      if (akk == (T)0 || akk != akk || (tk.spd && akk < (T)0)) {
        if (!singular && tid == 0 && tk.info) atomicCAS(tk.info, 0, k + 1);
        singular = true;
        if (tid == 0) s_skip[k] = 1;
        __syncthreads();
        continue;
      }
      if (tid == 0) s_skip[k] = 0;
      const T inv = (T)1 / akk;
      for (int i = k + 1 + tid; i < m; i += NT) P[i * LWP + c] = P[i * LWP + c] * inv;
      __syncthreads();
      const int rows = m - k - 1, cols = w - c - 1;
      for (int e = tid; e < rows * cols; e += NT) {
        const int i = k + 1 + e % rows, j = c + 1 + e / rows;
        P[i * LWP + j] = P[i * LWP + j] - P[i * LWP + c] * P[k * LWP + j];
      }
      __syncthreads();
    }
    // the panel's interchanges on the finished columns to its left, then
    // the panel back to global memory
    for (int j = tid; j < p0; j += NT) {
      for (int c = 0; c < w; ++c) {
        const int k = p0 + c, p = s_piv[k];
        if (p != k) {
          const T a = A[k + (long long)j * lda];
          A[k + (long long)j * lda] = A[p + (long long)j * lda];
          A[p + (long long)j * lda] = a;
        }
      }
    }
    for (int e = tid; e < m * w; e += NT) {
      const int i = e % m, c = e / m;
      A[i + (long long)(p0 + c) * lda] = P[i * LWP + c];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Left triangular solve B <- op(A)^-1 B on a 32-column chunk held in shared
// memory; A read from global memory.  Optional row interchanges first.
// Column by column (FP64): each step divides x_j (non-unit diagonal) and
// updates the rows beyond j with column j of op(A).
// ---------------------------------------------------------------------------
constexpr int TS_COLS = 32;


template <typename T, bool LOWER, bool UNIT, bool TRANSA>
__global__ void __launch_bounds__(NT) trsm_kernel(const TrsmTask* __restrict__ tasks) {
  const TrsmTask tk = tasks[blockIdx.x];
  const int c0 = blockIdx.y * TS_COLS;
  if (c0 >= tk.nrhs) return;
  const int nc = min(TS_COLS, tk.nrhs - c0);
  const int n = tk.n;
  const T* A = reinterpret_cast<const T*>(tk.A);
  T* B = reinterpret_cast<T*>(tk.B) + (long long)c0 * tk.ldb;
  extern __shared__ unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);   // n x (TS_COLS+1)
  const int LDX = TS_COLS + 1;
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    int i = e % n, c = e / n;
    X[i * LDX + c] = B[i + (long long)c * tk.ldb];
  }
  __syncthreads();
  if (tk.piv) {
    if (threadIdx.x < nc) {
      int c = threadIdx.x;
      for (int k = 0; k < n; ++k) {
        int p = tk.piv[k];
        if (p != k) {
          T a = X[k * LDX + c];
          X[k * LDX + c] = X[p * LDX + c];
          X[p * LDX + c] = a;
        }
      }
    }
    __syncthreads();
  }
  auto aij = [&](int i, int j) -> T {
    return TRANSA ? A[j + (long long)i * tk.lda] : A[i + (long long)j * tk.lda];
  };
  const int c = threadIdx.x % TS_COLS, r0 = threadIdx.x / TS_COLS;   // 8 row groups
  const int RG = NT / TS_COLS;
  if (LOWER) {
    for (int j = 0; j < n; ++j) {
      if (!UNIT) {
        if (threadIdx.x < nc) X[j * LDX + threadIdx.x] /= aij(j, j);
        __syncthreads();
      }
      if (c < nc) {
        T xj = X[j * LDX + c];
        int i = j + 1 + r0;
        for (; i + 3 * RG < n; i += 4 * RG) {   // four independent loads in flight
          const T a0 = aij(i, j), a1 = aij(i + RG, j), a2 = aij(i + 2 * RG, j), a3 = aij(i + 3 * RG, j);
          X[i * LDX + c] -= a0 * xj;
          X[(i + RG) * LDX + c] -= a1 * xj;
          X[(i + 2 * RG) * LDX + c] -= a2 * xj;
          X[(i + 3 * RG) * LDX + c] -= a3 * xj;
        }
        for (; i < n; i += RG) X[i * LDX + c] -= aij(i, j) * xj;
      }
      __syncthreads();
    }
  } else {
    for (int j = n - 1; j >= 0; --j) {
      if (!UNIT) {
        if (threadIdx.x < nc) X[j * LDX + threadIdx.x] /= aij(j, j);
        __syncthreads();
      }
      if (c < nc) {
        T xj = X[j * LDX + c];
        int i = r0;
        for (; i + 3 * RG < j; i += 4 * RG) {
          const T a0 = aij(i, j), a1 = aij(i + RG, j), a2 = aij(i + 2 * RG, j), a3 = aij(i + 3 * RG, j);
          X[i * LDX + c] -= a0 * xj;
          X[(i + RG) * LDX + c] -= a1 * xj;
          X[(i + 2 * RG) * LDX + c] -= a2 * xj;
          X[(i + 3 * RG) * LDX + c] -= a3 * xj;
        }
        for (; i < j; i += RG) X[i * LDX + c] -= aij(i, j) * xj;
      }
      __syncthreads();
    }
  }
  for (int e = threadIdx.x; e < n * nc; e += NT) {
    int i = e % n, cc = e / n;
    B[i + (long long)cc * tk.ldb] = X[i * LDX + cc];
  }
}

// ---------------------------------------------------------------------------
// The same solve blocked by 32 rows (FP32): the
// diagonal block of op(A) is staged in shared memory and solved by warps
// (one right-hand side column at a time, lanes = rows), then the rows beyond
// it take the block's 32 updates with their op(A) entries read from global
// memory once.  Every entry receives the updates x -= a x_j in the order of
// the column-by-column substitution (j ascending for lower, descending for
// upper; the division by a_jj first when the diagonal is not unit).
// ---------------------------------------------------------------------------

template <typename T, bool LOWER, bool UNIT, bool TRANSA>
__global__ void __launch_bounds__(NT, 2) trsm_blocked_kernel(const TrsmTask* __restrict__ tasks) {
  const TrsmTask tk = tasks[blockIdx.x];
  const int c0 = blockIdx.y * TS_COLS;
  if (c0 >= tk.nrhs) return;
  const int nc = min(TS_COLS, tk.nrhs - c0);
  const int n = tk.n;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T* A = reinterpret_cast<const T*>(tk.A);
  T* B = reinterpret_cast<T*>(tk.B) + (long long)c0 * tk.ldb;
  extern __shared__ unsigned char smem_raw[];
  T* X = reinterpret_cast<T*>(smem_raw);   // n x (TS_COLS+1)
  const int LDX = TS_COLS + 1;
  __shared__ T Ad[32 * 33];                // diagonal block of op(A)
  for (int e = tid; e < n * nc; e += NT) {
    int i = e % n, c = e / n;
    X[i * LDX + c] = B[i + (long long)c * tk.ldb];
  }
  __syncthreads();
  if (tk.piv) {
    if (tid < nc) {
      int c = tid;
      for (int k = 0; k < n; ++k) {
        int p = tk.piv[k];
        if (p != k) {
          T a = X[k * LDX + c];
          X[k * LDX + c] = X[p * LDX + c];
          X[p * LDX + c] = a;
        }
      }
    }
    __syncthreads();
  }
  auto aij = [&](int i, int j) -> T {
    return TRANSA ? A[j + (long long)i * tk.lda] : A[i + (long long)j * tk.lda];
  };
  const int nblk = (n + 31) / 32;
  for (int bb = 0; bb < nblk; ++bb) {
    const int blk = LOWER ? bb : nblk - 1 - bb;
    const int b = blk * 32, bw = min(32, n - b);
    for (int e = tid; e < 32 * 32; e += NT) {
      const int r = e % 32, k = e / 32;
      Ad[r * 33 + k] = (r < bw && k < bw) ? aij(b + r, b + k) : (T)0;
    }
    __syncthreads();
    // the diagonal block
    for (int c = warp; c < nc; c += NT / 32) {
      for (int t = 0; t < bw; ++t) {
        const int k = LOWER ? t : bw - 1 - t;
        if (!UNIT) {
          if (lane == k) X[(b + k) * LDX + c] /= Ad[k * 33 + k];
          __syncwarp();
        }
        const T xk = X[(b + k) * LDX + c];
        if (LOWER ? (lane > k && lane < bw) : (lane < k))
          X[(b + lane) * LDX + c] = X[(b + lane) * LDX + c] - Ad[lane * 33 + k] * xk;
        __syncwarp();
      }
    }
    __syncthreads();
    // the rows beyond the block: below it (lower) or above it (upper)
    const int r_lo = LOWER ? b + bw : 0, nr = LOWER ? n - r_lo : b;
    for (int e = tid; e < 2 * nr; e += NT) {   // each row in two halves of 16 columns
      const int r = r_lo + e % nr, h = (e / nr) * (TS_COLS / 2);
      T av[32], acc[TS_COLS / 2];
#pragma unroll
      for (int k = 0; k < 32; ++k) av[k] = k < bw ? aij(r, b + k) : (T)0;
#pragma unroll
      for (int c = 0; c < TS_COLS / 2; ++c) acc[c] = X[r * LDX + h + c];
#pragma unroll
      for (int t = 0; t < 32; ++t) {
        const int k = LOWER ? t : 31 - t;
        if (k >= bw) continue;
#pragma unroll
        for (int c = 0; c < TS_COLS / 2; ++c) acc[c] = acc[c] - av[k] * X[(b + k) * LDX + h + c];
      }
#pragma unroll
      for (int c = 0; c < TS_COLS / 2; ++c) X[r * LDX + h + c] = acc[c];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * nc; e += NT) {
    int i = e % n, cc = e / n;
    B[i + (long long)cc * tk.ldb] = X[i * LDX + cc];
  }
}

// ---------------------------------------------------------------------------
// Pivoted Cholesky of a Gram matrix G = B B^T (FP64).  Its pivots and R are
// those of the column-pivoted Householder QR of B^T: pivot on the largest
// remaining diagonal of the Schur complement (ties -> lowest index); stop
// when G_kk <= tol^2 G_11 (|R_kk| <= tol |R_11|) or at max_rank.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) pchol_kernel(const CholTask* __restrict__ tasks) {
  // Left-looking: step k forms only column k of the factor, from G's pivot
  // column and the k columns already computed (kept column-major in L so
  // that their reads coalesce), and downdates the diagonal.  Stopping at
  // rank r costs about n r^2 / 2 multiply-adds instead of the n^2 r of
  // updating the whole trailing matrix.  Positions are spread over the
  // threads (n <= NMAX).
  const CholTask tk = tasks[blockIdx.x];
  const double* G = tk.G;
  const int n = tk.n, ld = tk.ldg;
  double* R = tk.R;    // ld n
  double* L = tk.L;    // ld n: L(i, c) at L[i + c n], i in pivoted position order
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ double d[NMAX];     // diagonal of the remaining Schur complement
  __shared__ int perm[NMAX];
  __shared__ double lk[NMAX];    // row k of L
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += NT) {
    d[i] = G[i + (long long)i * ld];
    perm[i] = i;
  }
  __syncthreads();
  double d1 = 0.0;
  int rank = min(n, tk.max_rank);
  for (int k = 0; k < n; ++k) {
    double best = -INFINITY;
    int bi = 0x7fffffff;
    for (int i = k + tid; i < n; i += NT)
      if (d[i] > best || bi == 0x7fffffff) {   // first candidate, then strictly larger (lowest index on ties)
        best = d[i];
        bi = i;
      }
    double pv;
    int p;
    block_argmax(best, bi, s_val, s_idx, pv, p);
    if (p < k || p >= n || pv != pv || pv == INFINITY) {   // non-finite diagonal: stop, flag it
      if (tid == 0 && tk.info) *tk.info = 1;
      rank = k;
      break;
    }
    if (k == 0) d1 = pv;
    if (k >= tk.max_rank || pv <= tk.tol * tk.tol * d1 || pv <= 0.0) {
      rank = k;
      break;
    }
    if (p != k) {
      for (int c = tid; c < k; c += NT) {   // rows k and p of the computed columns
        const double a = L[k + (long long)c * n];
        L[k + (long long)c * n] = L[p + (long long)c * n];
        L[p + (long long)c * n] = a;
      }
      if (tid == 0) {
        const double t = d[k];
        d[k] = d[p];
        d[p] = t;
        const int q = perm[k];
        perm[k] = perm[p];
        perm[p] = q;
      }
      __syncthreads();
    }
    for (int c = tid; c < k; c += NT) lk[c] = L[k + (long long)c * n];
    __syncthreads();
    const double rkk = sqrt(d[k]);
    const int pk = perm[k];
    for (int i = k + 1 + tid; i < n; i += NT) {
      double c = G[perm[i] + (long long)pk * ld];
      int q = 0;
      double c1 = 0.0, c2 = 0.0, c3 = 0.0;
      for (; q + 3 < k; q += 4) {   // four independent loads in flight
        const double l0 = L[i + (long long)q * n], l1 = L[i + (long long)(q + 1) * n];
        const double l2 = L[i + (long long)(q + 2) * n], l3 = L[i + (long long)(q + 3) * n];
        c -= l0 * lk[q];
        c1 -= l1 * lk[q + 1];
        c2 -= l2 * lk[q + 2];
        c3 -= l3 * lk[q + 3];
      }
      for (; q < k; ++q) c -= L[i + (long long)q * n] * lk[q];
      c += (c1 + c2) + c3;
      const double v = c / rkk;
      L[i + (long long)k * n] = v;
      d[i] -= v * v;
    }
    if (tid == 0) L[k + (long long)k * n] = rkk;
    __syncthreads();
  }
  // R = L^T (rows 0 .. rank-1), zero elsewhere; pivots in position order
  for (int e = threadIdx.x; e < n * n; e += NT) {
    const int c = e % n, j = e / n;   // R(c, j)
    R[e] = (c < rank && c <= j) ? L[j + (long long)c * n] : 0.0;
  }
  for (int i = tid; i < n; i += NT) tk.piv[i] = perm[i];
  if (threadIdx.x == 0) *tk.rank = rank;
}

// ---------------------------------------------------------------------------
// Householder QR with column pivoting (FP64) of an m x n matrix (n <= NMAX):
// pivot = remaining column of largest 2-norm, recomputed at every step
// (ties -> lowest index); stop at |R_kk| <= tol |R_11| or max_rank.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) pqr_kernel(const PqrTask* __restrict__ tasks) {
  const PqrTask tk = tasks[blockIdx.x];
  double* A = tk.A;
  const int m = tk.m, n = tk.n, lda = tk.lda;
  double* R = tk.R;
  __shared__ double s_val[32];
  __shared__ int s_idx[32];
  __shared__ double nrm[NMAX];
  __shared__ double s_beta, s_r11;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = NT / 32;
  for (int e = threadIdx.x; e < n * n; e += NT) R[e] = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) tk.piv[i] = i;
  __syncthreads();
  const int kmax = min(m, n);
  int rank = min(kmax, tk.max_rank);
  for (int k = 0; k < kmax; ++k) {
    // column norms of A[k:, j], warp per column
    for (int j = k + warp; j < n; j += nwarp) {
      double s = 0.0;
      for (int i = k + lane; i < m; i += 32) {
        double a = A[i + (long long)j * lda];
        s += a * a;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) nrm[j] = sqrt(s);
    }
    __syncthreads();
    double best = -1.0;
    int bi = 0x7fffffff;
    for (int j = k + threadIdx.x; j < n; j += NT) {
      double v = nrm[j];
      if (v > best || (v == best && j < bi)) { best = v; bi = j; }
    }
    double pv;
    int p;
    block_argmax(best, bi, s_val, s_idx, pv, p);
    if (p < k || p >= n || pv == INFINITY) {   // non-finite column norms: stop here, flag it
      if (threadIdx.x == 0 && tk.info) *tk.info = 1;
      rank = k;
      break;
    }
    if (p != k) {
      for (int i = threadIdx.x; i < m; i += NT) {
        double a = A[i + (long long)k * lda];
        A[i + (long long)k * lda] = A[i + (long long)p * lda];
        A[i + (long long)p * lda] = a;
      }
      for (int i = threadIdx.x; i < k; i += NT) {
        double a = R[i + (long long)k * n];
        R[i + (long long)k * n] = R[i + (long long)p * n];
        R[i + (long long)p * n] = a;
      }
      if (threadIdx.x == 0) {
        int t = tk.piv[k];
        tk.piv[k] = tk.piv[p];
        tk.piv[p] = t;
      }
      __syncthreads();
    }
    double alpha = pv;
    if (k == 0 && threadIdx.x == 0) s_r11 = alpha;
    __syncthreads();
    if (k >= tk.max_rank || alpha <= tk.tol * s_r11 || alpha == 0.0) {
      rank = k;
      break;
    }
    // Householder vector in place: v = x - beta e1, normalised so H = I - 2 v v^T
    double x0 = A[k + (long long)k * lda];
    double beta = x0 >= 0.0 ? -alpha : alpha;
    double v0 = x0 - beta;
    double vnorm2 = alpha * alpha - x0 * x0 + v0 * v0;
    double inv = 1.0 / sqrt(vnorm2);
    __syncthreads();
    if (threadIdx.x == 0) {
      A[k + (long long)k * lda] = v0 * inv;
      s_beta = beta;
    }
    for (int i = k + 1 + threadIdx.x; i < m; i += NT) A[i + (long long)k * lda] *= inv;
    __syncthreads();
    // apply to trailing columns: w_j = v^T A[k:, j]
    for (int j = k + 1 + warp; j < n; j += nwarp) {
      double s = 0.0;
      for (int i = k + lane; i < m; i += 32) s += A[i + (long long)k * lda] * A[i + (long long)j * lda];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      s = __shfl_sync(0xffffffffu, s, 0);
      for (int i = k + lane; i < m; i += 32) A[i + (long long)j * lda] -= 2.0 * A[i + (long long)k * lda] * s;
    }
    __syncthreads();
    if (threadIdx.x == 0) R[k + (long long)k * n] = s_beta;
    for (int j = k + 1 + threadIdx.x; j < n; j += NT) R[k + (long long)j * n] = A[k + (long long)j * lda];
    __syncthreads();
  }
  if (threadIdx.x == 0) *tk.rank = rank;
}

// ---------------------------------------------------------------------------
// Householder QR of M (n x r) with explicit Q: Q = [q_0 .. q_{n-1}], first r
// columns span range(M) (U^S), the rest its complement (U^R).  Output
// columns are ordered [U^R U^S]; W = the r x r triangular factor.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) hqr_kernel(const HqrTask* __restrict__ tasks) {
  const HqrTask tk = tasks[blockIdx.x];
  const int n = tk.n, r = tk.r, m = n - r;
  T* M = reinterpret_cast<T*>(tk.M);
  T* V = reinterpret_cast<T*>(tk.V);
  T* Q = reinterpret_cast<T*>(tk.Q);
  T* W = reinterpret_cast<T*>(tk.W);
  __shared__ T s_red[32];
  __shared__ T s_beta;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = NT / 32;
  for (int k = 0; k < r; ++k) {
    T s = 0;
    for (int i = k + threadIdx.x; i < n; i += NT) {
      T a = M[i + (long long)k * n];
      s += a * a;
    }
    T alpha2 = block_sum(s, s_red);
    T alpha = sqrt(alpha2);
    T x0 = M[k + (long long)k * n];
    T beta = x0 >= (T)0 ? -alpha : alpha;
    T v0 = x0 - beta;
    T vn2 = alpha2 - x0 * x0 + v0 * v0;
    T inv = vn2 > (T)0 ? (T)1 / sqrt(vn2) : (T)0;
    for (int i = threadIdx.x; i < n; i += NT) {
      T v = (i < k) ? (T)0 : (i == k ? v0 * inv : M[i + (long long)k * n] * inv);
      V[i + (long long)k * n] = v;
    }
    if (threadIdx.x == 0) s_beta = (vn2 > (T)0) ? beta : x0;
    __syncthreads();
    // reflector k applied to columns k+1 .. r-1, four columns per warp pass
    // (the reflector entries are loaded once for the four)
    for (int j0 = k + 1 + 4 * warp; j0 < r; j0 += 4 * nwarp) {
      const int nj = min(4, r - j0);
      T s[4] = {0, 0, 0, 0};
      for (int i = k + lane; i < n; i += 32) {
        const T v = V[i + (long long)k * n];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nj) s[q] += v * M[i + (long long)(j0 + q) * n];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
        s[q] = __shfl_sync(0xffffffffu, s[q], 0);
      }
      for (int i = k + lane; i < n; i += 32) {
        const T v = (T)2 * V[i + (long long)k * n];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nj) M[i + (long long)(j0 + q) * n] -= v * s[q];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) M[k + (long long)k * n] = s_beta;
    __syncthreads();
  }
  // W = upper triangle of M[0:r, 0:r]
  for (int e = threadIdx.x; e < r * r; e += NT) {
    int i = e % r, j = e / r;
    W[i + (long long)j * r] = (i <= j) ? M[i + (long long)j * n] : (T)0;
  }
  // Q = H_0 ... H_{r-1} I, written with columns permuted to [U^R U^S]:
  // column c of the Householder Q goes to position c < r ? m + c : c - r.
  for (int e = threadIdx.x; e < n * n; e += NT) {
    int i = e % n, c = e / n;
    int pos = c < r ? m + c : c - r;
    Q[i + (long long)pos * n] = (i == c) ? (T)1 : (T)0;
  }
  __syncthreads();
  for (int k = r - 1; k >= 0; --k) {
    // H_k applied to every column, four columns per warp pass
    for (int c0 = 4 * warp; c0 < n; c0 += 4 * nwarp) {
      const int nc = min(4, n - c0);
      T* qc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + min(q, nc - 1);
        qc[q] = Q + (long long)(c < r ? m + c : c - r) * n;
      }
      T s[4] = {0, 0, 0, 0};
      for (int i = k + lane; i < n; i += 32) {
        const T v = V[i + (long long)k * n];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc) s[q] += v * qc[q][i];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], o);
        s[q] = __shfl_sync(0xffffffffu, s[q], 0);
      }
      for (int i = k + lane; i < n; i += 32) {
        const T v = (T)2 * V[i + (long long)k * n];
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (q < nc && s[q] != (T)0) qc[q][i] -= v * s[q];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Streamed fold of a block row B (n x cols): R (n x n, upper) with
// R^T R = B B^T, by Householder elimination of 32-row chunks of B^T against
// the running triangle (the pivoted QR of R then has the pivots and R of the
// pivoted QR of B^T, eq. u / eq. fillu).  The rows of B^T come from explicit
// blocks (FoldTerm: the fill-in products, near blocks, a transformed
// triangle) and then from the far-field samples, whose kernel values are
// evaluated straight into shared memory (never stored).
// ---------------------------------------------------------------------------
constexpr int FC = 32;      // rows per chunk (one per lane of a warp)
constexpr int FNB = 16;     // panel width of the blocked elimination

// Shared state of one fold CTA for boxes of at most NW columns.
template <int NW>
struct FoldSmem {
  double C[FC][NW + 1];     // the chunk of rows being folded (zero-padded to FC rows)
  double Rp[FNB][NW + 1];   // R rows [k0, k0 + nb) of the current panel, columns k0 ..
  double V[FC][FNB];        // Householder vectors of the panel (C part; the R part is e_k)
  double T[FNB][FNB];       // block reflector: H_0 ... H_{nb-1} = I - Y T Y^T (upper)
  double tau[FNB];
  double scol[FNB];
  double cx[NW], cy[NW], cz[NW];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fold the chunk S.C (FC x n) into R (n x n upper, global, ld n): the QR of
// [R; C] by panels of FNB columns.  In a panel, reflector k (acting on R row
// k and the chunk rows) annihilates column k of C and is applied at once to
// the panel's other columns (one warp per column); the panel's reflectors
// are then accumulated into the compact form I - Y T Y^T and applied to the
// trailing columns together (W = R_p + V^T C, W <- T^T W, R_p -= W,
// C -= V W), one column per thread with W in registers.
template <int NW>
__device__ void fold_chunk(double* __restrict__ R, int n, FoldSmem<NW>& S) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = NT / 32;
  for (int k0 = 0; k0 < n; k0 += FNB) {
    const int nb = min(FNB, n - k0), w0 = n - k0;
    // panel rows of R into shared memory (column by column, coalesced)
    for (int e = tid; e < nb * w0; e += NT) {
      const int i = e % nb, jj = e / nb;
      S.Rp[i][jj] = R[(long long)(k0 + i) + (long long)(k0 + jj) * n];
    }
    for (int e = tid; e < FC * FNB; e += NT) S.V[e / FNB][e % FNB] = 0.0;
    __syncthreads();
    // panel factorization
    for (int kk = 0; kk < nb; ++kk) {
      const int k = k0 + kk;
      if (warp == 0) {
        const double x = S.C[lane][k];
        const double sq = warp_sum(x * x);
        const double r = S.Rp[kk][kk];
        double v = 0.0, t = 0.0, beta = r;
        if (sq != 0.0) {
          const double alpha = sqrt(r * r + sq);
          beta = r >= 0.0 ? -alpha : alpha;
          const double v0 = r - beta;
          v = x / v0;
          t = -v0 / beta;
        }
        S.V[lane][kk] = v;
        if (lane == 0) {
          S.tau[kk] = t;
          S.Rp[kk][kk] = beta;
        }
      }
      __syncthreads();
      const double t = S.tau[kk];
      if (t != 0.0) {
        for (int jj = kk + 1 + warp; jj < nb; jj += nwarp) {
          const double vq = S.V[lane][kk];
          const double c = S.C[lane][k0 + jj];
          const double w = t * (S.Rp[kk][jj] + warp_sum(vq * c));
          S.C[lane][k0 + jj] = c - vq * w;
          __syncwarp();
          if (lane == 0) S.Rp[kk][jj] -= w;
        }
      }
      __syncthreads();
    }
    // T of the panel (one warp): T(i, i) = tau_i, T(0:i, i) = -tau_i T(0:i, 0:i) (V^T v_i)
    if (warp == 0) {
      for (int i = 0; i < FNB; ++i) {
        double sv = 0.0;
        if (lane < i && i < nb)
          for (int q = 0; q < FC; ++q) sv += S.V[q][lane] * S.V[q][i];
        if (lane < FNB) S.scol[lane] = sv;
        __syncwarp();
        const double ti = (i < nb) ? S.tau[i] : 0.0;
        if (lane < i) {
          double acc = 0.0;
          for (int l = lane; l < i; ++l) acc += S.T[lane][l] * S.scol[l];
          S.T[lane][i] = -ti * acc;
        } else if (lane < FNB) {
          S.T[lane][i] = (lane == i) ? ti : 0.0;
        }
        __syncwarp();
      }
    }
    __syncthreads();
    // ---- trailing columns j >= k0 + nb: one column per thread at a time
    for (int jj = nb + tid; jj < w0; jj += NT) {
      {
        double w[FNB];
#pragma unroll
        for (int i = 0; i < FNB; ++i) w[i] = (i < nb) ? S.Rp[i][jj] : 0.0;
#pragma unroll 8
        for (int q = 0; q < FC; ++q) {
          const double cq = S.C[q][k0 + jj];
#pragma unroll
          for (int i = 0; i < FNB; ++i) w[i] = fma(S.V[q][i], cq, w[i]);
        }
        // w <- T^T w, in place from the last entry down
#pragma unroll
        for (int i = FNB - 1; i >= 0; --i) {
          double a = 0.0;
#pragma unroll
          for (int p = 0; p <= i; ++p) a = fma(S.T[p][i], w[p], a);
          w[i] = a;
        }
#pragma unroll
        for (int i = 0; i < FNB; ++i)
          if (i < nb) S.Rp[i][jj] -= w[i];
        for (int q0 = 0; q0 < FC; q0 += 8) {   // eight independent chunk rows at a time
          double c[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) c[q] = S.C[q0 + q][k0 + jj];
#pragma unroll
          for (int i = 0; i < FNB; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q) c[q] = fma(-S.V[q0 + q][i], w[i], c[q]);
#pragma unroll
          for (int q = 0; q < 8; ++q) S.C[q0 + q][k0 + jj] = c[q];
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < nb * w0; e += NT) {
      const int i = e % nb, jj = e / nb;
      R[(long long)(k0 + i) + (long long)(k0 + jj) * n] = S.Rp[i][jj];
    }
    __syncthreads();
  }
}

template <int NW>
__global__ void __launch_bounds__(NT, NW <= 256 ? 2 : 1) fold_kernel(const FoldTask* __restrict__ tasks,
                                                                    const FoldTerm* __restrict__ terms, Points pts,
                                                                    KParams kp) {
  const FoldTask tk = tasks[blockIdx.x];
  const int n = tk.n;
  double* R = tk.R;
  extern __shared__ __align__(16) unsigned char fold_raw[];
  FoldSmem<NW>& S = *reinterpret_cast<FoldSmem<NW>*>(fold_raw);
  if (!tk.accumulate)
    for (int e = threadIdx.x; e < n * n; e += NT) R[e] = 0.0;
  if (tk.m > 0)
    for (int i = threadIdx.x; i < n; i += NT) {
      int g = tk.cand[i];
      S.cx[i] = pts.x[g];
      S.cy[i] = pts.y[g];
      S.cz[i] = pts.z[g];
    }
  __syncthreads();
  // explicit rows: row q of a term, element j = tr ? X[q + j ld] : X[j + q ld]
  for (int t = tk.t0; t < tk.t0 + tk.nt; ++t) {
    const FoldTerm ft = terms[t];
    for (int q0 = 0; q0 < ft.rows; q0 += FC) {
      const int c = min(FC, ft.rows - q0);
      if (ft.tr) {   // the chunk's rows are columns of X: threads along q read contiguously
        for (int e = threadIdx.x; e < FC * n; e += NT) {
          const int q = e % FC, j = e / FC;
          S.C[q][j] = q < c ? ft.X[(long long)(q0 + q) + (long long)j * ft.ld] : 0.0;
        }
      } else {
        for (int e = threadIdx.x; e < FC * n; e += NT) {
          const int q = e / n, j = e % n;
          S.C[q][j] = q < c ? ft.X[(long long)j + (long long)(q0 + q) * ft.ld] : 0.0;
        }
      }
      __syncthreads();
      fold_chunk(R, n, S);
    }
  }
  // far-field samples: row q = K(x[samp[q]], x[cand[:]])
  for (int s0 = 0; s0 < tk.m; s0 += FC) {
    const int c = min(FC, tk.m - s0);
    for (int e = threadIdx.x; e < FC * n; e += NT) {
      int q = e / n, j = e % n;
      double v = 0.0;
      if (q < c) {
        int g = tk.samp[s0 + q];
        v = kernel_eval(kp, S.cx[j] - pts.x[g], S.cy[j] - pts.y[g], S.cz[j] - pts.z[g]);
      }
      S.C[q][j] = v;
    }
    __syncthreads();
    fold_chunk(R, n, S);
  }
}

// ---------------------------------------------------------------------------
// G (+)= B B^T for B = K(x[cand], x[samp]), tiles 64 x 64, kernel values
// generated on the fly (never stored).  Computed in T, accumulated in FP64.
// In FP32 the coordinates are taken relative to the box's first candidate
// (one FP64 subtraction per point and tile), so that the kernel evaluations
// run on the FP32 pipes; the samples are far from the box.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) kgram_kernel(const KgramTask* __restrict__ tasks, Points pts,
                                                   KParams kp) {
  const KgramTask tk = tasks[blockIdx.x];
  const int tiles = (tk.n + 63) / 64;
  if ((int)blockIdx.y >= tiles * tiles) return;
  const int i0 = (blockIdx.y % tiles) * 64, j0 = (blockIdx.y / tiles) * 64;
  __shared__ T As[16][68];
  __shared__ T Bs[16][68];
  __shared__ double ax[64], ay[64], az[64], bx[64], by[64], bz[64];
  constexpr bool F32 = sizeof(T) == 4;
  __shared__ float fa[3][64], fb[3][64], fs[3][16];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int g0 = tk.cand[0];
  const double cx = pts.x[g0], cy = pts.y[g0], cz = pts.z[g0];
  if (tid < 64) {
    int i = i0 + tid;
    int g = i < tk.n ? tk.cand[i] : tk.cand[0];
    ax[tid] = pts.x[g]; ay[tid] = pts.y[g]; az[tid] = pts.z[g];
    if (F32) {
      fa[0][tid] = (float)(ax[tid] - cx); fa[1][tid] = (float)(ay[tid] - cy); fa[2][tid] = (float)(az[tid] - cz);
    }
  } else if (tid < 128) {
    int j = j0 + tid - 64;
    int g = j < tk.n ? tk.cand[j] : tk.cand[0];
    bx[tid - 64] = pts.x[g]; by[tid - 64] = pts.y[g]; bz[tid - 64] = pts.z[g];
    if (F32) {
      fb[0][tid - 64] = (float)(bx[tid - 64] - cx);
      fb[1][tid - 64] = (float)(by[tid - 64] - cy);
      fb[2][tid - 64] = (float)(bz[tid - 64] - cz);
    }
  }
  __syncthreads();
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
  for (int k0 = 0; k0 < tk.m; k0 += 16) {
    if (F32) {
      if (tid < 16 && k0 + tid < tk.m) {
        const int g = tk.samp[k0 + tid];
        fs[0][tid] = (float)(pts.x[g] - cx);
        fs[1][tid] = (float)(pts.y[g] - cy);
        fs[2][tid] = (float)(pts.z[g] - cz);
      }
      __syncthreads();
    }
    {
      int i = tid % 64, kk = tid / 64;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int k = kk + 4 * q;
        int gk = k0 + k;
        T va = (T)0, vb = (T)0;
        if (gk < tk.m) {
          if (F32) {
            const float sx = fs[0][k], sy = fs[1][k], sz = fs[2][k];
            if (i0 + i < tk.n) va = (T)kernel_eval_ff(kp, fa[0][i] - sx, fa[1][i] - sy, fa[2][i] - sz);
            if (j0 + i < tk.n) vb = (T)kernel_eval_ff(kp, fb[0][i] - sx, fb[1][i] - sy, fb[2][i] - sz);
          } else {
            int g = tk.samp[gk];
            double sx = pts.x[g], sy = pts.y[g], sz = pts.z[g];
            if (i0 + i < tk.n) va = KEval<T>::eval(kp, ax[i] - sx, ay[i] - sy, az[i] - sz);
            if (j0 + i < tk.n) vb = KEval<T>::eval(kp, bx[i] - sx, by[i] - sy, bz[i] - sz);
          }
        }
        As[k][i] = va;
        Bs[k][i] = vb;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
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
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    int gi = i0 + ty + 16 * p;
    if (gi >= tk.n) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int gj = j0 + tx + 16 * q;
      if (gj >= tk.n) continue;
      double v = (double)acc[p][q];
      long long o = gi + (long long)gj * tk.ldg;
      tk.G[o] = tk.accumulate ? tk.G[o] + v : v;
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel-block assembly: out(i, j) = K(x[ridx[i]], x[cidx[j]]).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(NT) assemble_kernel(const AsmTask* __restrict__ tasks, Points pts,
                                                      KParams kp) {
  const AsmTask tk = tasks[blockIdx.x];
  const int j = blockIdx.y;
  if (j >= tk.nc) return;
  const int gj = tk.cidx ? tk.cidx[j] : tk.c0 + j;
  const double xj = pts.x[gj], yj = pts.y[gj], zj = pts.z[gj];
  T* out = reinterpret_cast<T*>(tk.out) + (long long)j * tk.ld;
  for (int i = threadIdx.x; i < tk.nr; i += NT) {
    int gi = tk.ridx ? tk.ridx[i] : tk.r0 + i;
    out[i] = KEval<T>::eval(kp, pts.x[gi] - xj, pts.y[gi] - yj, pts.z[gi] - zj);
  }
}

// Far-field block row in FP32: out(i, j) = K(x[ridx[i]], x[cidx[j]]) with
// coordinates taken relative to the box's first row point (one FP64
// subtraction per point, the rest on the FP32 pipes); the columns are far
// from the box, so the differences lose no relative accuracy.
__global__ void __launch_bounds__(NT) assemble_far_f32_kernel(const AsmTask* __restrict__ tasks, Points pts,
                                                              KParams kp) {
  const AsmTask tk = tasks[blockIdx.x];
  __shared__ float fx[NMAX], fy[NMAX], fz[NMAX];
  __shared__ float sx[32], sy[32], sz[32];
  const int g0 = tk.ridx[0];
  const double cx = pts.x[g0], cy = pts.y[g0], cz = pts.z[g0];
  for (int i = threadIdx.x; i < tk.nr; i += NT) {
    const int g = tk.ridx[i];
    fx[i] = (float)(pts.x[g] - cx);
    fy[i] = (float)(pts.y[g] - cy);
    fz[i] = (float)(pts.z[g] - cz);
  }
  float* out = reinterpret_cast<float*>(tk.out);
  for (int j0 = blockIdx.y * 32; j0 < tk.nc; j0 += gridDim.y * 32) {
    __syncthreads();
    if (threadIdx.x < 32 && j0 + threadIdx.x < tk.nc) {
      const int g = tk.cidx[j0 + threadIdx.x];
      sx[threadIdx.x] = (float)(pts.x[g] - cx);
      sy[threadIdx.x] = (float)(pts.y[g] - cy);
      sz[threadIdx.x] = (float)(pts.z[g] - cz);
    }
    __syncthreads();
    const int nj = min(32, tk.nc - j0);
    for (int e = threadIdx.x; e < nj * tk.nr; e += NT) {
      const int i = e % tk.nr, jj = e / tk.nr;
      out[i + (long long)(j0 + jj) * tk.ld] = kernel_eval_ff(kp, fx[i] - sx[jj], fy[i] - sy[jj], fz[i] - sz[jj]);
    }
  }
}

template <typename TS, typename TD, bool TR>
__global__ void __launch_bounds__(NT) copy_kernel(const CopyTask* __restrict__ tasks) {
  const CopyTask tk = tasks[blockIdx.x];
  const TS* s = reinterpret_cast<const TS*>(tk.src);
  TD* d = reinterpret_cast<TD*>(tk.dst);
  if (!TR) {
    // column by column: a column takes the rows rounded up to whole warps
    // (at most all threads), the CTA's threads cover several columns at
    // once, and the CTAs of a task take interleaved column groups (no index
    // division per element)
    const int R = tk.rows;
    const int tpc = R >= NT ? NT : ((R + 31) & ~31);
    const int cpp = NT / tpc;
    const int sub = threadIdx.x / tpc, i0 = threadIdx.x % tpc;
    if (sub >= cpp) return;
    const int js = gridDim.y * cpp;
    int j = blockIdx.y * cpp + sub;
    // four columns per pass: their loads are in flight together
    for (; j + 3 * js < tk.cols; j += 4 * js) {
      for (int i = i0; i < R; i += tpc) {
        const TS v0 = s[i + (long long)j * tk.lds], v1 = s[i + (long long)(j + js) * tk.lds];
        const TS v2 = s[i + (long long)(j + 2 * js) * tk.lds], v3 = s[i + (long long)(j + 3 * js) * tk.lds];
        d[i + (long long)j * tk.ldd] = (TD)v0;
        d[i + (long long)(j + js) * tk.ldd] = (TD)v1;
        d[i + (long long)(j + 2 * js) * tk.ldd] = (TD)v2;
        d[i + (long long)(j + 3 * js) * tk.ldd] = (TD)v3;
      }
    }
    for (; j < tk.cols; j += js) {
      const TS* sc = s + (long long)j * tk.lds;
      TD* dc = d + (long long)j * tk.ldd;
      for (int i = i0; i < R; i += tpc) dc[i] = (TD)sc[i];
    }
    return;
  }
  const long long cnt = (long long)tk.rows * tk.cols;
  for (long long e = (long long)blockIdx.y * NT + threadIdx.x; e < cnt; e += (long long)gridDim.y * NT) {
    int i = (int)(e % tk.rows), j = (int)(e / tk.rows);
    TS v = s[j + (long long)i * tk.lds];
    d[i + (long long)j * tk.ldd] = (TD)v;
  }
}

// dst(i, j) += src(i, j): an FP32 block added into an FP64 one
__global__ void __launch_bounds__(NT) add_copy_kernel(const CopyTask* __restrict__ tasks) {
  const CopyTask tk = tasks[blockIdx.x];
  const float* s = reinterpret_cast<const float*>(tk.src);
  double* d = reinterpret_cast<double*>(tk.dst);
  const long long cnt = (long long)tk.rows * tk.cols;
  for (long long e = (long long)blockIdx.y * NT + threadIdx.x; e < cnt; e += (long long)gridDim.y * NT) {
    const int i = (int)(e % tk.rows), j = (int)(e / tk.rows);
    d[i + (long long)j * tk.ldd] += (double)s[i + (long long)j * tk.lds];
  }
}

// P (n x r): P[piv[i], i] = 1 (i < r); P[piv[c], :] = T[:, c - r]^T (c >= r).
template <typename T>
__global__ void __launch_bounds__(NT) interp_kernel(const InterpTask* __restrict__ tasks) {
  const InterpTask tk = tasks[blockIdx.x];
  T* P = reinterpret_cast<T*>(tk.P);
  const T* Tm = reinterpret_cast<const T*>(tk.T);
  const int n = tk.n, r = tk.r;
  for (long long e = threadIdx.x; e < (long long)n * r; e += NT) {
    int c = (int)(e % n), j = (int)(e / n);
    int row = tk.piv[c];
    T v;
    if (c < r) v = (c == j) ? (T)1 : (T)0;
    else v = Tm[j + (long long)(c - r) * tk.ldt];
    P[row + (long long)j * n] = v;
  }
}

__global__ void colnorm2_kernel(const double* X, int n, int nrhs, long long ld, double* out) {
  __shared__ double s[32];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += NT) {
    double v = X[i + (long long)c * ld];
    acc += v * v;
  }
  double t = block_sum(acc, s);
  if (threadIdx.x == 0) out[c] = t;
}

__global__ void axpy_cols_kernel(double* Y, const double* X, int n, int nrhs, long long ldy, long long ldx,
                                 double alpha) {
  long long cnt = (long long)n * nrhs;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < cnt; e += (long long)gridDim.x * NT) {
    int i = (int)(e % n), c = (int)(e / n);
    Y[i + c * ldy] += alpha * X[i + c * ldx];
  }
}

__global__ void permute_rows_kernel(const double* src, long long lds, double* dst, long long ldd,
                                    const int64_t* map, long long n, int nrhs, bool scatter) {
  long long cnt = n * nrhs;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < cnt; e += (long long)gridDim.x * NT) {
    long long i = e % n;
    int c = (int)(e / n);
    if (scatter) dst[map[i] + c * ldd] = src[i + c * lds];
    else dst[i + c * ldd] = src[map[i] + c * lds];
  }
}

// out[i] = sum_n V[n + i*ldv] * w[n], i < k <= 32: per-block partials, then
// a fixed-order reduction over blocks (deterministic).
constexpr int MDOT_MAXK = 32;
__global__ void __launch_bounds__(NT) mdot_partial_kernel(const double* __restrict__ V, long long ldv, int k,
                                                          const double* __restrict__ w, long long n,
                                                          double* __restrict__ partial) {
  __shared__ double s[32];
  double acc[MDOT_MAXK];
#pragma unroll
  for (int i = 0; i < MDOT_MAXK; ++i) acc[i] = 0.0;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) {
    const double wv = w[e];
#pragma unroll
    for (int i = 0; i < MDOT_MAXK; ++i)
      if (i < k) acc[i] = fma(V[e + i * ldv], wv, acc[i]);
  }
#pragma unroll 1
  for (int i = 0; i < k; ++i) {
    double t = block_sum(acc[i], s);
    if (threadIdx.x == 0) partial[(long long)blockIdx.x * MDOT_MAXK + i] = t;
  }
}

__global__ void mdot_reduce_kernel(const double* __restrict__ partial, int nblk, int k, double* __restrict__ out) {
  int i = threadIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(long long)b * MDOT_MAXK + i];
  out[i] = s;
}

// v = w / sqrt(norm2[0])
__global__ void normalize_kernel(double* v, const double* w, long long n, const double* norm2) {
  const double inv = 1.0 / sqrt(norm2[0]);
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < n; e += (long long)gridDim.x * NT) v[e] = w[e] * inv;
}

__global__ void gather_rows_kernel(const double* src, long long lds, double* dst, long long ldd, const int* idx,
                                   long long n, int nrhs) {
  long long cnt = n * nrhs;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < cnt; e += (long long)gridDim.x * NT) {
    long long i = e % n;
    int c = (int)(e / n);
    dst[i + c * ldd] = src[idx[i] + c * lds];
  }
}

template <typename T> __global__ void eye_kernel(T* A, int n, int ld) {
  long long cnt = (long long)n * n;
  for (long long e = (long long)blockIdx.x * NT + threadIdx.x; e < cnt; e += (long long)gridDim.x * NT) {
    int i = (int)(e % n), j = (int)(e / n);
    A[i + (long long)j * ld] = (i == j) ? (T)1 : (T)0;
  }
}

// Apply row interchanges piv[k0..k1) to columns [cb, ce) of A.
template <typename T>
__global__ void laswp_kernel(T* A, int lda, const int* piv, int k0, int k1, int cb, int ce) {
  for (int j = cb + blockIdx.x * NT + threadIdx.x; j < ce; j += gridDim.x * NT) {
    T* col = A + (long long)j * lda;
    for (int k = k0; k < k1; ++k) {
      int p = piv[k];
      if (p != k) {
        T a = col[k];
        col[k] = col[p];
        col[p] = a;
      }
    }
  }
}

// log|det| and sign of LU (or Cholesky: 2 sum log L_kk) factors, one CTA
// per factored block; results per task.
__global__ void logdet_kernel(const LuTask* __restrict__ tasks, double* out_log, double* out_sign,
                              bool chol) {
  const LuTask tk = tasks[blockIdx.x];
  __shared__ double s[32];
  const double* A = reinterpret_cast<const double*>(tk.A);
  double acc = 0.0, neg = 0.0;
  for (int k = threadIdx.x; k < tk.nc; k += NT) {
    double d = A[k + (long long)k * tk.lda];
    acc += log(fabs(d));
    if (!chol) {
      if (d < 0.0) neg += 1.0;
      if (tk.piv[k] != k) neg += 1.0;
    }
  }
  double t = block_sum(acc, s);
  double ng = block_sum(neg, s);
  if (threadIdx.x == 0) {
    out_log[blockIdx.x] = chol ? 2.0 * t : t;
    out_sign[blockIdx.x] = (fmod(ng, 2.0) == 0.0) ? 1.0 : -1.0;
  }
}

}  // namespace

// ------------------------------------------------------------ launchers ----
void launch_getrf(Prec p, const LuTask* d, int ntasks, int maxm, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps(p == Prec::F64 ? "getrf_f64" : "getrf_f32", s);
  if (maxm <= NMAX) {
    // blocked kernel: one m x 32 panel in shared memory
    const size_t smem = (size_t)std::max(maxm, 1) * LWP * (p == Prec::F64 ? 8 : 4);
    if (p == Prec::F64) {
      H2_CUDA(cudaFuncSetAttribute(getrf_blocked_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      getrf_blocked_kernel<double><<<ntasks, NT, smem, s>>>(d);
    } else {
      H2_CUDA(cudaFuncSetAttribute(getrf_blocked_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem));
      getrf_blocked_kernel<float><<<ntasks, NT, smem, s>>>(d);
    }
    H2_LAUNCH_CHECK();
    return;
  }
  // taller panels: unblocked kernel, column k and row k staged in shared
  // memory
  size_t smem = (size_t)2 * maxm * (p == Prec::F64 ? 8 : 4);   // nc <= m
  if (p == Prec::F64) {
    H2_CUDA(cudaFuncSetAttribute(getrf_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    getrf_kernel<double><<<ntasks, NT, smem, s>>>(d);
  } else {
    H2_CUDA(cudaFuncSetAttribute(getrf_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    getrf_kernel<float><<<ntasks, NT, smem, s>>>(d);
  }
  H2_LAUNCH_CHECK();
}

template <typename T>
static void trsm_dispatch(bool lower, bool unit, bool transA, const TrsmTask* d, dim3 grid, size_t smem,
                          cudaStream_t s) {
#define H2_TRSM_CASE(L, U, TR)                                                                        \
  if (lower == L && unit == U && transA == TR) {                                                      \
    if constexpr (sizeof(T) == 4) {                                                                   \
      H2_CUDA(cudaFuncSetAttribute(trsm_blocked_kernel<T, L, U, TR>,                                  \
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));          \
      trsm_blocked_kernel<T, L, U, TR><<<grid, NT, smem, s>>>(d);                                     \
    } else {                                                                                          \
      H2_CUDA(cudaFuncSetAttribute(trsm_kernel<T, L, U, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                   (int)smem));                                                       \
      trsm_kernel<T, L, U, TR><<<grid, NT, smem, s>>>(d);                                             \
    }                                                                                                 \
    return;                                                                                           \
  }
  H2_TRSM_CASE(true, true, false)
  H2_TRSM_CASE(true, false, false)
  H2_TRSM_CASE(false, false, false)
  H2_TRSM_CASE(false, true, false)
  H2_TRSM_CASE(true, false, true)
  H2_TRSM_CASE(false, false, true)
  H2_TRSM_CASE(true, true, true)
  H2_TRSM_CASE(false, true, true)
#undef H2_TRSM_CASE
}

void launch_trsm(Prec p, bool lower, bool unit, bool transA, const TrsmTask* d, int ntasks, int maxnrhs, int maxn,
                 cudaStream_t s) {
  if (ntasks <= 0 || maxnrhs <= 0 || maxn <= 0) return;
  if (maxn > NMAX) throw StatusError(1, "trsm: triangle larger than NMAX");
  ProfScope ps(p == Prec::F64 ? "trsm_f64" : "trsm_f32", s);
  dim3 grid(ntasks, (maxnrhs + TS_COLS - 1) / TS_COLS);
  size_t smem = (size_t)maxn * (TS_COLS + 1) * (p == Prec::F64 ? 8 : 4);
  if (p == Prec::F64) trsm_dispatch<double>(lower, unit, transA, d, grid, smem, s);
  else trsm_dispatch<float>(lower, unit, transA, d, grid, smem, s);
  H2_LAUNCH_CHECK();
}

void launch_pchol(const CholTask* d, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("pchol_f64", s);
  pchol_kernel<<<ntasks, NT, 0, s>>>(d);
  H2_LAUNCH_CHECK();
}

void launch_pqr(const PqrTask* d, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("pqr_f64", s);
  pqr_kernel<<<ntasks, NT, 0, s>>>(d);
  H2_LAUNCH_CHECK();
}

void launch_hqr(Prec p, const HqrTask* d, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps(p == Prec::F64 ? "hqr_f64" : "hqr_f32", s);
  if (p == Prec::F64) hqr_kernel<double><<<ntasks, NT, 0, s>>>(d);
  else hqr_kernel<float><<<ntasks, NT, 0, s>>>(d);
  H2_LAUNCH_CHECK();
}

template <int NW>
static void fold_launch(const FoldTask* d, int ntasks, const FoldTerm* terms, Points pts, KParams kp, cudaStream_t s) {
  size_t smem = sizeof(FoldSmem<NW>);
  H2_CUDA(cudaFuncSetAttribute(fold_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  H2_CUDA(cudaFuncSetAttribute(fold_kernel<NW>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  fold_kernel<NW><<<ntasks, NT, smem, s>>>(d, terms, pts, kp);
}

void launch_fold(const FoldTask* d, int ntasks, int maxn, const FoldTerm* terms, Points pts, KParams kp,
                 cudaStream_t s) {
  if (ntasks <= 0) return;
  if (maxn > NMAX) throw StatusError(1, "fold: box wider than NMAX");
  ProfScope ps("fold_f64", s);
  if (maxn <= 256) fold_launch<256>(d, ntasks, terms, pts, kp, s);
  else fold_launch<NMAX>(d, ntasks, terms, pts, kp, s);
  H2_LAUNCH_CHECK();
}

void launch_kgram(Prec p, const KgramTask* d, int ntasks, int maxn, Points pts, KParams kp, cudaStream_t s) {
  if (ntasks <= 0 || maxn <= 0) return;
  ProfScope ps(p == Prec::F64 ? "kgram_f64" : "kgram_f32", s);
  int t = (maxn + 63) / 64;
  dim3 grid(ntasks, t * t);
  if (p == Prec::F64) kgram_kernel<double><<<grid, NT, 0, s>>>(d, pts, kp);
  else kgram_kernel<float><<<grid, NT, 0, s>>>(d, pts, kp);
  H2_LAUNCH_CHECK();
}

void launch_assemble(Prec p, const AsmTask* d, int ntasks, int maxr, int maxc, Points pts, KParams kp,
                     cudaStream_t s) {
  if (ntasks <= 0 || maxc <= 0) return;
  ProfScope ps(p == Prec::F64 ? "assemble_f64" : "assemble_f32", s);
  dim3 grid(ntasks, maxc);
  if (p == Prec::F64) assemble_kernel<double><<<grid, NT, 0, s>>>(d, pts, kp);
  else assemble_kernel<float><<<grid, NT, 0, s>>>(d, pts, kp);
  H2_LAUNCH_CHECK();
}

void launch_assemble_far_f32(const AsmTask* d, int ntasks, int maxc, Points pts, KParams kp, cudaStream_t s) {
  if (ntasks <= 0 || maxc <= 0) return;
  ProfScope ps("assemble_far_f32", s);
  dim3 grid(ntasks, std::min(64, (maxc + 31) / 32));
  assemble_far_f32_kernel<<<grid, NT, 0, s>>>(d, pts, kp);
  H2_LAUNCH_CHECK();
}

void launch_copy(Prec src, Prec dst, bool transpose, const CopyTask* d, int ntasks, int maxr, int maxc,
                 cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("copy", s);
  long long cnt = (long long)maxr * maxc;
  int gy = (int)std::min<long long>(64, (cnt + NT - 1) / NT);
  if (gy < 1) gy = 1;
  dim3 grid(ntasks, gy);
#define H2_COPY(TS, TD)                                                  \
  if (transpose) copy_kernel<TS, TD, true><<<grid, NT, 0, s>>>(d);      \
  else copy_kernel<TS, TD, false><<<grid, NT, 0, s>>>(d);
  if (src == Prec::F64 && dst == Prec::F64) { H2_COPY(double, double) }
  else if (src == Prec::F64 && dst == Prec::F32) { H2_COPY(double, float) }
  else if (src == Prec::F32 && dst == Prec::F64) { H2_COPY(float, double) }
  else { H2_COPY(float, float) }
#undef H2_COPY
  H2_LAUNCH_CHECK();
}

void launch_add_copy(const CopyTask* d, int ntasks, int maxr, int maxc, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("add_copy", s);
  long long cnt = (long long)maxr * maxc;
  int gy = (int)std::min<long long>(64, (cnt + NT - 1) / NT);
  if (gy < 1) gy = 1;
  add_copy_kernel<<<dim3(ntasks, gy), NT, 0, s>>>(d);
  H2_LAUNCH_CHECK();
}

void launch_interp(Prec p, const InterpTask* d, int ntasks, cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("interp", s);
  if (p == Prec::F64) interp_kernel<double><<<ntasks, NT, 0, s>>>(d);
  else interp_kernel<float><<<ntasks, NT, 0, s>>>(d);
  H2_LAUNCH_CHECK();
}

void launch_colnorm2(const double* X, int n, int nrhs, int64_t ld, double* out, cudaStream_t s) {
  if (nrhs <= 0) return;
  ProfScope ps("colnorm", s);
  colnorm2_kernel<<<nrhs, NT, 0, s>>>(X, n, nrhs, ld, out);
  H2_LAUNCH_CHECK();
}

void launch_axpy_cols(double* Y, const double* X, int n, int nrhs, int64_t ldy, int64_t ldx, double alpha,
                      cudaStream_t s) {
  long long cnt = (long long)n * nrhs;
  if (cnt <= 0) return;
  ProfScope ps("axpy", s);
  int g = (int)std::min<long long>(152 * 8, (cnt + NT - 1) / NT);
  axpy_cols_kernel<<<g, NT, 0, s>>>(Y, X, n, nrhs, ldy, ldx, alpha);
  H2_LAUNCH_CHECK();
}

void launch_permute_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* map,
                         int64_t n, int nrhs, bool scatter, cudaStream_t s) {
  long long cnt = (long long)n * nrhs;
  if (cnt <= 0) return;
  ProfScope ps("permute", s);
  int g = (int)std::min<long long>(152 * 8, (cnt + NT - 1) / NT);
  permute_rows_kernel<<<g, NT, 0, s>>>(src, lds, dst, ldd, map, n, nrhs, scatter);
  H2_LAUNCH_CHECK();
}

constexpr int MDOT_BLOCKS = 152 * 4;
void launch_mdot(const double* V, int64_t ldv, int kvec, const double* w, int64_t n, double* partial, double* out,
                 cudaStream_t s) {
  if (kvec <= 0) return;
  if (kvec > MDOT_MAXK) throw StatusError(1, "mdot: more than 32 vectors");
  ProfScope ps("mdot_f64", s);
  mdot_partial_kernel<<<MDOT_BLOCKS, NT, 0, s>>>(V, ldv, kvec, w, n, partial);
  mdot_reduce_kernel<<<1, 32, 0, s>>>(partial, MDOT_BLOCKS, kvec, out);
  H2_LAUNCH_CHECK();
}

void launch_normalize(double* v, const double* w, int64_t n, const double* norm2, cudaStream_t s) {
  ProfScope ps("normalize", s);
  int g = (int)std::min<long long>(152 * 8, (n + NT - 1) / NT);
  normalize_kernel<<<g, NT, 0, s>>>(v, w, n, norm2);
  H2_LAUNCH_CHECK();
}

void launch_gather_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int* idx, int64_t n, int nrhs,
                        cudaStream_t s) {
  long long cnt = (long long)n * nrhs;
  if (cnt <= 0) return;
  ProfScope ps("gather_rows", s);
  int g = (int)std::min<long long>(152 * 8, (cnt + NT - 1) / NT);
  gather_rows_kernel<<<g, NT, 0, s>>>(src, lds, dst, ldd, idx, n, nrhs);
  H2_LAUNCH_CHECK();
}

void launch_fill_eye(Prec p, void* A, int n, int ld, cudaStream_t s) {
  ProfScope ps("eye", s);
  long long cnt = (long long)n * n;
  int g = (int)std::min<long long>(152 * 8, (cnt + NT - 1) / NT);
  if (p == Prec::F64) eye_kernel<double><<<g, NT, 0, s>>>((double*)A, n, ld);
  else eye_kernel<float><<<g, NT, 0, s>>>((float*)A, n, ld);
  H2_LAUNCH_CHECK();
}

__global__ void add_offset_kernel(int* p, int n, int k) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] += k;
}

void launch_add_offset(int* p, int n, int k, cudaStream_t s) {
  if (n <= 0) return;
  ProfScope ps("piv_offset", s);
  add_offset_kernel<<<(n + NT - 1) / NT, NT, 0, s>>>(p, n, k);
  H2_LAUNCH_CHECK();
}

void launch_laswp_cols(Prec p, void* A, int lda, int ncols, const int* piv, int k0, int k1, int cb, int ce,
                       cudaStream_t s) {
  (void)ncols;
  if (ce <= cb || k1 <= k0) return;
  ProfScope ps("laswp", s);
  int g = std::min(152 * 4, (ce - cb + NT - 1) / NT);
  if (p == Prec::F64) laswp_kernel<double><<<g, NT, 0, s>>>((double*)A, lda, piv, k0, k1, cb, ce);
  else laswp_kernel<float><<<g, NT, 0, s>>>((float*)A, lda, piv, k0, k1, cb, ce);
  H2_LAUNCH_CHECK();
}

// dst += parts in list order, element by element (a fixed summation order)
template <typename T>
__global__ void __launch_bounds__(NT) accum_parts_kernel(const AccumTask* __restrict__ tasks,
                                                         const void* const* __restrict__ parts) {
  const AccumTask tk = tasks[blockIdx.x];
  T* dst = reinterpret_cast<T*>(tk.dst);
  for (long long e = (long long)blockIdx.y * NT + threadIdx.x; e < tk.n; e += (long long)gridDim.y * NT) {
    T s = dst[e];
    for (int q = tk.p0; q < tk.p0 + tk.np; ++q) s += reinterpret_cast<const T*>(parts[q])[e];
    dst[e] = s;
  }
}

void launch_accum_parts(Prec p, const AccumTask* d, int ntasks, const void* const* parts, long long maxn,
                        cudaStream_t s) {
  if (ntasks <= 0 || maxn <= 0) return;
  ProfScope ps(p == Prec::F64 ? "accum_f64" : "accum_f32", s);
  dim3 grid(ntasks, (unsigned)std::min<long long>(64, (maxn + NT - 1) / NT));
  if (p == Prec::F64) accum_parts_kernel<double><<<grid, NT, 0, s>>>(d, parts);
  else accum_parts_kernel<float><<<grid, NT, 0, s>>>(d, parts);
  H2_LAUNCH_CHECK();
}

void launch_logdet_lu(const LuTask* d, int ntasks, double* out_log, double* out_sign, bool cholesky,
                      cudaStream_t s) {
  if (ntasks <= 0) return;
  ProfScope ps("logdet", s);
  logdet_kernel<<<ntasks, NT, 0, s>>>(d, out_log, out_sign, cholesky);
  H2_LAUNCH_CHECK();
}

}  // namespace h2
