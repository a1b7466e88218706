// Shared device definitions of the H^2-ULV CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdexcept>
#include <string>
#include <vector>

namespace h2 {

// ---------------------------------------------------------------------------
// Error handling: CUDA errors become C++ exceptions inside the library and a
// status code at the C ABI.
// ---------------------------------------------------------------------------
struct CudaError : std::runtime_error {
  explicit CudaError(const std::string& s) : std::runtime_error(s) {}
};
struct StatusError : std::runtime_error {
  int status;
  StatusError(int st, const std::string& s) : std::runtime_error(s), status(st) {}
};

#define H2_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      throw ::h2::CudaError(std::string(#call) + ": " + cudaGetErrorString(e_) +      \
                            " at " + __FILE__ + ":" + std::to_string(__LINE__));       \
  } while (0)

#define H2_LAUNCH_CHECK() H2_CUDA(cudaGetLastError())

// ---------------------------------------------------------------------------
// Kernel functions (Sec. IV Laplace Green's function, Sec. V Yukawa), with
// the point singularity regularised by delta; Matern-3/2 for covariances.
// ---------------------------------------------------------------------------
struct KParams {
  int kind;  // 0 laplace, 1 yukawa, 2 matern32
  double delta, kappa, ell, nugget;
};

__device__ __forceinline__ double kernel_eval(const KParams& kp, double dx, double dy, double dz) {
  double r2 = dx * dx + dy * dy + dz * dz;
  double r = sqrt(r2);
  if (kp.kind == 0) return 1.0 / (r + kp.delta);
  if (kp.kind == 1) return exp(-kp.kappa * r) / (r + kp.delta);
  double s = 1.7320508075688772 * r / kp.ell;
  double v = (1.0 + s) * exp(-s);
  return r2 == 0.0 ? v + kp.nugget : v;
}

__device__ __forceinline__ float kernel_eval_f(const KParams& kp, double dx, double dy, double dz) {
  // coordinate differences in FP64 (close points keep their relative
  // accuracy), the rest in FP32
  float r2 = (float)(dx * dx + dy * dy + dz * dz);
  float r = sqrtf(r2);
  if (kp.kind == 0) return 1.0f / (r + (float)kp.delta);
  if (kp.kind == 1) return expf(-(float)kp.kappa * r) / (r + (float)kp.delta);
  float s = 1.7320508f * r / (float)kp.ell;
  float v = (1.0f + s) * expf(-s);
  return r2 == 0.0f ? v + (float)kp.nugget : v;
}

// FP32 throughout, for well-separated points only (far-field samples), whose
// coordinate differences lose no relative accuracy to FP32 rounding
__device__ __forceinline__ float kernel_eval_ff(const KParams& kp, float dx, float dy, float dz) {
  float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  float r = sqrtf(r2);
  if (kp.kind == 0) return 1.0f / (r + (float)kp.delta);
  if (kp.kind == 1) return expf(-(float)kp.kappa * r) / (r + (float)kp.delta);
  float s = 1.7320508f * r / (float)kp.ell;
  float v = (1.0f + s) * expf(-s);
  return r2 == 0.0f ? v + (float)kp.nugget : v;
}

template <typename T> struct KEval;
template <> struct KEval<double> {
  static __device__ __forceinline__ double eval(const KParams& kp, double dx, double dy, double dz) {
    return kernel_eval(kp, dx, dy, dz);
  }
};
template <> struct KEval<float> {
  static __device__ __forceinline__ float eval(const KParams& kp, double dx, double dy, double dz) {
    return kernel_eval_f(kp, dx, dy, dz);
  }
};

// Largest box size in level coordinates: a leaf holds at most 256 points and
// a parent box the skeletons of its two children, r_a + r_b <= 2 * 256.
constexpr int NMAX = 512;

// Tree-order points, structure of arrays.
struct Points {
  const double* x;
  const double* y;
  const double* z;
};

// ---------------------------------------------------------------------------
// Task descriptors of the batched kernels.  Matrices are column-major.
// ---------------------------------------------------------------------------
struct GemmTerm {
  const void* A;
  const void* B;
  int K, lda, ldb;
  int flags;          // bit 0: op(A) = A^T, bit 1: op(B) = B^T
};
struct GemmTask {
  void* C;            // output
  const void* Cin;    // beta * Cin is added (may alias C); null = no beta term
  int M, N, ldc, ldcin;
  int t0, nt;         // terms [t0, t0+nt)
  double alpha, beta;
};

struct LuTask {        // in-place LU with partial pivoting of an m x nc panel
  void* A;
  int m, nc, lda;
  int* piv;            // nc pivots (0-based row index within the panel)
  int* info;           // set to k+1 at the first zero pivot (if non-null)
  int spd;             // 1: no pivoting, every pivot must be > 0 (symmetric positive definite)
};

struct TrsmTask {      // B <- op(A)^-1 B, A n x n triangular, B n x nrhs
  const void* A;
  void* B;
  int n, nrhs, lda, ldb;
  const int* piv;      // row interchanges applied to B first (getrs), or null
};

struct CholTask {      // pivoted Cholesky of an n x n Gram matrix (G is read only)
  double* G;
  int n, ldg;
  int* piv;            // n
  double* R;           // n x n, ld n: rows 0..rank-1 hold R
  int* rank;
  double tol;
  int max_rank;
  int* info;           // set to 1 if a non-finite value is met (may be null)
  double* L;           // n x n scratch (the factor column by column)
};

struct PqrTask {       // Householder QR with column pivoting of an m x n matrix
  double* A;
  int m, n, lda;
  int* piv;
  double* R;           // n x n, ld n
  int* rank;
  double tol;
  int max_rank;
  int* info;           // set to 1 if a non-finite column norm is met (may be null)
};

struct HqrTask {       // QR of M (n x r): Q = [U^R U^S] (n x n), W (r x r)
  void* M;             // n x r, ld n, destroyed
  void* V;             // scratch n x r, ld n
  void* Q;             // n x n, ld n
  void* W;             // r x r, ld r
  int n, r;
};

struct FoldTerm {      // explicit rows of B^T: row q (< rows), element j (< n)
  const double* X;     // tr = 0: X[j + q ld] (rows are columns of X); tr = 1: X[q + j ld]
  int rows, ld, tr;
};
struct FoldTask {      // R (n x n upper) <- triangle of [R; rows of the terms; K(cand, samples)^T]
  const int* cand;     // n point indices (read when m > 0)
  const int* samp;     // m point indices
  double* R;           // n x n, ld n
  int n, m;
  int t0, nt;          // explicit-row terms [t0, t0 + nt), folded first
  int accumulate;      // 0: start from R = 0; 1: continue from the R in memory
};

struct KgramTask {     // G (+)= K(cand, samp) K(cand, samp)^T
  const int* cand;
  const int* samp;
  double* G;
  int n, m, ldg;
  int accumulate;
};

struct AsmTask {       // out(i, j) = K(x[ridx[i]], x[cidx[j]])
  void* out;
  const int* ridx;     // null = contiguous from r0
  const int* cidx;     // null = contiguous from c0
  int r0, c0, nr, nc, ld;
};

struct CopyTask {      // dst(i, j) = src(i, j) or src(j, i) (transpose)
  const void* src;
  void* dst;
  int rows, cols, lds, ldd;
};

struct InterpTask {    // P (n x r) from piv, T = R11^-1 R12 (r x (n-r), ld ldt)
  const int* piv;
  const void* T;
  void* P;
  int n, r, ldt;
};

struct SymPairTask {   // stored block (I, J), I <= J: partials u (box I) and v (box J)
  const void* A;
  int nI, nJ, lda;
  long long sI, sJ;    // tree-order starts of the boxes' rows in x
  long long uo, vo;    // element offsets of u (nI x nrhs) and v (nJ x nrhs) in the partial buffer
};
struct AccumTask {     // dst[0:n] += parts[p0], then += parts[p0+1], ... (in order)
  void* dst;
  long long n;
  int p0, np;
};

struct GatherTask {    // y[s : s+n] = sum of partials p0 .. p0+np-1
  long long s;
  int n, p0, np;
};

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the k_*.cu files).  Each takes a device array
// of tasks plus a host-side count and maxima for the grid.
// ---------------------------------------------------------------------------
enum class Prec { F64 = 0, F32 = 1 };

// Terms carry their own transposition flags (GemmTerm::flags).  ksum = the
// largest summed K of a task (selects the autotuned kernel for FP32 data).
void launch_gemm(Prec p, const GemmTask* d_tasks, const GemmTerm* d_terms,
                 int ntasks, int maxM, int maxN, cudaStream_t s, bool inputs_f64 = false, int ksum = 0);
std::string autotune_report();
void launch_getrf(Prec p, const LuTask* d, int ntasks, int maxm, cudaStream_t s);
void launch_trsm(Prec p, bool lower, bool unit, bool transA, const TrsmTask* d, int ntasks,
                 int maxnrhs, int maxn, cudaStream_t s);
void launch_pchol(const CholTask* d, int ntasks, cudaStream_t s);
void launch_pqr(const PqrTask* d, int ntasks, cudaStream_t s);
void launch_hqr(Prec p, const HqrTask* d, int ntasks, cudaStream_t s);
void launch_fold(const FoldTask* d, int ntasks, int maxn, const FoldTerm* terms, Points pts, KParams kp,
                 cudaStream_t s);
void launch_kgram(Prec p, const KgramTask* d, int ntasks, int maxn, Points pts, KParams kp,
                  cudaStream_t s);
void launch_assemble(Prec p, const AsmTask* d, int ntasks, int maxr, int maxc, Points pts,
                     KParams kp, cudaStream_t s);
void launch_copy(Prec src, Prec dst, bool transpose, const CopyTask* d, int ntasks, int maxr,
                 int maxc, cudaStream_t s);
void launch_interp(Prec p, const InterpTask* d, int ntasks, cudaStream_t s);
// FP32 far-field block rows (ridx: the box's points, at most NMAX; cidx: far samples)
void launch_assemble_far_f32(const AsmTask* d, int ntasks, int maxc, Points pts, KParams kp, cudaStream_t s);
// dst += src for FP32 src and FP64 dst blocks (CopyTask layout)
void launch_add_copy(const CopyTask* d, int ntasks, int maxr, int maxc, cudaStream_t s);
void launch_colnorm2(const double* X, int n, int nrhs, int64_t ld, double* out, cudaStream_t s);
void launch_axpy_cols(double* Y, const double* X, int n, int nrhs, int64_t ldy, int64_t ldx,
                      double alpha, cudaStream_t s);
void launch_permute_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int64_t* map,
                         int64_t n, int nrhs, bool scatter, cudaStream_t s);
// out[i] = <V_i, w> for i < kvec <= 32 (V_i = V + i*ldv); partial needs 608*32 doubles
void launch_mdot(const double* V, int64_t ldv, int kvec, const double* w, int64_t n, double* partial, double* out,
                 cudaStream_t s);
void launch_normalize(double* v, const double* w, int64_t n, const double* norm2, cudaStream_t s);
void launch_gather_rows(const double* src, int64_t lds, double* dst, int64_t ldd, const int* idx, int64_t n, int nrhs,
                        cudaStream_t s);
void launch_fill_eye(Prec p, void* A, int n, int ld, cudaStream_t s);
// p[0:n] += k (block-relative pivots of a panel LU to absolute rows)
void launch_add_offset(int* p, int n, int k, cudaStream_t s);
void launch_laswp_cols(Prec p, void* A, int lda, int ncols, const int* piv, int k0, int k1,
                       int col_begin, int col_end, cudaStream_t s);
void launch_symv_pairs(const SymPairTask* d, int ntasks, const double* x, int64_t ldx, double* part, int nrhs,
                       cudaStream_t s);
void launch_accum_parts(Prec p, const AccumTask* d, int ntasks, const void* const* parts, long long maxn,
                        cudaStream_t s);
// symv_pairs with one right-hand side writes (hi, lo) FP32 pairs into the
// 8-byte partial slots, and gather_parts with one right-hand side reads them
// that way; with two right-hand sides both use FP64 partials.
void launch_gather_parts(const GatherTask* d, int ntasks, const long long* offs, const double* part, double* y,
                         int64_t ldy, int nrhs, cudaStream_t s);
int tc_error_flag_read_and_clear(cudaStream_t s);
void launch_logdet_lu(const LuTask* d, int ntasks, double* out_log, double* out_sign,
                      bool cholesky, cudaStream_t s);

}  // namespace h2
