// Tensor-core (tcgen05, sm_103a) batched segmented GEMM in split 3xTF32:
//   C = alpha * sum_t op(A_t) op(B_t) + beta * Cin     (FP32 data)
// Each FP32 operand element a is split into a_hi = tf32(a) (low 13 mantissa
// bits cleared) and a_lo = a - a_hi, and the product is accumulated as
// A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 in tensor memory, which keeps
// close to FP32 accuracy (the dropped A_lo B_lo term is ~2^-22 relative).
//
// One CTA computes a 128 x 128 output tile of one task.  Operands are
// staged by the CTA itself (per-term transposition, bounds and the hi/lo
// split happen in the load path) into the canonical no-swizzle K-major
// shared-memory layout: 8-row x 16-byte core matrices, core matrices
// adjacent along K at LBO = 128 bytes, 8-row groups at SBO = (BK/4)*128.
// One elected thread issues tcgen05.mma (kind::tf32, M = 128, N = 128,
// K = 8 per instruction) into a 128-column TMEM accumulator; completion is
// tracked with tcgen05.commit on an mbarrier whose waits are bounded.  The
// epilogue reads TMEM with tcgen05.ld.32x32b.
#include "h2_common.cuh"
#include "h2_prof.h"

namespace h2 {

namespace {

constexpr int TM = 128, TN = 128, BK = 32, NTH = 256;
constexpr int SBO = (BK / 4) * 128;                // bytes between 8-row groups
constexpr int TILE_BYTES = TM * BK * 4;            // one operand tile (A or B), 16 KB
constexpr long long SPIN_LIMIT = 1ll << 26;        // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) in a canonical no-swizzle K-major tile
__device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
  return (uint32_t)((row & 7) * 16 + (row >> 3) * SBO + (k >> 2) * 128 + (k & 3) * 4);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);               // start address
  d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;          // leading byte offset (along K)
  d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;          // stride byte offset (8-row groups)
  d |= (uint64_t)1 << 46;                              // descriptor version (sm_100 family)
  // base offset 0, lbo mode 0, layout type 0 = no swizzle
  return d;
}

// instruction descriptor: D = F32, A = B = TF32, both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t instr_desc() {
  uint32_t d = 0;
  d |= 1u << 4;                 // c_format = F32
  d |= 2u << 7;                 // a_format = TF32
  d |= 2u << 10;                // b_format = TF32
  d |= (uint32_t)(TN >> 3) << 17;
  d |= (uint32_t)(TM >> 4) << 24;
  return d;
}

__device__ __forceinline__ float tf32_hi(float a) {
  return __uint_as_float(__float_as_uint(a) & 0xFFFFE000u);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  uint32_t addr = smem_u32(bar);
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(phase));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

template <typename TIN>
__device__ __forceinline__ float ldg(const void* p, long long idx) {
  return (float)reinterpret_cast<const TIN*>(p)[idx];
}

template <typename TIN>
__global__ void __launch_bounds__(NTH, 1) tc_gemm_kernel(const GemmTask* __restrict__ tasks,
                                                         const GemmTerm* __restrict__ terms, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  // 4 operand tiles (A_hi, A_lo, B_hi, B_lo), 1024-byte aligned
  unsigned char* base = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
  unsigned char* sAhi = base;
  unsigned char* sAlo = base + TILE_BYTES;
  unsigned char* sBhi = base + 2 * TILE_BYTES;
  unsigned char* sBlo = base + 3 * TILE_BYTES;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const GemmTask tk = tasks[blockIdx.x];
  const int tiles_m = (tk.M + TM - 1) / TM;
  const int tiles_n = (tk.N + TN - 1) / TN;
  const int tile = blockIdx.y;
  if (tile >= tiles_m * tiles_n) return;
  const int i0 = (tile % tiles_m) * TM, j0 = (tile / tiles_m) * TN;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    mbar_init(&mbar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc();
  uint32_t phase = 0;
  bool first = true;

  for (int t = tk.t0; t < tk.t0 + tk.nt && !s_fail; ++t) {
    const GemmTerm tm = terms[t];
    const bool TRA = (tm.flags & 1) != 0, TRB = (tm.flags & 2) != 0;
    for (int k0 = 0; k0 < tm.K; k0 += BK) {
      // ---- stage op(A)[i0:i0+128, k0:k0+32] and op(B)^T[j0:j0+128, k0:k0+32]
      for (int e = tid; e < TM * BK; e += NTH) {
        int r, k;
        if (!TRA) { r = e % TM; k = e / TM; } else { k = e % BK; r = e / BK; }
        int gi = i0 + r, gk = k0 + k;
        float v = 0.f;
        if (gi < tk.M && gk < tm.K)
          v = TRA ? ldg<TIN>(tm.A, (long long)gk + (long long)gi * tm.lda)
                  : ldg<TIN>(tm.A, (long long)gi + (long long)gk * tm.lda);
        float hi = tf32_hi(v);
        uint32_t o = kmaj_off(r, k);
        *reinterpret_cast<float*>(sAhi + o) = hi;
        *reinterpret_cast<float*>(sAlo + o) = v - hi;
      }
      for (int e = tid; e < TN * BK; e += NTH) {
        int r, k;
        if (TRB) { r = e % TN; k = e / TN; } else { k = e % BK; r = e / BK; }
        int gj = j0 + r, gk = k0 + k;
        float v = 0.f;
        if (gj < tk.N && gk < tm.K)
          v = TRB ? ldg<TIN>(tm.B, (long long)gj + (long long)gk * tm.ldb)
                  : ldg<TIN>(tm.B, (long long)gk + (long long)gj * tm.ldb);
        float hi = tf32_hi(v);
        uint32_t o = kmaj_off(r, k);
        *reinterpret_cast<float*>(sBhi + o) = hi;
        *reinterpret_cast<float*>(sBlo + o) = v - hi;
      }
      // make the generic-proxy smem writes visible to the tensor core
      asm volatile("fence.proxy.async.shared::cta;");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t aH = smem_u32(sAhi), aL = smem_u32(sAlo), bH = smem_u32(sBhi), bL = smem_u32(sBlo);
#pragma unroll
        for (int ks = 0; ks < BK / 8; ++ks) {
          const uint32_t off = ks * 2 * 128;   // K = 8 tf32 = two 16-byte core-matrix columns
          mma_tf32(tmem, smem_desc(aH + off), smem_desc(bH + off), idesc, first ? 0u : 1u);
          first = false;
          mma_tf32(tmem, smem_desc(aH + off), smem_desc(bL + off), idesc, 1u);
          mma_tf32(tmem, smem_desc(aL + off), smem_desc(bH + off), idesc, 1u);
        }
        mma_commit(&mbar);
      }
      first = false;
      __syncthreads();
      // wait for the MMAs to finish reading shared memory (bounded)
      bool ok = mbar_wait(&mbar, phase);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (!ok) {
        if (tid == 0) {
          s_fail = 1;
          atomicExch(err, 1);
        }
      }
      __syncthreads();
      if (s_fail) break;
    }
  }

  // ---- epilogue: TMEM -> registers -> global (warps 0-3 and 4-7 split the columns)
  if (!s_fail && !first) {
    const int lane_grp = warp & 3;          // TMEM lanes 32*lane_grp .. +31
    const int col_half = warp >> 2;         // columns [0,64) or [64,128)
    const int row = i0 + lane_grp * 32 + lane;
    float* C = reinterpret_cast<float*>(tk.C);
    const float* Cin = reinterpret_cast<const float*>(tk.Cin);
#pragma unroll 1
    for (int c0 = col_half * 64; c0 < col_half * 64 + 64; c0 += 8) {
      uint32_t r[8];
      uint32_t taddr = tmem + ((uint32_t)(lane_grp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (row < tk.M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          int col = j0 + c0 + q;
          if (col < tk.N) {
            float v = (float)tk.alpha * __uint_as_float(r[q]);
            if (Cin != nullptr && tk.beta != 0.0) v += (float)tk.beta * Cin[row + (long long)col * tk.ldcin];
            C[row + (long long)col * tk.ldc] = v;
          }
        }
      }
    }
  } else if (!s_fail && first) {
    // task without terms: C = beta * Cin
    float* C = reinterpret_cast<float*>(tk.C);
    const float* Cin = reinterpret_cast<const float*>(tk.Cin);
    for (int e = tid; e < TM * TN; e += NTH) {
      int r = i0 + e % TM, c = j0 + e / TM;
      if (r < tk.M && c < tk.N) {
        float v = 0.f;
        if (Cin != nullptr && tk.beta != 0.0) v = (float)tk.beta * Cin[r + (long long)c * tk.ldcin];
        C[r + (long long)c * tk.ldc] = v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TN));
  }
}

}  // namespace

static int* tc_err_flag() {
  static int* p = nullptr;
  if (!p) {
    H2_CUDA(cudaMalloc(&p, sizeof(int)));
    H2_CUDA(cudaMemset(p, 0, sizeof(int)));
  }
  return p;
}

void launch_gemm_tc(const GemmTask* d_tasks, const GemmTerm* d_terms, int ntasks, int maxM, int maxN,
                    cudaStream_t s) {
  if (ntasks <= 0 || maxM <= 0 || maxN <= 0) return;
  const size_t smem = 4 * TILE_BYTES + 1024;
  H2_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(ntasks, ((maxM + TM - 1) / TM) * ((maxN + TN - 1) / TN));
  ProfScope ps("gemm_tc3xtf32", s);
  tc_gemm_kernel<float><<<grid, NTH, smem, s>>>(d_tasks, d_terms, tc_err_flag());
  H2_LAUNCH_CHECK();
}

int tc_error_flag_read_and_clear(cudaStream_t s) {
  int v = 0;
  int* p = tc_err_flag();
  H2_CUDA(cudaMemcpyAsync(&v, p, sizeof(int), cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  if (v) H2_CUDA(cudaMemsetAsync(p, 0, sizeof(int), s));
  return v;
}

}  // namespace h2
