// Tensor-core (tcgen05, sm_103a) batched segmented GEMM in split 3xTF32:
//   C = alpha * sum_t op(A_t) op(B_t) + beta * Cin     (FP32 data)
// Each FP32 operand element a is split into a_hi = tf32(a) (low 13 mantissa
// bits cleared) and a_lo = a - a_hi, and the product is accumulated as
// A_hi B_hi + A_hi B_lo + A_lo B_hi in FP32 in tensor memory, which keeps
// close to FP32 accuracy (the dropped A_lo B_lo term is ~2^-22 relative).
//
// One CTA computes a 128 x 256 output tile of one task (MMA N sized to the
// task, a multiple of 16), or a 128 x 128 tile when no output of the launch
// is wider than 128 columns.  Operands are staged by the CTA itself
// (per-term transposition, bounds and the hi/lo split happen in the load
// path) into the canonical no-swizzle K-major shared-memory layout: 8-row x
// 16-byte core matrices, adjacent along K at LBO = 128 bytes, 8-row groups
// at SBO = (BK/4)*128; each thread writes whole 16-byte core-matrix rows.
// A register prefetch of the next K-chunk overlaps the global loads with the
// tensor core; one shared-memory stage (96 KB) and at most 128 registers per
// thread let two CTAs share an SM, so one CTA's MMA wait is covered by the
// other's staging.  One elected thread issues
// tcgen05.mma (kind::tf32, M = 128, K = 8 per instruction) into a
// 256-column TMEM accumulator; completion is tracked per stage with
// tcgen05.commit on mbarriers, waited for (bounded) by one thread while the
// others sleep in a CTA barrier.  The epilogue reads
// TMEM with tcgen05.ld.32x32b.
#include "h2_common.cuh"
#include "h2_prof.h"

namespace h2 {

namespace {

constexpr int TM = 128, BK = 32, NTH = 256;
constexpr int SBO = (BK / 4) * 128;                // bytes between 8-row groups
constexpr long long SPIN_LIMIT = 1ll << 26;        // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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


// Staging: an operand tile is R rows x BK k; its 16-byte units (one row, 4
// consecutive k) are distributed so that each thread owns whole units and
// writes them with one 16-byte shared store.  A 16-byte store is served per
// quarter warp, so every group of 8 consecutive lanes must write 8 different
// rows of one core matrix (128 contiguous bytes) to be free of bank
// conflicts.  Two mappings keep that property: "row-fast" (consecutive lanes
// take consecutive rows; global loads coalesce when the operand is
// contiguous along rows) and "k-fast" (a warp covers 8 rows x 16 k, each row
// read as 64 contiguous bytes, for operands contiguous along k).
template <int R>
struct Stage {
  static constexpr int UNITS = R * (BK / 4);
  static constexpr int PER = UNITS / NTH;      // units per thread
  float v[PER][4];
};

template <int R>
__device__ __forceinline__ void unit_coords(int u, bool contig_k, int& row, int& kc) {
  if (contig_k) {
    const int w = u >> 5;                      // 32-unit group: 8 rows x 4 units of k
    row = (u & 7) + 8 * (w >> 1);
    kc = ((u >> 3) & 3) + 4 * (w & 1);
  } else {
    row = u % R;
    kc = u / R;
  }
}

// element (row, k) of op(X) with X column-major: rowmajor_k = true means
// op(X)(row, k) = X[k + row*ld] (contiguous along k), else X[row + k*ld]
template <int R>
__device__ __forceinline__ void stage_load(Stage<R>& st, const float* X, long long ld, bool contig_k, int row0,
                                           int rows, int k0, int K) {
  const int tid = threadIdx.x;
  // 16-byte vector loads along k when every unit start is 16-byte aligned
  const bool vec = contig_k && ((reinterpret_cast<uintptr_t>(X) & 15) == 0) && ((ld & 3) == 0) && ((k0 & 3) == 0);
#pragma unroll
  for (int q = 0; q < Stage<R>::PER; ++q) {
    const int u = tid + q * NTH;
    int row, kc;
    unit_coords<R>(u, contig_k, row, kc);
    const int gr = row0 + row;
    const int gk = k0 + kc * 4;
    if (vec && gr < rows && gk + 3 < K) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(X + gk + (long long)gr * ld));
      st.v[q][0] = t.x;
      st.v[q][1] = t.y;
      st.v[q][2] = t.z;
      st.v[q][3] = t.w;
      continue;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float v = 0.f;
      if (gr < rows && gk + j < K) v = contig_k ? X[(gk + j) + (long long)gr * ld] : X[gr + (long long)(gk + j) * ld];
      st.v[q][j] = v;
    }
  }
}

template <int R>
__device__ __forceinline__ void stage_store(const Stage<R>& st, bool contig_k, unsigned char* hi, unsigned char* lo) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < Stage<R>::PER; ++q) {
    const int u = tid + q * NTH;
    int row, kc;
    unit_coords<R>(u, contig_k, row, kc);
    const uint32_t o = (uint32_t)((row & 7) * 16 + (row >> 3) * SBO + kc * 128);
    float4 h, l;
    h.x = tf32_hi(st.v[q][0]); l.x = st.v[q][0] - h.x;
    h.y = tf32_hi(st.v[q][1]); l.y = st.v[q][1] - h.y;
    h.z = tf32_hi(st.v[q][2]); l.z = st.v[q][2] - h.z;
    h.w = tf32_hi(st.v[q][3]); l.w = st.v[q][3] - h.w;
    *reinterpret_cast<float4*>(hi + o) = h;
    *reinterpret_cast<float4*>(lo + o) = l;
  }
}

constexpr int TNB = 256;                              // output tile columns (TMEM columns)
constexpr int ABYTES = TM * BK * 4, BBYTES = TNB * BK * 4;
constexpr int STAGE_BYTES = 2 * ABYTES + 2 * BBYTES;  // hi + lo of A and B
constexpr int NSTAGE = 1;

__device__ __forceinline__ uint32_t instr_desc_n(int n_mma) {
  uint32_t d = 0;
  d |= 1u << 4;
  d |= 2u << 7;
  d |= 2u << 10;
  d |= (uint32_t)(n_mma >> 3) << 17;
  d |= (uint32_t)(TM >> 4) << 24;
  return d;
}

// TNB_ = 256: one 128 x 256 output tile per CTA; TNB_ = 128 (launches whose
// outputs are at most 128 columns wide, e.g. the r-wide projections): a
// 128 x 128 tile with half the B staging, TMEM and shared memory.
template <int TNB_>
__global__ void __launch_bounds__(NTH, TNB_ == 128 ? 3 : 2) tc_gemm_kernel(const GemmTask* __restrict__ tasks,
                                                         const GemmTerm* __restrict__ terms, int* err) {
  constexpr int BBYTES_ = TNB_ * BK * 4;
  constexpr int STAGE_ = 2 * ABYTES + 2 * BBYTES_;
  constexpr int CHALF = TNB_ / 2;                      // epilogue columns per warp group
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* base = smem + ((1024 - (smem_u32(smem) & 1023)) & 1023);
  __shared__ uint64_t mbar[NSTAGE];
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const GemmTask tk = tasks[blockIdx.x];
  const int tiles_m = (tk.M + TM - 1) / TM;
  const int tiles_n = (tk.N + TNB_ - 1) / TNB_;
  const int tile = blockIdx.y;
  if (tile >= tiles_m * tiles_n) return;
  const int i0 = (tile % tiles_m) * TM, j0 = (tile / tiles_m) * TNB_;
  const int ncols = min(TNB_, tk.N - j0);
  const int n_mma = ((ncols + 15) / 16) * 16;          // MMA N: multiple of 16, <= 256
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(TNB_));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < NSTAGE; ++q) mbar_init(&mbar[q], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = instr_desc_n(n_mma);

  // flatten (term, k-chunk) pairs
  int nchunks = 0;
  for (int t = tk.t0; t < tk.t0 + tk.nt; ++t) nchunks += (terms[t].K + BK - 1) / BK;

  Stage<TM> ra;
  Stage<TNB_> rb;
  int cur_t = tk.t0, cur_k = 0;
  GemmTerm tm{};
  auto load_chunk = [&](int t, int k0) {
    const GemmTerm g = terms[t];
    const bool TRA = (g.flags & 1) != 0, TRB = (g.flags & 2) != 0;
    // op(A)(i, k): TRA -> A[k + i*lda] (contiguous along k)
    stage_load<TM>(ra, reinterpret_cast<const float*>(g.A), g.lda, TRA, i0, tk.M, k0, g.K);
    // B operand rows are output columns n: op(B)(k, n) = TRB ? B[n + k*ldb] : B[k + n*ldb]
    stage_load<TNB_>(rb, reinterpret_cast<const float*>(g.B), g.ldb, !TRB, j0, tk.N, k0, g.K);
  };
  bool contigA = false, contigB = false;
  if (nchunks > 0) {
    // first term with K > 0
    while (cur_t < tk.t0 + tk.nt && terms[cur_t].K <= 0) ++cur_t;
    tm = terms[cur_t];
    contigA = (tm.flags & 1) != 0;
    contigB = (tm.flags & 2) == 0;
    load_chunk(cur_t, 0);
  }
  uint32_t phase[NSTAGE] = {};
  int committed = 0;                                   // chunks whose MMAs were committed (thread 0)
  for (int c = 0; c < nchunks; ++c) {
    const int st = c % NSTAGE;
    unsigned char* sA_hi = base + st * STAGE_;
    unsigned char* sA_lo = sA_hi + ABYTES;
    unsigned char* sB_hi = sA_lo + ABYTES;
    unsigned char* sB_lo = sB_hi + BBYTES_;
    if (c >= NSTAGE) {
      // the MMAs of chunk c - NSTAGE read this stage: one thread waits for
      // them (bounded), the others sleep in the barrier instead of polling
      if (tid == 0 && !s_fail && !mbar_wait(&mbar[st], phase[st])) {
        s_fail = 1;
        atomicExch(err, 1);
      }
      phase[st] ^= 1u;
      __syncthreads();
    }
    stage_store<TM>(ra, contigA, sA_hi, sA_lo);
    stage_store<TNB_>(rb, contigB, sB_hi, sB_lo);
    // prefetch the next chunk into registers while the tensor core works
    {
      int nt = cur_t, nk = cur_k + BK;
      if (nk >= terms[cur_t].K) {
        nt = cur_t + 1;
        nk = 0;
        while (nt < tk.t0 + tk.nt && terms[nt].K <= 0) ++nt;
      }
      if (c + 1 < nchunks) {
        load_chunk(nt, nk);
        const GemmTerm g = terms[nt];
        // remember the layouts of the prefetched chunk for its store
        cur_t = nt;
        cur_k = nk;
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0 && !s_fail) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t aH = smem_u32(sA_hi), aL = smem_u32(sA_lo), bH = smem_u32(sB_hi), bL = smem_u32(sB_lo);
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint32_t off = ks * 2 * 128;
            mma_tf32(tmem, smem_desc(aH + off), smem_desc(bH + off), idesc, (c == 0 && ks == 0) ? 0u : 1u);
            mma_tf32(tmem, smem_desc(aH + off), smem_desc(bL + off), idesc, 1u);
            mma_tf32(tmem, smem_desc(aL + off), smem_desc(bH + off), idesc, 1u);
          }
          mma_commit(&mbar[st]);
          committed = c + 1;
        }
        contigA = (g.flags & 1) != 0;
        contigB = (g.flags & 2) == 0;
      } else {
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0 && !s_fail) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t aH = smem_u32(sA_hi), aL = smem_u32(sA_lo), bH = smem_u32(sB_hi), bL = smem_u32(sB_lo);
#pragma unroll
          for (int ks = 0; ks < BK / 8; ++ks) {
            const uint32_t off = ks * 2 * 128;
            mma_tf32(tmem, smem_desc(aH + off), smem_desc(bH + off), idesc, (c == 0 && ks == 0) ? 0u : 1u);
            mma_tf32(tmem, smem_desc(aH + off), smem_desc(bL + off), idesc, 1u);
            mma_tf32(tmem, smem_desc(aL + off), smem_desc(bH + off), idesc, 1u);
          }
          mma_commit(&mbar[st]);
          committed = c + 1;
        }
      }
    }
  }
  // wait for the last commit (it completes after every earlier MMA).  After
  // a wait that gave up, thread 0 stopped issuing; it still waits (bounded)
  // for the MMAs it did commit before the TMEM below is released.
  if (tid == 0 && committed > 0) {
    const int last = committed - 1;
    const int st = last % NSTAGE;
    // phase of the last commit: the waits of chunks last + NSTAGE, ... (if
    // any happened) toggled phase[st] past it
    const uint32_t ph = (uint32_t)((last / NSTAGE) & 1);
    const bool seen = (nchunks - 1 > last);   // a later iteration already waited on it (or gave up)
    if ((!seen || s_fail) && !mbar_wait(&mbar[st], ph)) {
      if (!s_fail) atomicExch(err, 1);
      s_fail = 1;
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;");
  __syncthreads();

  float* C = reinterpret_cast<float*>(tk.C);
  const float* Cin = reinterpret_cast<const float*>(tk.Cin);
  if (!s_fail && nchunks > 0) {
    const int lane_grp = warp & 3;             // TMEM lanes 32*lane_grp .. +31
    const int col_half = warp >> 2;            // columns [0, CHALF) or [CHALF, TNB_)
    const int row = i0 + lane_grp * 32 + lane;
#pragma unroll 1
    for (int c0 = col_half * CHALF; c0 < col_half * CHALF + CHALF; c0 += 8) {
      if (c0 >= n_mma) break;
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
  } else if (!s_fail) {
    for (int e = tid; e < TM * TNB_; e += NTH) {
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TNB_));
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
  ProfScope ps("gemm_tc3xtf32", s);
  if (maxN <= 128) {
    constexpr int W = 128;
    const size_t smem = (size_t)NSTAGE * (2 * ABYTES + 2 * W * BK * 4) + 1024;
    static bool attr = false;
    if (!attr) {
      H2_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
    dim3 grid(ntasks, ((maxM + TM - 1) / TM) * ((maxN + W - 1) / W));
    tc_gemm_kernel<W><<<grid, NTH, smem, s>>>(d_tasks, d_terms, tc_err_flag());
  } else {
    const size_t smem = (size_t)NSTAGE * STAGE_BYTES + 1024;
    static bool attr = false;
    if (!attr) {
      H2_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<TNB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
    dim3 grid(ntasks, ((maxM + TM - 1) / TM) * ((maxN + TNB - 1) / TNB));
    tc_gemm_kernel<TNB><<<grid, NTH, smem, s>>>(d_tasks, d_terms, tc_err_flag());
  }
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
