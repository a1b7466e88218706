// Host orchestration and C ABI of the H^2-ULV library.
//
// Level loop of the dependency-free H^2-ULV factorization (arXiv 2208.10907,
// Sec. III): every step below is one batched launch over all boxes of all
// problems at the same height above the leaves; there is no dependency
// between boxes of a height, only between heights.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <memory>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/h2ulv.h"
#include "h2_common.cuh"
#include "h2_mlp.h"
#include "h2_prof.h"
#include "h2_tree.h"

namespace h2 {

// ------------------------------------------------------------------ memory --
// Allocation registry for the host-side task validator (H2_CHECK=1): every
// task's address range is checked against the live device allocations
// before its launch is issued.
static std::map<uintptr_t, size_t>& registry() {
  static std::map<uintptr_t, size_t> r;
  return r;
}
static bool g_check = [] {
  const char* e = getenv("H2_CHECK");
  return e && e[0] == '1';
}();

static void check_range(const void* p, size_t bytes, const char* what) {
  if (!g_check || p == nullptr || bytes == 0) return;
  uintptr_t a = (uintptr_t)p;
  auto& r = registry();
  auto it = r.upper_bound(a);
  if (it == r.begin())
    throw StatusError(H2_ERR_ARG, std::string("validator: ") + what + " pointer outside every allocation");
  --it;
  if (a + bytes > it->first + it->second)
    throw StatusError(H2_ERR_ARG, std::string("validator: ") + what + " range exceeds its allocation by " +
                                      std::to_string((long long)(a + bytes - (it->first + it->second))) +
                                      " bytes (offset " + std::to_string((long long)(a - it->first)) + " of " +
                                      std::to_string((long long)it->second) + ")");
}
// extent in elements of an r x c column-major block with leading dim ld
static size_t ext(long long r, long long c, long long ld) {
  if (r <= 0 || c <= 0) return 0;
  return (size_t)((c - 1) * ld + r);
}

static bool scratch_cache_release();   // frees cached scratch; true if anything was held

struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  explicit DBuf(size_t b) { alloc(b); }
  void alloc(size_t b) {
    release();
    bytes = b;
    if (b) {
      cudaError_t e = cudaMalloc(&p, b);
      if (e != cudaSuccess && scratch_cache_release()) {
        (void)cudaGetLastError();
        e = cudaMalloc(&p, b);
      }
      if (e != cudaSuccess) {
        p = nullptr;
        (void)cudaGetLastError();
        throw StatusError(H2_ERR_OOM, "device allocation of " + std::to_string(b) + " bytes failed");
      }
      registry()[(uintptr_t)p] = b;
    }
  }
  void release() {
    if (p) registry().erase((uintptr_t)p);
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  ~DBuf() { release(); }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};
using DBufP = std::shared_ptr<DBuf>;

// Device buffers of finished Scratch objects, kept for reuse by later ones
// on the same stream: work on one stream runs in order, so a buffer handed
// back after its last launch was queued can be handed out again at once.
// Emptied when a device allocation fails and by h2_destroy.
struct ScratchCache {
  struct Entry {
    DBufP b;
    cudaStream_t s;
  };
  std::vector<Entry> v;
  size_t total = 0;
  std::mutex mu;
  static constexpr size_t LIMIT = size_t(48) << 30;
  DBufP take(size_t bytes, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(mu);
    size_t best = v.size();
    for (size_t i = 0; i < v.size(); ++i) {
      const size_t b = v[i].b->bytes;
      if (v[i].s != s || b < bytes || b > bytes + bytes / 4 + (size_t(64) << 20)) continue;
      if (best == v.size() || b < v[best].b->bytes) best = i;
    }
    if (best == v.size()) return nullptr;
    DBufP r = v[best].b;
    total -= r->bytes;
    v.erase(v.begin() + best);
    return r;
  }
  void give(DBufP b, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(mu);
    if (!b || b.use_count() != 1 || total + b->bytes > LIMIT) return;
    total += b->bytes;
    v.push_back(Entry{std::move(b), s});
  }
};
static ScratchCache& scratch_cache() {
  static ScratchCache c;
  return c;
}
static bool scratch_cache_release() {
  ScratchCache& c = scratch_cache();
  std::vector<ScratchCache::Entry> drop;
  {
    std::lock_guard<std::mutex> lk(c.mu);
    drop.swap(c.v);
    c.total = 0;
  }
  return !drop.empty();   // the buffers are freed here
}

// A buffer of at least `bytes` on stream s: the cached one if it fits, else
// a new allocation.
static DBufP cached_or_new(size_t bytes, cudaStream_t s) {
  DBufP b = scratch_cache().take(bytes, s);
  return b ? b : std::make_shared<DBuf>(bytes);
}
// Keep b when it is large enough (and not much larger) and nobody else holds
// it; otherwise replace it.  Its contents are not preserved.
static void ensure(DBufP& b, size_t bytes) {
  if (b && b.use_count() == 1 && b->bytes >= bytes && b->bytes <= bytes + bytes / 4 + (size_t(64) << 20)) return;
  b.reset();
  b = std::make_shared<DBuf>(bytes);
}

// Pinned host staging for task-array uploads, one ring per stream: a copy
// from pageable memory would make the host wait for the stream, so task
// arrays are first copied into pinned memory and uploaded asynchronously,
// and the host builds the next launch's tasks while the GPU works.  When the
// ring is full, the stream is synchronised (every earlier upload from it has
// then completed) and the ring starts over.
struct PinnedRing {
  char* buf = nullptr;
  size_t cap = 0, pos = 0;
  ~PinnedRing() {
    if (buf) cudaFreeHost(buf);
  }
  void* stage(const void* src, size_t n, cudaStream_t s) {
    const size_t need = (n + 255) & ~size_t(255);
    if (need > cap) {
      H2_CUDA(cudaStreamSynchronize(s));
      if (buf) cudaFreeHost(buf);
      buf = nullptr;
      cap = std::max(need, size_t(64) << 20);
      H2_CUDA(cudaHostAlloc((void**)&buf, cap, cudaHostAllocDefault));
      pos = 0;
    } else if (pos + need > cap) {
      H2_CUDA(cudaStreamSynchronize(s));
      pos = 0;
    }
    void* p = buf + pos;
    std::memcpy(p, src, n);
    pos += need;
    return p;
  }
};
static void* pinned_stage(const void* src, size_t n, cudaStream_t s) {
  static std::mutex mu;
  static std::map<cudaStream_t, std::unique_ptr<PinnedRing>> rings;
  std::lock_guard<std::mutex> lk(mu);
  auto& r = rings[s];
  if (!r) r.reset(new PinnedRing());
  return r->stage(src, n, s);
}

// Stream-ordered scratch: everything lives until the Scratch is destroyed.
// Task lists and small buffers are carved from 32 MB arenas (one device
// allocation per arena instead of one per launch); large buffers get their
// own allocation.  Both come from, and go back to, the scratch cache.
struct Scratch {
  static constexpr size_t ARENA = size_t(32) << 20, SMALL = size_t(1) << 20;
  std::vector<DBufP> bufs;
  std::vector<uintptr_t> subs;   // validator entries of arena carvings
  cudaStream_t s;
  DBufP arena;
  size_t apos = 0;
  explicit Scratch(cudaStream_t st) : s(st) {}
  ~Scratch() {
    for (uintptr_t k : subs) registry().erase(k);
    arena.reset();
    for (DBufP& b : bufs) scratch_cache().give(std::move(b), s);
  }
  DBufP fresh(size_t bytes) {
    DBufP b = scratch_cache().take(bytes, s);
    if (!b) b = std::make_shared<DBuf>(bytes);
    bufs.push_back(b);
    return b;
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  void* carve(size_t bytes) {
    const size_t b = (std::max<size_t>(bytes, 16) + 255) & ~size_t(255);
    if (!arena || apos + b > arena->bytes) {
      arena = fresh(ARENA);
      apos = 0;
    }
    void* p = (char*)arena->p + apos;
    apos += b;
    if (g_check) {
      registry()[(uintptr_t)p] = bytes;
      subs.push_back((uintptr_t)p);
    }
    return p;
  }
  template <class T> T* up(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    const size_t nb = v.size() * sizeof(T);
    void* p;
    p = nb <= SMALL ? carve(nb) : fresh(nb)->p;
    H2_CUDA(cudaMemcpyAsync(p, pinned_stage(v.data(), nb, s), nb, cudaMemcpyHostToDevice, s));
    return reinterpret_cast<T*>(p);
  }
  void* alloc(size_t bytes, bool zero = false) {
    void* p;
    p = bytes <= SMALL ? carve(bytes) : fresh(bytes)->p;
    if (zero) H2_CUDA(cudaMemsetAsync(p, 0, std::max<size_t>(bytes, 16), s));
    return p;
  }
};

static size_t esz(Prec p) { return p == Prec::F64 ? 8 : 4; }

static void validate(const std::vector<GemmTask>& tasks, const std::vector<GemmTerm>& terms, size_t es) {
  if (!g_check) return;
  for (const GemmTask& t : tasks) {
    check_range(t.C, ext(t.M, t.N, t.ldc) * es, "gemm C");
    if (t.Cin && t.beta != 0.0) check_range(t.Cin, ext(t.M, t.N, t.ldcin) * es, "gemm Cin");
    if (t.ldc < t.M) throw StatusError(H2_ERR_ARG, "validator: gemm ldc < M");
    for (int q = t.t0; q < t.t0 + t.nt; ++q) {
      const GemmTerm& m = terms[q];
      bool ta = m.flags & 1, tb = m.flags & 2;
      check_range(m.A, (ta ? ext(m.K, t.M, m.lda) : ext(t.M, m.K, m.lda)) * es, "gemm A");
      check_range(m.B, (tb ? ext(t.N, m.K, m.ldb) : ext(m.K, t.N, m.ldb)) * es, "gemm B");
      if ((ta ? m.K : t.M) > m.lda || (tb ? t.N : m.K) > m.ldb)
        throw StatusError(H2_ERR_ARG, "validator: gemm leading dimension too small");
    }
  }
}
static void validate(const std::vector<TrsmTask>& v, size_t es) {
  if (!g_check) return;
  for (const TrsmTask& t : v) {
    if (t.n > NMAX) throw StatusError(H2_ERR_ARG, "validator: trsm n > NMAX");
    check_range(t.A, ext(t.n, t.n, t.lda) * es, "trsm A");
    check_range(t.B, ext(t.n, t.nrhs, t.ldb) * es, "trsm B");
    if (t.piv) check_range(t.piv, (size_t)t.n * 4, "trsm piv");
  }
}
static void validate(const std::vector<LuTask>& v, size_t es) {
  if (!g_check) return;
  for (const LuTask& t : v) {
    check_range(t.A, ext(t.m, t.nc, t.lda) * es, "getrf A");
    check_range(t.piv, (size_t)t.nc * 4, "getrf piv");
  }
}
static void validate(const std::vector<CopyTask>& v, size_t es_s, size_t es_d, bool tr) {
  if (!g_check) return;
  for (const CopyTask& t : v) {
    check_range(t.src, (tr ? ext(t.cols, t.rows, t.lds) : ext(t.rows, t.cols, t.lds)) * es_s, "copy src");
    check_range(t.dst, ext(t.rows, t.cols, t.ldd) * es_d, "copy dst");
  }
}
static void validate(const std::vector<CholTask>& v) {
  if (!g_check) return;
  for (const CholTask& t : v) {
    if (t.n > NMAX) throw StatusError(H2_ERR_ARG, "validator: pchol n > NMAX");
    check_range(t.G, ext(t.n, t.n, t.ldg) * 8, "pchol G");
    check_range(t.R, (size_t)t.n * t.n * 8, "pchol R");
    check_range(t.piv, (size_t)t.n * 4, "pchol piv");
    check_range(t.rank, 4, "pchol rank");
  }
}
static void validate(const std::vector<KgramTask>& v) {
  if (!g_check) return;
  for (const KgramTask& t : v) {
    check_range(t.G, ext(t.n, t.n, t.ldg) * 8, "kgram G");
    check_range(t.cand, (size_t)t.n * 4, "kgram cand");
    check_range(t.samp, (size_t)t.m * 4, "kgram samp");
  }
}
static void validate(const std::vector<AsmTask>& v, size_t es) {
  if (!g_check) return;
  for (const AsmTask& t : v) {
    check_range(t.out, ext(t.nr, t.nc, t.ld) * es, "assemble out");
    if (t.ridx) check_range(t.ridx, (size_t)t.nr * 4, "assemble ridx");
    if (t.cidx) check_range(t.cidx, (size_t)t.nc * 4, "assemble cidx");
  }
}
static void validate(const std::vector<HqrTask>& v, size_t es) {
  if (!g_check) return;
  for (const HqrTask& t : v) {
    check_range(t.M, (size_t)t.n * t.r * es, "hqr M");
    check_range(t.V, (size_t)t.n * t.r * es, "hqr V");
    check_range(t.Q, (size_t)t.n * t.n * es, "hqr Q");
    check_range(t.W, (size_t)t.r * t.r * es, "hqr W");
  }
}
static void validate(const std::vector<InterpTask>& v, size_t es) {
  if (!g_check) return;
  for (const InterpTask& t : v) {
    check_range(t.P, (size_t)t.n * t.r * es, "interp P");
    check_range(t.piv, (size_t)t.n * 4, "interp piv");
    if (t.r < t.n) check_range(t.T, ext(t.r, t.n - t.r, t.ldt) * es, "interp T");
  }
}

// ---------------------------------------------------------- GEMM batches --
struct GemmBatch {
  std::vector<GemmTask> tasks;
  std::vector<GemmTerm> terms;
  int maxM = 0, maxN = 0, ksum = 0;
  double flops = 0.0, bytes = 0.0;
  void add(void* C, int ldc, int M, int N, double alpha, double beta, const void* Cin, int ldcin,
           const std::vector<GemmTerm>& ts) {
    if (M <= 0 || N <= 0) return;
    int kt = 0;
    for (const GemmTerm& g : ts) kt += std::max(0, g.K);
    ksum = std::max(ksum, kt);
    GemmTask t;
    t.C = C;
    t.Cin = Cin;
    t.M = M;
    t.N = N;
    t.ldc = ldc;
    t.ldcin = ldcin;
    t.t0 = (int)terms.size();
    t.nt = 0;
    for (const GemmTerm& g : ts)
      if (g.K > 0) {
        terms.push_back(g);
        ++t.nt;
        flops += 2.0 * M * N * g.K;
        bytes += (double)M * g.K + (double)g.K * N;
      }
    bytes += (double)M * N * ((beta != 0.0 && Cin) ? 2.0 : 1.0);
    t.alpha = alpha;
    t.beta = beta;
    tasks.push_back(t);
    maxM = std::max(maxM, M);
    maxN = std::max(maxN, N);
  }
  // one term; trA / trB flip the operands (combined with the run-level flags)
  void add1(void* C, int ldc, int M, int N, const void* A, int lda, const void* B, int ldb, int K,
            double alpha = 1.0, double beta = 0.0, const void* Cin = nullptr, int ldcin = 0, int flags = 0) {
    add(C, ldc, M, N, alpha, beta, Cin ? Cin : (beta != 0.0 ? C : nullptr), Cin ? ldcin : ldc,
        {GemmTerm{A, B, K, lda, ldb, flags}});
  }
  void run(Prec p, bool trA, bool trB, Scratch& sc) {
    if (tasks.empty()) return;
    const int fl = (trA ? 1 : 0) | (trB ? 2 : 0);
    for (GemmTerm& t : terms) t.flags ^= fl;
    validate(tasks, terms, esz(p));
    GemmTerm* dm = sc.up(terms);
    const size_t CH = 1u << 20;
    for (size_t o = 0; o < tasks.size(); o += CH) {
      size_t cnt = std::min(CH, tasks.size() - o);
      std::vector<GemmTask> sub(tasks.begin() + o, tasks.begin() + o + cnt);
      GemmTask* dt = sc.up(sub);
      if (o == 0) prof_note(flops, bytes * esz(p));
      launch_gemm(p, dt, dm, (int)cnt, maxM, maxN, sc.s, false, ksum);
    }
  }
};


// One (box, list position) pair with its scratch slot; the pairs of one
// batched launch share a scratch buffer.
struct PairSlot {
  int g, k, j;       // box, position in its near/far list, partner box
  size_t bytes, off; // slot size and offset in the chunk buffer
};

// The pairs (g, list[g][k]) accepted by `keep`, ordered by list position
// and then by box, so that a chunk holds the same positions of every box.
template <class Keep, class Bytes>
static std::vector<PairSlot> near_pairs(const std::vector<std::vector<int>>& list, Keep keep, Bytes bytes) {
  std::vector<PairSlot> v;
  size_t maxdeg = 0;
  for (const auto& l : list) maxdeg = std::max(maxdeg, l.size());
  for (size_t k = 0; k < maxdeg; ++k)
    for (int g = 0; g < (int)list.size(); ++g) {
      if (k >= list[g].size()) continue;
      const int j = list[g][k];
      if (keep(g, j)) v.push_back(PairSlot{g, (int)k, j, bytes(g, j), 0});
    }
  return v;
}

// End of the chunk of pairs starting at p0 whose slots fit in `budget`
// bytes (at least one pair); assigns the slot offsets.
static size_t chunk_pairs(std::vector<PairSlot>& v, size_t p0, size_t budget) {
  size_t tot = 0, p1 = p0;
  for (; p1 < v.size(); ++p1) {
    const size_t b = (v[p1].bytes + 255) & ~size_t(255);
    if (p1 > p0 && tot + b > budget) break;
    v[p1].off = tot;
    tot += b;
  }
  return p1;
}

// Algorithmic work of the batched dense kernels (flops and the bytes their
// operands and results occupy, each counted once), noted for the profiler
// before each launch.  LU of an m x c panel: m c^2 - c^3/3 flops; triangular
// solve of n x n with r right-hand sides: n^2 r; Householder QR of n x r with
// the full n x n Q formed: 2 r^2 (n - r/3) + 4 n^2 r - 2 n r^2; far-field
// Gram of n candidates and m samples: 2 n^2 m (plus 2 n m kernel values).
static double work_getrf(const std::vector<LuTask>& v, size_t es, double& bytes) {
  double f = 0.0;
  bytes = 0.0;
  for (const LuTask& t : v) {
    f += (double)t.m * t.nc * t.nc - (double)t.nc * t.nc * t.nc / 3.0;
    bytes += 2.0 * es * t.m * t.nc;
  }
  return f;
}
static double work_trsm(const std::vector<TrsmTask>& v, size_t es, double& bytes) {
  double f = 0.0;
  bytes = 0.0;
  for (const TrsmTask& t : v) {
    f += (double)t.n * t.n * t.nrhs;
    bytes += es * (0.5 * t.n * t.n + 2.0 * t.n * t.nrhs);
  }
  return f;
}
static double work_copy(const std::vector<CopyTask>& v, size_t es_s, size_t es_d) {
  double b = 0.0;
  for (const CopyTask& t : v) b += (double)(es_s + es_d) * t.rows * t.cols;
  return b;
}

// Validate (H2_CHECK=1), upload and launch.
static void run_trsm(Prec p, bool lower, bool unit, bool tr, const std::vector<TrsmTask>& v, int maxrhs, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(p));
  double by = 0.0, f = work_trsm(v, esz(p), by);
  prof_note(f, by);
  int maxn = 0;
  for (const TrsmTask& t : v) maxn = std::max(maxn, t.n);
  launch_trsm(p, lower, unit, tr, sc.up(v), (int)v.size(), maxrhs, maxn, sc.s);
}
static void run_getrf(Prec p, const std::vector<LuTask>& v, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(p));
  double by = 0.0, f = work_getrf(v, esz(p), by);
  prof_note(f, by);
  int maxm = 0;
  for (const LuTask& t : v) maxm = std::max(maxm, t.m);
  launch_getrf(p, sc.up(v), (int)v.size(), maxm, sc.s);
}
static void run_copy(Prec a, Prec b, bool tr, const std::vector<CopyTask>& v, int mr, int mc, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(a), esz(b), tr);
  prof_note(0.0, work_copy(v, esz(a), esz(b)));
  launch_copy(a, b, tr, sc.up(v), (int)v.size(), mr, mc, sc.s);
}
// The pivoted Cholesky's work depends on the ranks it finds; it is added
// once they are read back (prof_add), at n r^2 - 2 r^3 / 3 flops per box.
static void run_pchol(const std::vector<CholTask>& v, Scratch& sc) {
  if (v.empty()) return;
  validate(v);
  double by = 0.0;
  for (const CholTask& t : v) by += 16.0 * t.n * t.n;
  prof_note(0.0, by);
  launch_pchol(sc.up(v), (int)v.size(), sc.s);
}
static void run_kgram(Prec p, const std::vector<KgramTask>& v, int maxn, Points pts, KParams kp, Scratch& sc) {
  if (v.empty()) return;
  validate(v);
  double f = 0.0, by = 0.0;
  for (const KgramTask& t : v) {
    f += 2.0 * t.n * t.n * t.m;
    by += 8.0 * t.n * t.n * (t.accumulate ? 2.0 : 1.0);
  }
  prof_note(f, by);
  launch_kgram(p, sc.up(v), (int)v.size(), maxn, pts, kp, sc.s);
}
static void run_assemble(Prec p, const std::vector<AsmTask>& v, int mr, int mc, Points pts, KParams kp, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(p));
  double by = 0.0;
  for (const AsmTask& t : v) by += (double)esz(p) * t.nr * t.nc;
  prof_note(0.0, by);
  launch_assemble(p, sc.up(v), (int)v.size(), mr, mc, pts, kp, sc.s);
}
static void run_hqr(Prec p, const std::vector<HqrTask>& v, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(p));
  double f = 0.0, by = 0.0;
  for (const HqrTask& t : v) {
    const double n = t.n, r = t.r;
    f += 2.0 * r * r * (n - r / 3.0) + 4.0 * n * n * r - 2.0 * n * r * r;
    by += (double)esz(p) * (2.0 * n * r + n * n + r * r);
  }
  prof_note(f, by);
  launch_hqr(p, sc.up(v), (int)v.size(), sc.s);
}
// Folds declare 2 rows n^2 flops per folded row block (a Householder QR of
// the rows appended to an n x n triangle) and the explicit rows' bytes.
static void run_fold(const std::vector<FoldTask>& v, const std::vector<FoldTerm>& terms, Points pts, KParams kp,
                     Scratch& sc) {
  if (v.empty()) return;
  double flops = 0.0, bytes = 0.0;
  for (const FoldTask& t : v) {
    double rows = t.m;
    for (int q = t.t0; q < t.t0 + t.nt; ++q) {
      rows += terms[q].rows;
      bytes += 8.0 * terms[q].rows * t.n;
    }
    flops += 2.0 * rows * t.n * t.n;
    bytes += 16.0 * t.n * t.n;
  }
  if (g_check)
    for (const FoldTask& t : v) {
      check_range(t.R, (size_t)t.n * t.n * 8, "fold R");
      for (int q = t.t0; q < t.t0 + t.nt; ++q) {
        const FoldTerm& f = terms[q];
        check_range(f.X, (f.tr ? ext(f.rows, t.n, f.ld) : ext(t.n, f.rows, f.ld)) * 8, "fold rows");
      }
    }
  prof_note(flops, bytes);
  int maxn = 0;
  for (const FoldTask& t : v) maxn = std::max(maxn, t.n);
  launch_fold(sc.up(v), (int)v.size(), maxn, sc.up(terms), pts, kp, sc.s);
}
// Column-pivoted QR of an n x n triangle stopped at rank r: 4 n^2 r -
// 2 (n + n) r^2 + 4 r^3 / 3 flops, added once the ranks are read back.
static void run_pqr(const std::vector<PqrTask>& v, Scratch& sc) {
  if (v.empty()) return;
  double by = 0.0;
  for (const PqrTask& t : v) by += 16.0 * t.n * t.n;
  prof_note(0.0, by);
  launch_pqr(sc.up(v), (int)v.size(), sc.s);
}
static void run_interp(Prec p, const std::vector<InterpTask>& v, Scratch& sc) {
  if (v.empty()) return;
  validate(v, esz(p));
  double by = 0.0;
  for (const InterpTask& t : v) by += (double)esz(p) * ((double)t.n * t.r + (double)t.r * (t.n - t.r));
  prof_note(0.0, by);
  launch_interp(p, sc.up(v), (int)v.size(), sc.s);
}


// ------------------------------------------------------------------ plans --
// A fixed sequence of batched launches with device-resident task arrays,
// replayed without host work; captured once into a CUDA graph.
struct Op {
  int kind;             // 0 gemm, 1 trsm, 2 copy, 3 symmetric near pairs, 4 gather partials
  Prec p, p2;
  bool f1, f2, f3;
  const void* tasks;
  const void* terms;
  int n, a, b;
  const char* tag;
  const double* x;      // kinds 3, 4
  double* y;
  long long ld;
  double flops, bytes;  // algorithmic work of the launch (profiling counters)
};

struct Plan {
  std::vector<Op> ops;
  std::vector<DBufP> bufs;   // task arrays and workspaces
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t s = nullptr;
  template <class T> T* up(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    auto b = std::make_shared<DBuf>(v.size() * sizeof(T));
    H2_CUDA(cudaMemcpy(b->p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    bufs.push_back(b);
    return b->template as<T>();
  }
  double* work(size_t elems, bool zero = false) {
    auto b = std::make_shared<DBuf>(std::max<size_t>(elems, 2) * 8);
    if (zero) H2_CUDA(cudaMemset(b->p, 0, b->bytes));
    bufs.push_back(b);
    return b->template as<double>();
  }
  void gemm(Prec p, GemmBatch& gb, bool trA, bool trB) {
    if (gb.tasks.empty()) return;
    const int fl = (trA ? 1 : 0) | (trB ? 2 : 0);
    for (GemmTerm& t : gb.terms) t.flags ^= fl;
    validate(gb.tasks, gb.terms, esz(p));
    Op o{};
    o.kind = 0;
    o.p = p;
    o.tasks = up(gb.tasks);
    o.terms = up(gb.terms);
    o.n = (int)gb.tasks.size();
    o.a = gb.maxM;
    o.b = gb.maxN;
    o.ld = gb.ksum;
    o.flops = gb.flops;
    o.bytes = gb.bytes * esz(p);
    o.tag = cur_tag;
    ops.push_back(o);
  }
  void trsm(Prec p, bool lower, bool unit, bool tr, const std::vector<TrsmTask>& v, int maxrhs) {
    if (v.empty()) return;
    validate(v, esz(p));
    Op o{};
    o.flops = work_trsm(v, esz(p), o.bytes);
    for (const TrsmTask& t : v) o.b = std::max(o.b, t.n);
    o.kind = 1;
    o.p = p;
    o.f1 = lower;
    o.f2 = unit;
    o.f3 = tr;
    o.tasks = up(v);
    o.n = (int)v.size();
    o.a = maxrhs;
    o.tag = cur_tag;
    ops.push_back(o);
  }
  void copy(Prec a, Prec b, bool tr, const std::vector<CopyTask>& v, int mr, int mc) {
    if (v.empty()) return;
    validate(v, esz(a), esz(b), tr);
    Op o{};
    o.bytes = work_copy(v, esz(a), esz(b));
    o.kind = 2;
    o.p = a;
    o.p2 = b;
    o.f1 = tr;
    o.tasks = up(v);
    o.n = (int)v.size();
    o.a = mr;
    o.b = mc;
    o.tag = cur_tag;
    ops.push_back(o);
  }
  const char* cur_tag = nullptr;
  void tag(const char* t) { cur_tag = t; }
  void symv(const std::vector<SymPairTask>& v, const double* x, long long ldx, double* part, int nrhs) {
    Op o{};
    o.kind = 3;
    o.tasks = up(v);
    o.n = (int)v.size();
    o.x = x;
    o.y = part;
    o.ld = ldx;
    o.a = nrhs;
    for (const SymPairTask& t : v) {   // every stored block read once, two products
      o.bytes += 8.0 * t.nI * t.nJ;
      o.flops += 4.0 * t.nI * t.nJ * nrhs;
    }
    o.tag = cur_tag;
    ops.push_back(o);
  }
  std::vector<long long> gather_n;
  void gather_rows(const double* src, long long lds, double* dst, long long ldd, const int* idx, long long n,
                   int nrhs) {
    Op o{};
    o.kind = 5;
    o.x = src;
    o.y = dst;
    o.ld = lds;
    o.tasks = idx;
    o.n = nrhs;
    o.a = (int)ldd;
    gather_n.push_back(n);
    o.b = (int)(gather_n.size() - 1);
    o.tag = cur_tag;
    ops.push_back(o);
  }
  void gather(const std::vector<GatherTask>& v, const std::vector<long long>& offs, const double* part, double* y,
              long long ldy, int nrhs) {
    Op o{};
    o.kind = 4;
    o.tasks = up(v);
    o.terms = up(offs);
    o.n = (int)v.size();
    o.x = part;
    o.y = y;
    o.ld = ldy;
    o.a = nrhs;
    o.tag = cur_tag;
    ops.push_back(o);
  }
  void issue(cudaStream_t st) const {
    for (const Op& o : ops) {
      prof_tag(o.tag);
      if (o.flops > 0.0 || o.bytes > 0.0) prof_note(o.flops, o.bytes);
      if (o.kind == 0)
        launch_gemm(o.p, (const GemmTask*)o.tasks, (const GemmTerm*)o.terms, o.n, o.a, o.b, st, false, (int)o.ld);
      else if (o.kind == 1) launch_trsm(o.p, o.f1, o.f2, o.f3, (const TrsmTask*)o.tasks, o.n, o.a, o.b, st);
      else if (o.kind == 2) launch_copy(o.p, o.p2, o.f1, (const CopyTask*)o.tasks, o.n, o.a, o.b, st);
      else if (o.kind == 3) launch_symv_pairs((const SymPairTask*)o.tasks, o.n, o.x, o.ld, o.y, o.a, st);
      else if (o.kind == 4)
        launch_gather_parts((const GatherTask*)o.tasks, o.n, (const long long*)o.terms, o.x, o.y, o.ld, o.a, st);
      else if (o.kind == 5)
        launch_gather_rows(o.x, o.ld, o.y, o.a, (const int*)o.tasks, gather_n[o.b], o.n, st);
    }
    prof_tag(nullptr);
  }
  // replay: through the captured graph when profiling is off, else launch by
  // launch (so each kernel is timed on its own)
  void run(cudaStream_t st) {
    if (prof().timing || getenv("H2_NO_GRAPH")) {
      issue(st);
      return;
    }
    if (!exec || st != s) {
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      exec = nullptr;
      graph = nullptr;
      s = st;
      cudaStream_t cs = st;
      bool own = false;
      if (cs == nullptr) {   // the legacy default stream cannot be captured
        H2_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        own = true;
      }
      H2_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
      issue(cs);
      H2_CUDA(cudaStreamEndCapture(cs, &graph));
      H2_CUDA(cudaGraphInstantiate(&exec, graph, 0));
      if (own) {
        H2_CUDA(cudaStreamSynchronize(cs));
        cudaStreamDestroy(cs);
      }
    }
    H2_CUDA(cudaGraphLaunch(exec, st));
    prof().total_launches += (long long)ops.size();
  }
  ~Plan() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};
using PlanP = std::shared_ptr<Plan>;

// ------------------------------------------------------- handle structure --
struct BoxRef {
  int prob, level, local;
};

struct Height {
  int nb = 0;                        // active boxes at this height
  std::vector<BoxRef> ref;
  std::vector<std::vector<int>> near, far;  // global ids at this height
  std::vector<int> parent;           // global id at height+1, or -1 (root)
  std::vector<int> root_slot;        // if parent == -1: index of the box in its problem's root
  std::vector<int> first_child;      // global id of the first child at height-1 (H > 0)
  // operator (H^2 matvec) basis
  std::vector<int> n_op, r_op;
  std::vector<std::vector<int>> cand_op, sk_op;   // global tree-order point ids
  std::vector<DBufP> P_op;           // n_op x r_op interpolation (FP64)
  DBufP Kcat_op;                     // per box: [K(sk_I, sk_J1) K(sk_I, sk_J2) ...] (r_I x sum r_J)
  std::vector<size_t> kcat_off;      // element offsets per box
  std::vector<int> kcat_cols;        // sum of r_J over the far list
  DBufP far_gidx;                    // gather index into the skeleton vector, per box concatenated
  std::vector<size_t> fg_off;        // offsets into far_gidx (= skeleton-gather vector offsets)
  size_t fg_len = 0;
  std::vector<int64_t> xh_off;       // skeleton-vector offsets
  int64_t xh_len = 0;
  // ULV factor
  std::vector<int> n, r;
  std::vector<std::vector<int>> cand, sk;
  DBufP Q;                           // per box n x n (FP64) [U^R U^S]
  std::vector<size_t> q_off;         // element offsets into Q / S buffers (n^2 each)
  DBufP Qw;                          // work-precision copy of Q (mixed mode)
  DBufP S;                           // per box n x n FP64: LU of S^RR, U^RS, S^SR
  DBufP Lt;                          // per box m x r FP64: (L^SR)^T
  std::vector<size_t> lt_off;
  DBufP pivRR;                       // per box m ints (offsets q_off-free: pv_off)
  std::vector<size_t> pv_off;
  DBufP W;                           // per box r x r FP64 (triangular factor of the ID)
  DBufP Linv, Uinv;                  // per box m x m FP64: L^-1 P^T and U^-1 of the S^RR LU (solve sweeps)
  std::vector<size_t> li_off;
  std::vector<int64_t> y_off;        // redundant-part vector offsets (solve)
  int64_t y_len = 0;
  std::vector<size_t> w_off;
  std::vector<int64_t> v_off;        // level-vector offsets (solve)
  int64_t v_len = 0;
};

struct Root {
  int n = 0;
  std::vector<int> off;              // offsets of the level-ltop boxes
  DBufP A;                           // work-precision assembled matrix
  DBufP LU;                          // FP64 LU factors
  DBufP piv;
  DBufP inv;                         // FP64 inverse
  double logdet = 0.0, sign = 1.0;
};

struct Problem {
  Tree t;
  int64_t off = 0;                   // global tree-order offset
  int H = 0;                         // number of ULV heights (L - ltop)
  Root root;
};

struct Handle {
  cudaStream_t s = nullptr;
  int dev = 0;                       // device current at construct (owns every buffer of the handle)
  KParams kp{};
  h2_options opt{};
  std::vector<Problem> probs;
  int64_t Ntot = 0;
  int Hmax = 0;
  DBuf px, py, pz;                   // tree-order points
  DBuf perm;                         // global tree position -> global caller row
  std::vector<Height> hs;            // heights 0 .. Hmax-1 (plus leaf blocks)
  // leaf near blocks (FP64), one per near pair at height 0 (also for H = 0
  // problems, whose root is their whole leaf level)
  std::vector<std::vector<int>> leaf_near;   // global leaf ids
  std::vector<BoxRef> leaf_ref;
  std::vector<size_t> leaf_blk_off;          // element offset per near pair
  std::vector<size_t> leaf_pair_ptr;         // CSR row pointer over leaves
  std::vector<size_t> leaf_mirror;           // pair index holding the stored block (i <= j)
  DBuf leaf_blk;
  std::vector<int> leaf_n;
  std::vector<int64_t> leaf_s;               // global tree-order start per leaf
  bool factored = false;
  int precision = 0, spd = 0;
  double tol_basis = 0.0;                    // rank tolerance the last factorization's bases used
  const char* basis_route = "none";          // "qr" or "gram" (route of the last factorization)
  // solve-time plans, per right-hand-side count: workspaces and launch lists
  struct SolvePlans {
    int nrhs = 0;
    double *B = nullptr, *X = nullptr, *R = nullptr, *Uin = nullptr, *Uout = nullptr, *nrm = nullptr;
    // GMRES workspace (allocated on first use)
    double *V = nullptr, *Xsol = nullptr, *hdev = nullptr, *part = nullptr, *ydev = nullptr;
    int m = 0;
    PlanP ulv, mv;
    std::vector<DBufP> bufs;
  };
  std::map<int, std::shared_ptr<SolvePlans>> plans;
  DBufP bstage, xstage;              // stacked right-hand sides / solutions (h2_solve_batched)
  bool per_problem = false;          // refinement checks every problem's columns on their own norms
  DBufP segnrm;                      // per (problem, column) squared norms
  std::vector<double> last_rel;      // per (problem, column) relative residuals of the last solve
  double t_construct_ms = 0, t_factor_ms = 0;
  std::vector<double> level_ms;
  // rank predictor (optional)
  const Mlp* predictor = nullptr;
  double pred_margin = 0.15;
  long long pred_hits = 0, pred_misses = 0;
  double pred_bytes = 0, worst_bytes = 0, exact_bytes = 0;
  std::string stats_extra;
};

static Points points(const Handle& h) {
  return Points{h.px.as<double>(), h.py.as<double>(), h.pz.as<double>()};
}

// Predictor features of every box at height H (8 per box).
static void height_features(const Handle& h, int H, std::vector<float>& F) {
  const Height& ht = h.hs[H];
  F.assign((size_t)ht.nb * MLP_FEATURES, 0.f);
  std::vector<int64_t> samp;
  for (int g = 0; g < ht.nb; ++g) {
    const BoxRef& b = ht.ref[g];
    const Problem& pb = h.probs[b.prob];
    const Box& bx = pb.t.boxes[b.level][b.local];
    far_samples(pb.t, b.level, b.local, h.opt.far_s0, h.opt.far_smin, samp);
    int n = ht.n.empty() ? (int)(bx.e - bx.s) : ht.n[g];
    box_features(n, bx.lo, bx.hi, (int)ht.near[g].size(), (int)ht.far[g].size(), H, (int)samp.size(),
                 &F[(size_t)g * MLP_FEATURES]);
  }
}

static bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ------------------------------------------------------------- construct --
static void build_heights(Handle& h) {
  // leaves (height 0) of every problem, including problems with H = 0
  int nleaf = 0;
  std::vector<int> leaf_base(h.probs.size());
  for (size_t p = 0; p < h.probs.size(); ++p) {
    leaf_base[p] = nleaf;
    nleaf += (int)h.probs[p].t.boxes[h.probs[p].t.L].size();
  }
  h.leaf_ref.resize(nleaf);
  h.leaf_near.resize(nleaf);
  h.leaf_n.resize(nleaf);
  h.leaf_s.resize(nleaf);
  for (size_t p = 0; p < h.probs.size(); ++p) {
    const Tree& t = h.probs[p].t;
    for (size_t i = 0; i < t.boxes[t.L].size(); ++i) {
      int g = leaf_base[p] + (int)i;
      h.leaf_ref[g] = BoxRef{(int)p, t.L, (int)i};
      for (int j : t.near[t.L][i]) h.leaf_near[g].push_back(leaf_base[p] + j);
      h.leaf_n[g] = (int)(t.boxes[t.L][i].e - t.boxes[t.L][i].s);
      h.leaf_s[g] = h.probs[p].off + t.boxes[t.L][i].s;
    }
  }
  // ULV / operator heights
  h.Hmax = 0;
  for (auto& pb : h.probs) h.Hmax = std::max(h.Hmax, pb.H);
  h.hs.assign(h.Hmax, Height());
  std::vector<std::vector<int>> base(h.Hmax, std::vector<int>(h.probs.size(), -1));
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    int nb = 0;
    for (size_t p = 0; p < h.probs.size(); ++p) {
      const Problem& pb = h.probs[p];
      if (H < pb.H) {
        base[H][p] = nb;
        nb += (int)pb.t.boxes[pb.t.L - H].size();
      }
    }
    ht.nb = nb;
    ht.ref.resize(nb);
    ht.near.resize(nb);
    ht.far.resize(nb);
    ht.parent.assign(nb, -1);
    ht.root_slot.assign(nb, -1);
    ht.first_child.assign(nb, -1);
  }
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    for (size_t p = 0; p < h.probs.size(); ++p) {
      const Problem& pb = h.probs[p];
      if (H >= pb.H) continue;
      int l = pb.t.L - H;
      for (size_t i = 0; i < pb.t.boxes[l].size(); ++i) {
        int g = base[H][p] + (int)i;
        ht.ref[g] = BoxRef{(int)p, l, (int)i};
        for (int j : pb.t.near[l][i]) ht.near[g].push_back(base[H][p] + j);
        for (int j : pb.t.far[l][i]) ht.far[g].push_back(base[H][p] + j);
        if (H + 1 < pb.H) ht.parent[g] = base[H + 1][p] + (int)i / 2;
        else ht.root_slot[g] = (int)i / 2;
        if (H > 0) ht.first_child[g] = base[H - 1][p] + 2 * (int)i;
      }
    }
  }
}

// Leaf near block of pair (g, q): only pairs with g <= j are stored (the
// kernels are symmetric, A_JI = A_IJ^T); the others reference the mirror.
struct BlkRef {
  const double* ptr;
  int ld;
  int tr;
};
static BlkRef leaf_block(const Handle& h, int g, size_t q) {
  size_t pi = h.leaf_pair_ptr[g] + q;
  int j = h.leaf_near[g][q];
  if (g <= j) return BlkRef{h.leaf_blk.as<double>() + h.leaf_blk_off[pi], h.leaf_n[g], 0};
  size_t mi = h.leaf_mirror[pi];
  return BlkRef{h.leaf_blk.as<double>() + h.leaf_blk_off[mi], h.leaf_n[j], 1};
}

// The H^2 operator: per height, nested interpolative bases from the sampled
// far-field block rows (eq. u with the low-rank blocks only), the far
// skeleton blocks K(sk_I, sk_J) and the dense leaf near blocks.
static void build_operator(Handle& h) {
  cudaStream_t s = h.s;
  Points pts = points(h);
  // leaf near blocks (FP64)
  int nleaf = (int)h.leaf_ref.size();
  h.leaf_pair_ptr.assign(nleaf + 1, 0);
  for (int g = 0; g < nleaf; ++g) h.leaf_pair_ptr[g + 1] = h.leaf_pair_ptr[g] + h.leaf_near[g].size();
  h.leaf_blk_off.assign(h.leaf_pair_ptr[nleaf] + 1, 0);
  h.leaf_mirror.assign(h.leaf_pair_ptr[nleaf], 0);
  size_t tot = 0;
  for (int g = 0; g < nleaf; ++g)
    for (size_t q = 0; q < h.leaf_near[g].size(); ++q) {
      int j = h.leaf_near[g][q];
      if (g <= j) {
        h.leaf_blk_off[h.leaf_pair_ptr[g] + q] = tot;
        tot += (size_t)h.leaf_n[g] * h.leaf_n[j];
      } else {
        const auto& nl = h.leaf_near[j];
        size_t qq = std::find(nl.begin(), nl.end(), g) - nl.begin();
        h.leaf_mirror[h.leaf_pair_ptr[g] + q] = h.leaf_pair_ptr[j] + qq;
      }
    }
  h.leaf_blk_off[h.leaf_pair_ptr[nleaf]] = tot;
  if (h.opt.hbm_budget_bytes > 0 && (int64_t)(tot * 8) > h.opt.hbm_budget_bytes)
    throw StatusError(H2_ERR_BUDGET, "leaf near blocks alone need " + std::to_string(tot * 8) + " bytes");
  h.leaf_blk.alloc(std::max<size_t>(1, tot) * 8);
  {
    Scratch sc(s);
    std::vector<AsmTask> tasks;
    int maxc = 0;
    for (int g = 0; g < nleaf; ++g)
      for (size_t q = 0; q < h.leaf_near[g].size(); ++q) {
        int j = h.leaf_near[g][q];
        if (g > j) continue;
        AsmTask a;
        a.out = h.leaf_blk.as<double>() + h.leaf_blk_off[h.leaf_pair_ptr[g] + q];
        a.ridx = nullptr;
        a.cidx = nullptr;
        a.r0 = (int)h.leaf_s[g];
        a.c0 = (int)h.leaf_s[j];
        a.nr = h.leaf_n[g];
        a.nc = h.leaf_n[j];
        a.ld = h.leaf_n[g];
        tasks.push_back(a);
        maxc = std::max(maxc, a.nc);
      }
    for (size_t o = 0; o < tasks.size(); o += (1u << 20)) {
      std::vector<AsmTask> sub(tasks.begin() + o, tasks.begin() + std::min(tasks.size(), o + (1u << 20)));
      run_assemble(Prec::F64, sub, 256, maxc, pts, h.kp, sc);
    }
    H2_CUDA(cudaStreamSynchronize(s));
  }
  // operator bases, height by height
  std::vector<int64_t> samp;
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    Scratch sc(s);
    ht.n_op.resize(ht.nb);
    ht.r_op.resize(ht.nb);
    ht.cand_op.resize(ht.nb);
    ht.sk_op.resize(ht.nb);
    for (int g = 0; g < ht.nb; ++g) {
      const BoxRef& b = ht.ref[g];
      const Problem& pb = h.probs[b.prob];
      if (H == 0) {
        const Box& bx = pb.t.boxes[b.level][b.local];
        ht.cand_op[g].resize(bx.e - bx.s);
        for (int64_t q = bx.s; q < bx.e; ++q) ht.cand_op[g][q - bx.s] = (int)(pb.off + q);
      }
      ht.n_op[g] = (int)ht.cand_op[g].size();
    }
    // samples and fold
    std::vector<int> samp_all;
    std::vector<size_t> samp_off(ht.nb + 1, 0);
    std::vector<int> cand_all;
    std::vector<size_t> cand_off(ht.nb + 1, 0);
    for (int g = 0; g < ht.nb; ++g) {
      const BoxRef& b = ht.ref[g];
      const Problem& pb = h.probs[b.prob];
      far_samples(pb.t, b.level, b.local, h.opt.far_s0, h.opt.far_smin, samp);
      for (int64_t q : samp) samp_all.push_back((int)(pb.off + q));
      samp_off[g + 1] = samp_all.size();
      cand_all.insert(cand_all.end(), ht.cand_op[g].begin(), ht.cand_op[g].end());
      cand_off[g + 1] = cand_all.size();
    }
    int* d_samp = sc.up(samp_all);
    int* d_cand = sc.up(cand_all);
    std::vector<size_t> r_off(ht.nb + 1, 0);
    for (int g = 0; g < ht.nb; ++g) r_off[g + 1] = r_off[g] + (size_t)ht.n_op[g] * ht.n_op[g];
    double* R0 = (double*)sc.alloc(r_off[ht.nb] * 8, true);
    double* Rq = (double*)sc.alloc(r_off[ht.nb] * 8, true);
    int* piv = (int*)sc.alloc(cand_off[ht.nb] * 4);
    int* rank = (int*)sc.alloc(ht.nb * 4);
    std::vector<FoldTask> ft;
    std::vector<PqrTask> qt;
    std::vector<int> has_far(ht.nb, 0);
    for (int g = 0; g < ht.nb; ++g) {
      int n = ht.n_op[g];
      int m = (int)(samp_off[g + 1] - samp_off[g]);
      if (m == 0 || n == 0) continue;
      has_far[g] = 1;
      ft.push_back(FoldTask{d_cand + cand_off[g], d_samp + samp_off[g], R0 + r_off[g], n, m});
      qt.push_back(PqrTask{R0 + r_off[g], n, n, n, piv + cand_off[g], Rq + r_off[g], rank + g, h.opt.tol,
                           h.opt.max_rank});
    }
    {
      int maxn = 0;
      for (const FoldTask& t : ft) maxn = std::max(maxn, t.n);
      launch_fold(sc.up(ft), (int)ft.size(), maxn, nullptr, pts, h.kp, s);
    }
    launch_pqr(sc.up(qt), (int)qt.size(), s);
    std::vector<int> hr(ht.nb), hpiv(cand_off[ht.nb]);
    H2_CUDA(cudaMemcpyAsync(hr.data(), rank, ht.nb * 4, cudaMemcpyDeviceToHost, s));
    if (!hpiv.empty())
      H2_CUDA(cudaMemcpyAsync(hpiv.data(), piv, hpiv.size() * 4, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    // ID: T = R11^-1 R12, P = interpolation matrix; sk = cand[piv[:r]]
    std::vector<TrsmTask> tt;
    std::vector<InterpTask> it;
    ht.P_op.resize(ht.nb);
    int maxrhs = 0;
    for (int g = 0; g < ht.nb; ++g) {
      int n = ht.n_op[g];
      int r = has_far[g] ? hr[g] : n;
      if (r == 0) r = n;   // empty far field or zero block row: keep every point
      bool keep_all = (!has_far[g]) || hr[g] == 0;
      ht.r_op[g] = r;
      ht.P_op[g] = std::make_shared<DBuf>((size_t)std::max(1, n * r) * 8);
      ht.sk_op[g].resize(r);
      if (keep_all) {
        for (int q = 0; q < r; ++q) ht.sk_op[g][q] = ht.cand_op[g][q];
        launch_fill_eye(Prec::F64, ht.P_op[g]->p, n, n, s);
        continue;
      }
      for (int q = 0; q < r; ++q) ht.sk_op[g][q] = ht.cand_op[g][hpiv[cand_off[g] + q]];
      if (r < n) {
        tt.push_back(TrsmTask{Rq + r_off[g], Rq + r_off[g] + (size_t)r * n, r, n - r, n, n, nullptr});
        maxrhs = std::max(maxrhs, n - r);
      }
      it.push_back(InterpTask{piv + cand_off[g], Rq + r_off[g] + (size_t)r * n, ht.P_op[g]->p, n, r, n});
    }
    run_trsm(Prec::F64, false, false, false, tt, maxrhs, sc);
    run_interp(Prec::F64, it, sc);
    // far skeleton blocks, concatenated per box: K(sk_I, [sk_J for J in far(I)])
    std::vector<int> sk_all;
    std::vector<size_t> sk_off(ht.nb + 1, 0);
    for (int g = 0; g < ht.nb; ++g) {
      sk_all.insert(sk_all.end(), ht.sk_op[g].begin(), ht.sk_op[g].end());
      sk_off[g + 1] = sk_all.size();
    }
    ht.kcat_off.assign(ht.nb + 1, 0);
    ht.kcat_cols.assign(ht.nb, 0);
    ht.fg_off.assign(ht.nb + 1, 0);
    std::vector<int> colpts;      // far skeleton points, per box concatenated
    std::vector<int> gidx;        // their positions in the height's skeleton vector
    std::vector<int64_t> xo(ht.nb + 1, 0);
    for (int g = 0; g < ht.nb; ++g) xo[g + 1] = xo[g] + ht.r_op[g];
    for (int g = 0; g < ht.nb; ++g) {
      int cols = 0;
      for (int j : ht.far[g]) {
        colpts.insert(colpts.end(), ht.sk_op[j].begin(), ht.sk_op[j].end());
        for (int q = 0; q < ht.r_op[j]; ++q) gidx.push_back((int)(xo[j] + q));
        cols += ht.r_op[j];
      }
      ht.kcat_cols[g] = cols;
      ht.kcat_off[g + 1] = ht.kcat_off[g] + (size_t)ht.r_op[g] * cols;
      ht.fg_off[g + 1] = ht.fg_off[g] + cols;
    }
    ht.fg_len = ht.fg_off[ht.nb];
    int* d_sk = sc.up(sk_all);
    int* d_cols = sc.up(colpts);
    ht.Kcat_op = std::make_shared<DBuf>(std::max<size_t>(1, ht.kcat_off[ht.nb]) * 8);
    ht.far_gidx = std::make_shared<DBuf>(std::max<size_t>(1, gidx.size()) * 4);
    if (!gidx.empty())
      H2_CUDA(cudaMemcpy(ht.far_gidx->p, gidx.data(), gidx.size() * 4, cudaMemcpyHostToDevice));
    std::vector<AsmTask> at;
    int maxc = 0;
    for (int g = 0; g < ht.nb; ++g) {
      if (ht.kcat_cols[g] == 0) continue;
      // stored transposed: K(far skeletons, sk_I), so each output row of the
      // far product is a contiguous column (warp dot products in the matvec)
      at.push_back(AsmTask{ht.Kcat_op->as<double>() + ht.kcat_off[g], d_cols + ht.fg_off[g], d_sk + sk_off[g], 0, 0,
                           ht.kcat_cols[g], ht.r_op[g], ht.kcat_cols[g]});
      maxc = std::max(maxc, ht.r_op[g]);
    }
    run_assemble(Prec::F64, at, 256, maxc, pts, h.kp, sc);
    // skeleton-vector offsets
    ht.xh_off.assign(ht.nb + 1, 0);
    for (int g = 0; g < ht.nb; ++g) ht.xh_off[g + 1] = ht.xh_off[g] + ht.r_op[g];
    ht.xh_len = ht.xh_off[ht.nb];
    // next height's candidates
    if (H + 1 < h.Hmax) {
      Height& up = h.hs[H + 1];
      up.cand_op.resize(up.nb);
      for (int g = 0; g < ht.nb; ++g) {
        int pg = ht.parent[g];
        if (pg < 0) continue;
        auto& c = up.cand_op[pg];
        c.insert(c.end(), ht.sk_op[g].begin(), ht.sk_op[g].end());
      }
    }
    H2_CUDA(cudaStreamSynchronize(s));
  }
}

// ------------------------------------------------------------- matvec ----
// Plan of y = A_H2 x in tree order (N x nrhs, column-major, ld = Ntot).
static PlanP build_matvec_plan(Handle& h, const double* x, double* y, int nrhs) {
  auto P = std::make_shared<Plan>();
  Plan& pl = *P;
  const int64_t ld = h.Ntot;
  // near part (leaf dense blocks): y_I = sum_J A_IJ x_J
  pl.tag("mv_near");
  if (nrhs <= 2) {
    // each stored block read once: partials for both boxes, then a fixed-order sum
    std::vector<SymPairTask> st;
    std::vector<size_t> pofs(h.leaf_pair_ptr.back(), 0);   // partial offset seen by pair (g, q)
    long long tot = 0;
    for (size_t g = 0; g < h.leaf_ref.size(); ++g)
      for (size_t q = 0; q < h.leaf_near[g].size(); ++q) {
        int j = h.leaf_near[g][q];
        if ((int)g > j) continue;
        SymPairTask t;
        t.A = h.leaf_blk.as<double>() + h.leaf_blk_off[h.leaf_pair_ptr[g] + q];
        t.nI = h.leaf_n[g];
        t.nJ = h.leaf_n[j];
        t.lda = h.leaf_n[g];
        t.sI = h.leaf_s[g];
        t.sJ = h.leaf_s[j];
        t.uo = tot;
        tot += (long long)t.nI * nrhs;
        t.vo = tot;
        tot += (long long)t.nJ * nrhs;
        pofs[h.leaf_pair_ptr[g] + q] = (size_t)t.uo;
        if ((int)g != j) {
          const auto& nl = h.leaf_near[j];
          size_t qq = std::find(nl.begin(), nl.end(), (int)g) - nl.begin();
          pofs[h.leaf_pair_ptr[j] + qq] = (size_t)t.vo;
        }
        st.push_back(t);
      }
    double* part = pl.work((size_t)tot);
    std::vector<GatherTask> gt;
    std::vector<long long> offs;
    for (size_t g = 0; g < h.leaf_ref.size(); ++g) {
      GatherTask t;
      t.s = h.leaf_s[g];
      t.n = h.leaf_n[g];
      t.p0 = (int)offs.size();
      for (size_t q = 0; q < h.leaf_near[g].size(); ++q) offs.push_back((long long)pofs[h.leaf_pair_ptr[g] + q]);
      t.np = (int)(offs.size() - t.p0);
      gt.push_back(t);
    }
    pl.symv(st, x, ld, part, nrhs);
    pl.gather(gt, offs, part, y, ld, nrhs);
  } else {
    GemmBatch gb;
    for (size_t g = 0; g < h.leaf_ref.size(); ++g) {
      std::vector<GemmTerm> ts;
      for (size_t q = 0; q < h.leaf_near[g].size(); ++q) {
        int j = h.leaf_near[g][q];
        BlkRef br = leaf_block(h, (int)g, q);
        ts.push_back(GemmTerm{br.ptr, x + h.leaf_s[j], h.leaf_n[j], br.ld, (int)ld, br.tr});
      }
      gb.add(y + h.leaf_s[g], (int)ld, h.leaf_n[g], nrhs, 1.0, 0.0, nullptr, 0, ts);
    }
    pl.gemm(Prec::F64, gb, false, false);
  }
  pl.tag("mv_far");
  if (h.Hmax == 0) return P;
  // upward pass
  std::vector<double*> xh(h.Hmax), yh(h.Hmax);
  for (int H = 0; H < h.Hmax; ++H) {
    xh[H] = pl.work((size_t)h.hs[H].xh_len * nrhs);
    yh[H] = pl.work((size_t)h.hs[H].xh_len * nrhs, true);
  }
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    GemmBatch gb;
    for (int g = 0; g < ht.nb; ++g) {
      const double* src;
      int64_t lds;
      if (H == 0) {
        const BoxRef& b = ht.ref[g];
        const Problem& pb = h.probs[b.prob];
        src = x + pb.off + pb.t.boxes[b.level][b.local].s;
        lds = ld;
      } else {
        // children a, b are adjacent in the skeleton vector of height H-1
        const Height& dn = h.hs[H - 1];
        int a = ht.first_child[g];
        src = xh[H - 1] + dn.xh_off[a];
        lds = dn.xh_len;
      }
      gb.add1(xh[H] + ht.xh_off[g], (int)ht.xh_len, ht.r_op[g], nrhs, ht.P_op[g]->p, ht.n_op[g], src, (int)lds,
              ht.n_op[g]);
    }
    pl.gemm(Prec::F64, gb, true, false);
  }
  // far interactions at every height: gather the far skeleton values of
  // each box into one contiguous vector, then one product per box with its
  // concatenated far block (every box gets a task, so the skeleton vectors
  // are overwritten on each replay)
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    double* xg = pl.work(std::max<size_t>(1, ht.fg_len) * nrhs);
    if (ht.fg_len)
      pl.gather_rows(xh[H], ht.xh_len, xg, (long long)ht.fg_len, ht.far_gidx->as<int>(), (long long)ht.fg_len, nrhs);
    GemmBatch gb;
    for (int g = 0; g < ht.nb; ++g) {
      std::vector<GemmTerm> ts;
      if (ht.kcat_cols[g])
        ts.push_back(GemmTerm{ht.Kcat_op->as<double>() + ht.kcat_off[g], xg + ht.fg_off[g], ht.kcat_cols[g],
                              ht.kcat_cols[g], (int)ht.fg_len, 1});
      gb.add(yh[H] + ht.xh_off[g], (int)ht.xh_len, ht.r_op[g], nrhs, 1.0, 0.0, nullptr, 0, ts);
    }
    pl.gemm(Prec::F64, gb, false, false);
  }
  // downward pass: yh(children) += P_P yh(P)
  for (int H = h.Hmax - 1; H >= 1; --H) {
    Height& ht = h.hs[H];
    const Height& dn = h.hs[H - 1];
    GemmBatch gb;
    for (int g = 0; g < ht.nb; ++g) {
      int a = ht.first_child[g];
      double* dst = yh[H - 1] + dn.xh_off[a];
      gb.add1(dst, (int)dn.xh_len, ht.n_op[g], nrhs, ht.P_op[g]->p, ht.n_op[g], yh[H] + ht.xh_off[g],
              (int)ht.xh_len, ht.r_op[g], 1.0, 1.0);
    }
    pl.gemm(Prec::F64, gb, false, false);
  }
  // leaf: y_I += P_I yh(I)
  {
    Height& ht = h.hs[0];
    GemmBatch gb;
    for (int g = 0; g < ht.nb; ++g) {
      const BoxRef& b = ht.ref[g];
      const Problem& pb = h.probs[b.prob];
      double* dst = y + pb.off + pb.t.boxes[b.level][b.local].s;
      gb.add1(dst, (int)ld, ht.n_op[g], nrhs, ht.P_op[g]->p, ht.n_op[g], yh[0] + ht.xh_off[g], (int)ht.xh_len,
              ht.r_op[g], 1.0, 1.0);
    }
    pl.gemm(Prec::F64, gb, false, false);
  }
  return P;
}

// ------------------------------------------------------------ root LU ----
// Blocked right-looking LU with partial pivoting of the dense top-level
// matrix (eq. BLR2final), then its inverse (the root solve becomes a GEMM).
// Factor the top-level dense matrix in precision P (in place in `Aw`, n x n,
// column-major): LU, log-determinant and the explicit inverse (FP64 in
// rt.inv, FP64 copy of the factors in rt.LU).  Mixed precision runs it in
// FP32 on the tensor-core GEMM: the root only preconditions there.
// The zero-pivot flag goes to `info` and log|det|, sign to `dlog` (device);
// the caller reads both once the whole factorization has been issued.
static void root_factor(Handle& h, Root& rt, int spd, Prec P, void* Aw, int* info, double* dlog) {
  cudaStream_t s = h.s;
  const int n = rt.n;
  if (n == 0) return;
  if (n > 8192) throw StatusError(H2_ERR_ARG, "top-level dense matrix larger than 8192");
  Scratch sc(s);
  const size_t es = esz(P);
  auto at = [&](void* base, size_t i, size_t j) -> char* { return (char*)base + (i + j * (size_t)n) * es; };
  int* piv = rt.piv->as<int>();
  // Blocked right-looking LU with pivoting inside each 64 x 64 diagonal
  // block: the panel factorization touches only that block (one CTA, L2
  // resident), and L21 = A21 U11^-1, U12 = L11^-1 A12 and the trailing
  // update are batched over the whole width.  The factorization is exact
  // (A = P L U, P a product of in-block row swaps).
  const int NB = 64;
  void* Tbuf = sc.alloc((size_t)NB * n * es);
  for (int k = 0; k < n; k += NB) {
    int nb = std::min(NB, n - k);
    const int rest = n - k - nb;
    std::vector<LuTask> lt{LuTask{at(Aw, k, k), nb, nb, n, piv + k, info, spd ? 1 : 0}};
    run_getrf(P, lt, sc);
    // block-relative pivots -> absolute rows, then swap the other columns
    launch_add_offset(piv + k, nb, k, s);
    launch_laswp_cols(P, Aw, n, n, piv, k, k + nb, 0, k, s);
    launch_laswp_cols(P, Aw, n, n, piv, k, k + nb, k + nb, n, s);
    if (rest > 0) {
      // U12 = L11^-1 A12
      std::vector<TrsmTask> tt{TrsmTask{at(Aw, k, k), at(Aw, k, k + nb), nb, rest, n, n, nullptr}};
      run_trsm(P, true, true, false, tt, rest, sc);
      // L21 = A21 U11^-1  via  U11^T L21^T = A21^T
      void* A21 = at(Aw, k + nb, k);
      std::vector<CopyTask> c1{CopyTask{A21, Tbuf, nb, rest, n, nb}};
      run_copy(P, P, true, c1, nb, rest, sc);
      std::vector<TrsmTask> t2{TrsmTask{at(Aw, k, k), Tbuf, nb, rest, n, nb, nullptr}};
      run_trsm(P, true, false, true, t2, rest, sc);
      std::vector<CopyTask> c2{CopyTask{Tbuf, A21, rest, nb, nb, n}};
      run_copy(P, P, true, c2, rest, nb, sc);
      // A22 -= L21 U12
      GemmBatch gb;
      gb.add1(at(Aw, k + nb, k + nb), n, rest, rest, A21, n, at(Aw, k, k + nb), n, nb, -1.0, 1.0);
      gb.run(P, false, false, sc);
    }
  }
  double* LU = rt.LU->as<double>();
  if (P != Prec::F64) {
    std::vector<CopyTask> ct{CopyTask{Aw, LU, n, n, n, n}};
    run_copy(P, Prec::F64, false, ct, n, n, sc);
  }
  // log-determinant (read by the caller with the other deferred results)
  {
    std::vector<LuTask> lt{LuTask{LU, n, n, n, piv, nullptr, 0}};
    launch_logdet_lu(sc.up(lt), 1, dlog, dlog + 1, false, s);
  }
  // inverse: X = U^-1 L^-1 P I, blocked by 256-row panels
  rt.inv = std::make_shared<DBuf>((size_t)n * n * 8);
  void* X = (P == Prec::F64) ? rt.inv->p : sc.alloc((size_t)n * n * es);
  launch_fill_eye(P, X, n, n, s);
  launch_laswp_cols(P, X, n, n, piv, 0, n, 0, n, s);
  const int TB = 256;
  // forward: L (unit lower)
  for (int k = 0; k < n; k += TB) {
    int nb = std::min(TB, n - k);
    std::vector<TrsmTask> tt{TrsmTask{at(Aw, k, k), at(X, k, 0), nb, n, n, n, nullptr}};
    run_trsm(P, true, true, false, tt, n, sc);
    if (k + nb < n) {
      GemmBatch gb;
      gb.add1(at(X, k + nb, 0), n, n - k - nb, n, at(Aw, k + nb, k), n, at(X, k, 0), n, nb, -1.0, 1.0);
      gb.run(P, false, false, sc);
    }
  }
  // backward: U (upper)
  for (int k = ((n - 1) / TB) * TB; k >= 0; k -= TB) {
    int nb = std::min(TB, n - k);
    std::vector<TrsmTask> tt{TrsmTask{at(Aw, k, k), at(X, k, 0), nb, n, n, n, nullptr}};
    run_trsm(P, false, false, false, tt, n, sc);
    if (k > 0) {
      GemmBatch gb;
      gb.add1(X, n, k, n, at(Aw, 0, k), n, at(X, k, 0), n, nb, -1.0, 1.0);
      gb.run(P, false, false, sc);
    }
  }
  if (P != Prec::F64) {
    std::vector<CopyTask> ct{CopyTask{X, rt.inv->p, n, n, n, n}};
    run_copy(P, Prec::F64, false, ct, n, n, sc);
  }
}

// ------------------------------------------------------------- factor ----
struct PairRef {
  void* ptr;   // stored block (work precision)
  int ld;
  int tr;      // 1: the pair's block is the transpose of the stored one
};

static void factor(Handle& h, int precision, int spd) {
  cudaStream_t s = h.s;
  const Prec W = precision == H2_MIXED ? Prec::F32 : Prec::F64;
  const size_t ws = esz(W);
  Points pts = points(h);
  h.level_ms.clear();
  // Results read back once, after the whole factorization has been issued:
  // [0] zero / non-positive pivot in a redundant-block LU (any height),
  // [1] zero pivot in the top-level LU of a problem, then per problem the
  // top-level log|det| and sign.  Only the ranks are read per height.
  Scratch fsc(s);
  const size_t P = h.probs.size();
  int* dflags = (int*)fsc.alloc(16, true);
  double* droot = (double*)fsc.alloc(std::max<size_t>(1, P) * 16, true);
  // scratch budget of the batched pair products (fill-in Gram, projection)
  size_t pair_budget = size_t(256) << 20;
  {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess)
      pair_budget = std::min<size_t>(size_t(4) << 30, std::max<size_t>(pair_budget, fr / 8));
  }
  std::vector<cudaEvent_t> hev;   // per-height start/end events (factor_ms per level)
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (cudaEvent_t e : v) cudaEventDestroy(e);
    }
  } evguard{hev};
  // near blocks of the current height, in work precision: A[g][q] for the
  // q-th near box of g
  std::vector<std::vector<PairRef>> Ablk;
  std::vector<DBufP> Aown;       // storage owned for the current height
  // height-0 inputs: the FP64 leaf near blocks (converted in mixed mode)
  std::vector<int> ncur;
  for (auto& pb : h.probs) {
    pb.root = Root();
  }
  // problems with no ULV height: root = their leaf level (all pairs near)
  auto setup_root = [&](Problem& pb, const std::vector<int>& sizes) {
    Root& rt = pb.root;
    rt.off.assign(sizes.size() + 1, 0);
    for (size_t i = 0; i < sizes.size(); ++i) rt.off[i + 1] = rt.off[i] + sizes[i];
    rt.n = rt.off.back();
    if (rt.n > 8192) throw StatusError(H2_ERR_ARG, "top-level dense matrix larger than 8192");
    rt.A = std::make_shared<DBuf>((size_t)rt.n * rt.n * ws);
    H2_CUDA(cudaMemsetAsync(rt.A->p, 0, rt.A->bytes, s));
    rt.LU = std::make_shared<DBuf>((size_t)rt.n * rt.n * 8);
    rt.piv = std::make_shared<DBuf>((size_t)rt.n * 4);
  };
  {
    Scratch sc(s);
    for (size_t p = 0; p < h.probs.size(); ++p) {
      Problem& pb = h.probs[p];
      if (pb.H > 0) continue;
      std::vector<int> sizes;
      for (auto& bx : pb.t.boxes[pb.t.L]) sizes.push_back((int)(bx.e - bx.s));
      setup_root(pb, sizes);
      // copy the leaf blocks into the root matrix
      std::vector<CopyTask> ct[2];
      int maxr = 0, maxc = 0;
      for (size_t g = 0; g < h.leaf_ref.size(); ++g) {
        if (h.leaf_ref[g].prob != (int)p) continue;
        int i = h.leaf_ref[g].local;
        for (size_t q = 0; q < h.leaf_near[g].size(); ++q) {
          int jg = h.leaf_near[g][q];
          int j = h.leaf_ref[jg].local;
          BlkRef br = leaf_block(h, (int)g, q);
          ct[br.tr].push_back(CopyTask{br.ptr,
                                (char*)pb.root.A->p + ((size_t)pb.root.off[i] + (size_t)pb.root.off[j] * pb.root.n) * ws,
                                h.leaf_n[g], h.leaf_n[jg], br.ld, pb.root.n});
          maxr = std::max(maxr, h.leaf_n[g]);
          maxc = std::max(maxc, h.leaf_n[jg]);
        }
      }
      run_copy(Prec::F64, W, false, ct[0], maxr, maxc, sc);
      run_copy(Prec::F64, W, true, ct[1], maxr, maxc, sc);
    }
    H2_CUDA(cudaStreamSynchronize(s));
  }
  if (h.Hmax > 0) {
    Height& h0 = h.hs[0];
    Ablk.assign(h0.nb, {});
    // map height-0 ids to leaf ids
    std::vector<int> leaf_of(h0.nb);
    {
      std::map<std::pair<int, int>, int> lid;
      for (size_t g = 0; g < h.leaf_ref.size(); ++g) lid[{h.leaf_ref[g].prob, h.leaf_ref[g].local}] = (int)g;
      for (int g = 0; g < h0.nb; ++g) leaf_of[g] = lid[{h0.ref[g].prob, h0.ref[g].local}];
    }
    if (W == Prec::F64) {
      for (int g = 0; g < h0.nb; ++g) {
        int lg = leaf_of[g];
        for (size_t q = 0; q < h0.near[g].size(); ++q) {
          BlkRef br = leaf_block(h, lg, q);
          Ablk[g].push_back(PairRef{(void*)br.ptr, br.ld, br.tr});
        }
      }
    } else {
      // FP32 copy of the stored (i <= j) leaf near blocks for the mixed pass
      size_t tot = h.leaf_blk_off[h.leaf_pair_ptr[h.leaf_ref.size()]];
      auto buf = cached_or_new(std::max<size_t>(1, tot) * 4, s);
      Aown.push_back(buf);
      Scratch sc(s);
      std::vector<CopyTask> ct;
      int maxr = 0, maxc = 0;
      for (size_t lg = 0; lg < h.leaf_ref.size(); ++lg)
        for (size_t q = 0; q < h.leaf_near[lg].size(); ++q) {
          int jg = h.leaf_near[lg][q];
          if ((int)lg > jg) continue;
          size_t o = h.leaf_blk_off[h.leaf_pair_ptr[lg] + q];
          ct.push_back(CopyTask{h.leaf_blk.as<double>() + o, buf->as<float>() + o, h.leaf_n[lg], h.leaf_n[jg],
                                h.leaf_n[lg], h.leaf_n[lg]});
          maxr = std::max(maxr, h.leaf_n[lg]);
          maxc = std::max(maxc, h.leaf_n[jg]);
        }
      run_copy(Prec::F64, Prec::F32, false, ct, maxr, maxc, sc);
      for (int g = 0; g < h0.nb; ++g) {
        int lg = leaf_of[g];
        for (size_t q = 0; q < h0.near[g].size(); ++q) {
          BlkRef br = leaf_block(h, lg, q);
          size_t o = (size_t)(br.ptr - h.leaf_blk.as<double>());
          Ablk[g].push_back(PairRef{buf->as<float>() + o, br.ld, br.tr});
        }
      }
      H2_CUDA(cudaStreamSynchronize(s));
    }
    h0.n.resize(h0.nb);
    h0.cand.resize(h0.nb);
    for (int g = 0; g < h0.nb; ++g) {
      h0.n[g] = h.leaf_n[leaf_of[g]];
      h0.cand[g].resize(h0.n[g]);
      for (int q = 0; q < h0.n[g]; ++q) h0.cand[g][q] = (int)(h.leaf_s[leaf_of[g]] + q);
    }
  }
  DBufP Tcur;                       // per box n x n FP64 transforms (H > 0)
  std::vector<size_t> t_off;
  std::vector<int64_t> samp;
  for (int H = 0; H < h.Hmax; ++H) {
    {
      cudaEvent_t e0;
      H2_CUDA(cudaEventCreate(&e0));
      hev.push_back(e0);
      H2_CUDA(cudaEventRecord(e0, s));
    }
    Height& ht = h.hs[H];
    Scratch sc(s);
    const int nb = ht.nb;
    void* pbuf = nullptr;
    size_t pcap = 0;
    auto pair_buf = [&](size_t need) -> void* {   // one buffer shared by the stream-ordered pair loops
      if (need > pcap) {
        pbuf = sc.alloc(need);
        pcap = need;
      }
      return pbuf;
    };
    std::vector<int>& n = ht.n;
    // n x n slots
    std::vector<size_t> off(nb + 1, 0);
    for (int g = 0; g < nb; ++g) off[g + 1] = off[g] + (size_t)n[g] * n[g];
    const size_t NN = off[nb];
    int maxn = 0;
    for (int g = 0; g < nb; ++g) maxn = std::max(maxn, n[g]);
    auto diag_q = [&](int g) -> int {
      for (size_t q = 0; q < ht.near[g].size(); ++q)
        if (ht.near[g][q] == g) return (int)q;
      return -1;
    };
    // ---------------- 0. predicted ranks: size the next level up front -----
    Height* upp = (H + 1 < h.Hmax) ? &h.hs[H + 1] : nullptr;
    std::vector<int> rcap;
    DBufP Apre;                          // next-level storage sized from predictions
    std::vector<std::vector<size_t>> pre_off;
    std::vector<int> pre_ld;
    if (h.predictor && upp) {
      prof_tag("predict");
      std::vector<float> Fh;
      height_features(h, H, Fh);
      const Mlp& m = *h.predictor;
      float* dX = (float*)sc.alloc(Fh.size() * 4);
      float* dH1 = (float*)sc.alloc((size_t)nb * MLP_WIDTH * 4);
      float* dH2 = (float*)sc.alloc((size_t)nb * MLP_WIDTH * 4);
      float* dY = (float*)sc.alloc((size_t)nb * 4);
      H2_CUDA(cudaMemcpyAsync(dX, pinned_stage(Fh.data(), Fh.size() * 4, s), Fh.size() * 4, cudaMemcpyHostToDevice, s));
      mlp_forward(m.prm, m.F, dX, nb, dH1, dH2, dY, nullptr, nullptr, s);
      std::vector<float> yh(nb);
      H2_CUDA(cudaMemcpyAsync(yh.data(), dY, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
      H2_CUDA(cudaStreamSynchronize(s));
      rcap.resize(nb);
      for (int g = 0; g < nb; ++g) {
        double rh = std::max(0.0, (double)yh[g]) * h.opt.max_rank;
        int c = (int)std::ceil(rh * (1.0 + h.pred_margin)) + 4;
        rcap[g] = std::max(1, std::min({c, n[g], h.opt.max_rank}));
      }
      std::vector<int> ncap(upp->nb, 0);
      for (int g = 0; g < nb; ++g)
        if (ht.parent[g] >= 0) ncap[ht.parent[g]] += rcap[g];
      size_t tot = 0, worst = 0;
      pre_off.assign(upp->nb, {});
      pre_ld = ncap;
      for (int pg = 0; pg < upp->nb; ++pg)
        for (int qg : upp->near[pg]) {
          pre_off[pg].push_back(tot);
          if (pg <= qg) {
            tot += (size_t)ncap[pg] * ncap[qg];
            worst += (size_t)(2 * h.opt.max_rank) * (2 * h.opt.max_rank);
          }
        }
      Apre = std::make_shared<DBuf>(std::max<size_t>(1, tot) * ws);
      h.pred_bytes += (double)tot * ws;
      h.worst_bytes += (double)worst * ws;
    }
    // ---------------- 1. fill-ins (Sec. III-B) --------------------------
    // Two routes to the basis of eq. fillu.
    // QR route: the fill-ins of row I share, per K, the row factor
    // A_KK^-1 [A_KJ]_J, whose column space is that of Z_K = A_KK^-1 R_K^T
    // with R_K the Householder triangle of [A_KJ]_J^T, so row I holds the
    // n x n blocks V_IK = A_IK Z_K; they and the far field are folded by
    // Householder QR and the pivoted QR decides (nothing is squared).
    // Gram route: the Gram matrix of the same block row (sum of GEMMs, on
    // the tensor cores in mixed precision) and pivoted Cholesky.  Squaring
    // the block row leaves its Gram with rounding noise of order eps times
    // its norm, so FP64 keeps the Gram route only while the rank threshold
    // tol^2 G_11 stays at least 2^12 units of roundoff above that noise
    // (tol >= 2^6 sqrt(eps) = 2^-20) and takes the QR route below; mixed
    // precision takes the Gram route with the 2^-10 floor below.
    const bool qr_route = (W == Prec::F64) && h.opt.tol < 0x1p-20;
    prof_tag("fillin");
    std::vector<int> has_lu(nb, 0);
    for (int g = 0; g < nb; ++g) has_lu[g] = ht.near[g].size() > 1;
    // scratch slots of maxn x maxn per box (V blocks are n_I x n_K)
    const size_t SL = (size_t)maxn * maxn;
    std::vector<size_t> so(nb + 1, 0);
    for (int g = 0; g <= nb; ++g) so[g] = (size_t)g * SL;
    int* finfo = (int*)sc.alloc(4, true);
    void* LUK = sc.alloc(so[nb] * ws);
    int* pivK = (int*)sc.alloc((size_t)nb * NMAX * 4);
    void* Mk = sc.alloc(so[nb] * ws, true);
    void* Tmp = sc.alloc(so[nb] * ws);
    {
      std::vector<CopyTask> ct;
      std::vector<LuTask> lu;
      GemmBatch ng;
      std::vector<FoldTask> fk;
      std::vector<FoldTerm> fkt;
      for (int g = 0; g < nb; ++g) {
        if (!has_lu[g]) continue;
        int dq = diag_q(g);
        void* dst = (char*)LUK + so[g] * ws;
        ct.push_back(CopyTask{Ablk[g][dq].ptr, dst, n[g], n[g], Ablk[g][dq].ld, n[g]});
        lu.push_back(LuTask{dst, n[g], n[g], n[g], pivK + (size_t)g * NMAX, finfo, 0});
        if (qr_route) {
          // R_K: rows of [A_KJ]_J^T = columns of every A_KJ, J != K
          FoldTask f{};
          f.R = (double*)((char*)Mk + so[g] * ws);
          f.n = n[g];
          f.t0 = (int)fkt.size();
          for (size_t q = 0; q < ht.near[g].size(); ++q) {
            int j = ht.near[g][q];
            if (j == g) continue;
            fkt.push_back(FoldTerm{(const double*)Ablk[g][q].ptr, n[j], Ablk[g][q].ld, Ablk[g][q].tr});
          }
          f.nt = (int)fkt.size() - f.t0;
          fk.push_back(f);
          continue;
        }
        std::vector<GemmTerm> ts;
        for (size_t q = 0; q < ht.near[g].size(); ++q) {
          int j = ht.near[g][q];
          if (j == g) continue;
          int t = Ablk[g][q].tr;
          ts.push_back(GemmTerm{Ablk[g][q].ptr, Ablk[g][q].ptr, n[j], Ablk[g][q].ld, Ablk[g][q].ld, t ? 3 : 0});
        }
        ng.add((char*)Mk + so[g] * ws, n[g], n[g], n[g], 1.0, 0.0, nullptr, 0, ts);
      }
      run_copy(W, W, false, ct, maxn, maxn, sc);
      run_getrf(W, lu, sc);
      if (qr_route) run_fold(fk, fkt, pts, h.kp, sc);
      else ng.run(W, false, true, sc);
    }
    if (W == Prec::F32) {
      // mixed precision: M_K = A_KK^-1 NG_K A_KK^-T through the explicit
      // inverse A_KK^-1 = U^-1 L^-1 P (two triangular solves on the
      // identity) and two tensor-core GEMMs
      void* I256 = sc.alloc((size_t)NMAX * NMAX * ws);
      launch_fill_eye(W, I256, NMAX, NMAX, s);
      std::vector<CopyTask> ci;
      std::vector<TrsmTask> tl, tu;
      GemmBatch x1, x2;
      for (int g = 0; g < nb; ++g) {
        if (!has_lu[g]) continue;
        void* L = (char*)LUK + so[g] * ws;
        void* Ai = (char*)Tmp + so[g] * ws;
        void* M = (char*)Mk + so[g] * ws;
        ci.push_back(CopyTask{I256, Ai, n[g], n[g], NMAX, n[g]});
        tl.push_back(TrsmTask{L, Ai, n[g], n[g], n[g], n[g], pivK + (size_t)g * NMAX});
        tu.push_back(TrsmTask{L, Ai, n[g], n[g], n[g], n[g], nullptr});
        x1.add1(L, n[g], n[g], n[g], Ai, n[g], M, n[g], n[g]);      // X = A^-1 NG (over the LU)
        x2.add1(M, n[g], n[g], n[g], L, n[g], Ai, n[g], n[g]);      // M = X A^-T
      }
      run_copy(W, W, false, ci, maxn, maxn, sc);
      run_trsm(W, true, true, false, tl, maxn, sc);
      run_trsm(W, false, false, false, tu, maxn, sc);
      x1.run(W, false, false, sc);
      x2.run(W, false, true, sc);
    } else if (!qr_route) {
      // M_K = A_KK^-1 NG_K A_KK^-T  (NG symmetric): X = A^-1 NG; M = A^-1 X^T
      std::vector<TrsmTask> tl, tu;
      std::vector<CopyTask> tr;
      for (int g = 0; g < nb; ++g) {
        if (!has_lu[g]) continue;
        void* L = (char*)LUK + so[g] * ws;
        void* M = (char*)Mk + so[g] * ws;
        tl.push_back(TrsmTask{L, M, n[g], n[g], n[g], n[g], pivK + (size_t)g * NMAX});
        tu.push_back(TrsmTask{L, M, n[g], n[g], n[g], n[g], nullptr});
        tr.push_back(CopyTask{M, (char*)Tmp + so[g] * ws, n[g], n[g], n[g], n[g]});
      }
      run_trsm(W, true, true, false, tl, maxn, sc);
      run_trsm(W, false, false, false, tu, maxn, sc);
      run_copy(W, W, true, tr, maxn, maxn, sc);
      std::vector<TrsmTask> tl2, tu2;
      for (int g = 0; g < nb; ++g) {
        if (!has_lu[g]) continue;
        void* L = (char*)LUK + so[g] * ws;
        void* X = (char*)Tmp + so[g] * ws;
        tl2.push_back(TrsmTask{L, X, n[g], n[g], n[g], n[g], pivK + (size_t)g * NMAX});
        tu2.push_back(TrsmTask{L, X, n[g], n[g], n[g], n[g], nullptr});
      }
      run_trsm(W, true, true, false, tl2, maxn, sc);
      run_trsm(W, false, false, false, tu2, maxn, sc);
      std::swap(Mk, Tmp);   // M = Tmp (symmetric up to rounding)
    } else {
      // Z_K = A_KK^-1 R_K^T (P L U = A_KK): transpose R_K, then L and U solves
      std::vector<TrsmTask> tl, tu;
      std::vector<CopyTask> tr;
      for (int g = 0; g < nb; ++g) {
        if (!has_lu[g]) continue;
        void* L = (char*)LUK + so[g] * ws;
        void* Z = (char*)Tmp + so[g] * ws;
        tr.push_back(CopyTask{(char*)Mk + so[g] * ws, Z, n[g], n[g], n[g], n[g]});
        tl.push_back(TrsmTask{L, Z, n[g], n[g], n[g], n[g], pivK + (size_t)g * NMAX});
        tu.push_back(TrsmTask{L, Z, n[g], n[g], n[g], n[g], nullptr});
      }
      run_copy(W, W, true, tr, maxn, maxn, sc);
      run_trsm(W, true, true, false, tl, maxn, sc);
      run_trsm(W, false, false, false, tu, maxn, sc);
      std::swap(Mk, Tmp);
    }
    // Fill-in block row of every box.  Both routes form V_IK = op(A_IK) X_K
    // for a chunk of near positions in one launch (X_K = Z_K or M_K).  The
    // QR route folds the V_IK of a box into its triangle RF one near
    // position after the other; the Gram route forms P_IK = V_IK A_IK^T and
    // adds them into GF in near-position order, so that neither result
    // depends on the chunking.
    void* GF = qr_route ? nullptr : sc.alloc(so[nb] * ws, true);
    double* RF = qr_route ? (double*)sc.alloc(NN * 8, true) : nullptr;
    std::vector<int> has_fill(nb, 0);
    {
      std::vector<PairSlot> prs = near_pairs(ht.near, [&](int g, int K) { return K != g && has_lu[K]; },
                                             [&](int g, int K) {
                                               return ((size_t)n[g] * n[K] + (qr_route ? 0 : (size_t)n[g] * n[g])) * ws;
                                             });
      std::vector<std::vector<int>> by_box(nb);
      for (size_t p0 = 0; p0 < prs.size();) {
        const size_t p1 = chunk_pairs(prs, p0, pair_budget);
        char* Vb = (char*)pair_buf(prs[p1 - 1].off + prs[p1 - 1].bytes);
        GemmBatch g1, g2;
        for (size_t q = p0; q < p1; ++q) {
          const PairSlot& pr = prs[q];
          const int g = pr.g, k = pr.k, K = pr.j;
          char* V = Vb + pr.off;
          g1.add1(V, n[g], n[g], n[K], Ablk[g][k].ptr, Ablk[g][k].ld, (char*)Mk + so[K] * ws, n[K], n[K], 1.0, 0.0,
                  nullptr, 0, Ablk[g][k].tr ? 1 : 0);
          if (!qr_route) {
            char* P = V + (size_t)n[g] * n[K] * ws;
            g2.add1(P, n[g], n[g], n[g], V, n[g], Ablk[g][k].ptr, Ablk[g][k].ld, n[K], 1.0, 0.0, nullptr, 0,
                    Ablk[g][k].tr ? 2 : 0);
          }
          by_box[g].push_back((int)q);
          has_fill[g] = 1;
        }
        g1.run(W, false, false, sc);
        if (qr_route) {
          prof_tag("fillin_fold");
          std::vector<FoldTask> ft;
          std::vector<FoldTerm> fterms;
          for (int g = 0; g < nb; ++g) {
            if (by_box[g].empty()) continue;
            FoldTask f{};
            f.R = RF + off[g];
            f.n = n[g];
            f.t0 = (int)fterms.size();
            f.accumulate = 1;
            for (int q : by_box[g]) fterms.push_back(FoldTerm{(const double*)(Vb + prs[q].off), n[prs[q].j], n[g], 0});
            f.nt = (int)fterms.size() - f.t0;
            ft.push_back(f);
            by_box[g].clear();
          }
          run_fold(ft, fterms, pts, h.kp, sc);
          prof_tag("fillin");
          p0 = p1;
          continue;
        }
        prof_tag("fillin_gram");
        g2.run(W, false, true, sc);
        std::vector<AccumTask> at;
        std::vector<const void*> parts;
        long long maxe = 0;
        for (int g = 0; g < nb; ++g) {
          if (by_box[g].empty()) continue;
          const long long ne = (long long)n[g] * n[g];
          at.push_back(AccumTask{(char*)GF + so[g] * ws, ne, (int)parts.size(), (int)by_box[g].size()});
          for (int q : by_box[g]) parts.push_back(Vb + prs[q].off + (size_t)n[g] * n[prs[q].j] * ws);
          by_box[g].clear();
          maxe = std::max(maxe, ne);
        }
        {
          double by = 0.0;
          for (const AccumTask& a : at) by += (double)ws * a.n * (a.np + 2.0);
          prof_note(0.0, by);
        }
        launch_accum_parts(W, sc.up(at), (int)at.size(), sc.up(parts), maxe, s);
        prof_tag("fillin");
        p0 = p1;
      }
    }
    // ---------------- 2. basis with fill-ins (eq. fillu) ---------------
    prof_tag("basis");
    double* R = (double*)sc.alloc(NN * 8);
    int* piv = (int*)sc.alloc((size_t)nb * NMAX * 4);
    int* rank = (int*)sc.alloc((size_t)nb * 4);
    int* cinfo = (int*)sc.alloc(8, true);   // [0] basis matrix non-finite, [1] fill-in LU zero pivot
    // far-field samples of every box (candidates in point form)
    std::vector<int> cand_all, samp_all;
    std::vector<size_t> co(nb + 1, 0), sof(nb + 1, 0);
    for (int g = 0; g < nb; ++g) {
      const BoxRef& b = ht.ref[g];
      const Problem& pb = h.probs[b.prob];
      far_samples(pb.t, b.level, b.local, h.opt.far_s0, h.opt.far_smin, samp);
      for (int64_t q : samp) samp_all.push_back((int)(pb.off + q));
      sof[g + 1] = samp_all.size();
      cand_all.insert(cand_all.end(), ht.cand[g].begin(), ht.cand[g].end());
      co[g + 1] = cand_all.size();
    }
    int* dc = sc.up(cand_all);
    int* ds = sc.up(samp_all);
    const double tol_basis = (W == Prec::F64) ? h.opt.tol : std::max(h.opt.tol, 1.0 / 1024.0);
    h.tol_basis = tol_basis;
    h.basis_route = qr_route ? "qr" : "gram";
    if (qr_route) {
      // point form of the fill-in rows: B_pt = T^-1 B_lev, and B_lev B_lev^T
      // = RF^T RF, so Y = T^-1 RF^T stands for them; fold [Y^T; far-field
      // rows] and take the pivoted QR of the triangle (at the leaves T = I
      // and the samples fold straight into RF)
      double* Rpt = RF;
      std::vector<FoldTask> ft;
      std::vector<FoldTerm> fterms;
      if (H > 0) {
        double* Y = (double*)sc.alloc(NN * 8);
        Rpt = (double*)sc.alloc(NN * 8);
        std::vector<CopyTask> tr;
        std::vector<TrsmTask> tt;
        for (int g = 0; g < nb; ++g) {
          if (!has_fill[g]) continue;
          tr.push_back(CopyTask{RF + off[g], Y + off[g], n[g], n[g], n[g], n[g]});
          tt.push_back(TrsmTask{Tcur->as<double>() + t_off[g], Y + off[g], n[g], n[g], n[g], n[g], nullptr});
        }
        run_copy(Prec::F64, Prec::F64, true, tr, maxn, maxn, sc);
        run_trsm(Prec::F64, false, false, false, tt, maxn, sc);
        for (int g = 0; g < nb; ++g) {
          FoldTask f{dc + co[g], ds + sof[g], Rpt + off[g], n[g], (int)(sof[g + 1] - sof[g]), (int)fterms.size(), 0, 0};
          if (has_fill[g]) {
            fterms.push_back(FoldTerm{Y + off[g], n[g], n[g], 0});
            f.nt = 1;
          }
          ft.push_back(f);
        }
      } else {
        for (int g = 0; g < nb; ++g) {
          const int m_s = (int)(sof[g + 1] - sof[g]);
          if (m_s > 0) ft.push_back(FoldTask{dc + co[g], ds + sof[g], RF + off[g], n[g], m_s, 0, 0, 1});
        }
      }
      run_fold(ft, fterms, pts, h.kp, sc);
      std::vector<PqrTask> qt;
      for (int g = 0; g < nb; ++g)
        qt.push_back(PqrTask{Rpt + off[g], n[g], n[g], n[g], piv + (size_t)g * NMAX, R + off[g], rank + g, tol_basis,
                             h.opt.max_rank, cinfo});
      run_pqr(qt, sc);
    } else {
    double* G = (double*)sc.alloc(NN * 8);
    {
      std::vector<CopyTask> ct;
      for (int g = 0; g < nb; ++g) ct.push_back(CopyTask{(char*)GF + so[g] * ws, G + off[g], n[g], n[g], n[g], n[g]});
      run_copy(W, Prec::F64, false, ct, maxn, maxn, sc);
      if (H > 0) {
        // point form: T^-1 G T^-T (T = blockdiag(W_a, W_b), upper triangular)
        double* G2 = (double*)sc.alloc(NN * 8);
        std::vector<TrsmTask> t1, t2;
        std::vector<CopyTask> tr;
        for (int g = 0; g < nb; ++g) {
          t1.push_back(TrsmTask{Tcur->as<double>() + t_off[g], G + off[g], n[g], n[g], n[g], n[g], nullptr});
          tr.push_back(CopyTask{G + off[g], G2 + off[g], n[g], n[g], n[g], n[g]});
          t2.push_back(TrsmTask{Tcur->as<double>() + t_off[g], G2 + off[g], n[g], n[g], n[g], n[g], nullptr});
        }
        run_trsm(Prec::F64, false, false, false, t1, maxn, sc);
        run_copy(Prec::F64, Prec::F64, true, tr, maxn, maxn, sc);
        run_trsm(Prec::F64, false, false, false, t2, maxn, sc);
        G = G2;
      }
      // far-field block row Gram K(cand, samples) K(cand, samples)^T
      if (W == Prec::F64) {
        std::vector<KgramTask> kt;
        for (int g = 0; g < nb; ++g) {
          int m = (int)(sof[g + 1] - sof[g]);
          if (m == 0) continue;
          kt.push_back(KgramTask{dc + co[g], ds + sof[g], G + off[g], n[g], m, n[g], 1});
        }
        run_kgram(W, kt, maxn, pts, h.kp, sc);
      } else {
        // mixed precision: each box's block row B = K(cand, samples) is
        // evaluated once (FP32, chunks of boxes within the pair budget), its
        // Gram B B^T formed by the batched tensor-core GEMM and added to G
        float* Gfar = (float*)sc.alloc(NN * 4);
        std::vector<int> boxes_far;
        for (int g = 0; g < nb; ++g)
          if (sof[g + 1] > sof[g]) boxes_far.push_back(g);
        size_t b0 = 0;
        while (b0 < boxes_far.size()) {
          size_t b1 = b0, tot = 0;
          std::vector<size_t> bo;
          while (b1 < boxes_far.size()) {
            const int g = boxes_far[b1];
            const size_t need = ((size_t)n[g] * (sof[g + 1] - sof[g]) * 4 + 255) & ~size_t(255);
            if (b1 > b0 && tot + need > pair_budget) break;
            bo.push_back(tot);
            tot += need;
            ++b1;
          }
          char* Bb = (char*)pair_buf(tot);
          std::vector<AsmTask> at;
          GemmBatch gb;
          int maxc = 0;
          for (size_t q = b0; q < b1; ++q) {
            const int g = boxes_far[q];
            const int m = (int)(sof[g + 1] - sof[g]);
            float* B = (float*)(Bb + bo[q - b0]);
            at.push_back(AsmTask{B, dc + co[g], ds + sof[g], 0, 0, n[g], m, n[g]});
            maxc = std::max(maxc, m);
            gb.add1(Gfar + off[g], n[g], n[g], n[g], B, n[g], B, n[g], m, 1.0, 0.0, nullptr, 0, 2);
          }
          validate(at, 4);
          {
            double by = 0.0;
            for (const AsmTask& a : at) by += 4.0 * a.nr * a.nc;
            prof_note(0.0, by);
          }
          launch_assemble_far_f32(sc.up(at), (int)at.size(), maxc, pts, h.kp, sc.s);
          prof_tag("basis_gram");
          gb.run(W, false, false, sc);
          prof_tag("basis");
          b0 = b1;
        }
        std::vector<CopyTask> ca;
        for (int g : boxes_far) ca.push_back(CopyTask{Gfar + off[g], G + off[g], n[g], n[g], n[g], n[g]});
        if (!ca.empty()) {
          prof_note(0.0, 12.0 * (double)NN);
          launch_add_copy(sc.up(ca), (int)ca.size(), maxn, maxn, sc.s);
        }
      }
    }
    {
      // Rank tolerance of the Gram route.  In mixed precision the Gram
      // matrix is accumulated in FP32, which resolves the block row only to
      // about 2^-10 of its norm; pivoting below that would select skeletons
      // from rounding noise (and grow the interpolation coefficients level
      // by level), so the threshold is floored there (tol_basis above).  The
      // FP64 refinement against the H^2 operator recovers the accuracy.
      std::vector<CholTask> ct;
      double* Lch = (double*)sc.alloc(NN * 8);
      for (int g = 0; g < nb; ++g)
        ct.push_back(CholTask{G + off[g], n[g], n[g], piv + (size_t)g * NMAX, R + off[g], rank + g, tol_basis,
                              h.opt.max_rank, cinfo, Lch + off[g]});
      run_pchol(ct, sc);
    }
    }
    H2_CUDA(cudaMemcpyAsync(cinfo + 1, finfo, 4, cudaMemcpyDeviceToDevice, s));
    std::vector<int> hr(nb), hpiv((size_t)nb * NMAX);
    int hci[2] = {0, 0};
    int hprev = 0;   // a redundant-block pivot of an earlier height failed (deferred flag)
    H2_CUDA(cudaMemcpyAsync(hr.data(), rank, nb * 4, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(hpiv.data(), piv, hpiv.size() * 4, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(hci, cinfo, 8, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(&hprev, dflags, 4, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    {
      // rank-dependent work of the pivoted Cholesky / pivoted QR just run
      double f = 0.0;
      for (int g = 0; g < nb; ++g) {
        const double nn = n[g], rr = std::min(hr[g], n[g]);
        f += qr_route ? 4.0 * nn * nn * rr - 4.0 * nn * rr * rr + 4.0 * rr * rr * rr / 3.0
                      : nn * rr * rr - 2.0 * rr * rr * rr / 3.0;
      }
      prof_add(qr_route ? "pqr_f64" : "pchol_f64", f);
    }
    // the first failure is the one reported: a bad pivot below this height
    // fills everything above it with non-finite values
    if (hprev)
      throw StatusError(spd ? H2_ERR_NOT_SPD : H2_ERR_SINGULAR,
                        spd ? "non-positive pivot in a redundant-block Cholesky" : "zero pivot in a redundant-block LU");
    if (hci[0]) throw StatusError(H2_ERR_NONFINITE, "non-finite value in a basis block row");
    if (hci[1]) throw StatusError(H2_ERR_SINGULAR, "zero or non-finite pivot in a diagonal-block LU (fill-ins)");
    ht.r.resize(nb);
    ht.sk.resize(nb);
    std::vector<int> keep_all(nb, 0);
    for (int g = 0; g < nb; ++g) {
      if (hr[g] == 0) {   // empty block row: nothing is redundant
        keep_all[g] = 1;
        hr[g] = n[g];
        for (int q = 0; q < n[g]; ++q) hpiv[(size_t)g * NMAX + q] = q;
      }
      ht.r[g] = hr[g];
      ht.sk[g].resize(hr[g]);
      for (int q = 0; q < hr[g]; ++q) ht.sk[g][q] = ht.cand[g][hpiv[(size_t)g * NMAX + q]];
    }
    if (std::count(keep_all.begin(), keep_all.end(), 1))
      H2_CUDA(cudaMemcpyAsync(piv, pinned_stage(hpiv.data(), hpiv.size() * 4, s), hpiv.size() * 4,
                              cudaMemcpyHostToDevice, s));
    std::vector<int>& r = ht.r;
    std::vector<int> m(nb);
    for (int g = 0; g < nb; ++g) m[g] = n[g] - r[g];
    // interpolation matrix P (n x r, FP64): T = R11^-1 R12
    double* P = (double*)sc.alloc(NN * 8, true);
    {
      std::vector<TrsmTask> tt;
      std::vector<InterpTask> it;
      std::vector<CopyTask> eye;
      int maxrhs = 0;
      for (int g = 0; g < nb; ++g) {
        if (keep_all[g]) continue;
        if (r[g] < n[g]) {
          tt.push_back(TrsmTask{R + off[g], R + off[g] + (size_t)r[g] * n[g], r[g], n[g] - r[g], n[g], n[g], nullptr});
          maxrhs = std::max(maxrhs, n[g] - r[g]);
        }
        it.push_back(InterpTask{piv + (size_t)g * NMAX, R + off[g] + (size_t)r[g] * n[g], P + off[g], n[g], r[g], n[g]});
      }
      run_trsm(Prec::F64, false, false, false, tt, maxrhs, sc);
      run_interp(Prec::F64, it, sc);
      for (int g = 0; g < nb; ++g)
        if (keep_all[g]) launch_fill_eye(Prec::F64, P + off[g], n[g], n[g], s);
    }
    // basis matrix in level coordinates: M = T P (n x r)
    double* Mm = P;
    if (H > 0) {
      Mm = (double*)sc.alloc(NN * 8);
      GemmBatch gb;
      for (int g = 0; g < nb; ++g)
        gb.add1(Mm + off[g], n[g], n[g], r[g], Tcur->as<double>() + t_off[g], n[g], P + off[g], n[g], n[g]);
      gb.run(Prec::F64, false, false, sc);
    }
    // orthogonalise: Q = [U^R U^S], W (r x r).  In mixed precision the
    // orthogonalisation runs in FP32 (Q and W only precondition there).
    ht.q_off = off;
    ensure(ht.Q, NN * 8);
    ht.w_off.assign(nb + 1, 0);
    for (int g = 0; g < nb; ++g) ht.w_off[g + 1] = ht.w_off[g] + (size_t)r[g] * r[g];
    ensure(ht.W, std::max<size_t>(1, ht.w_off[nb]) * 8);
    if (W == Prec::F64) {
      double* V = (double*)sc.alloc(NN * 8);
      std::vector<HqrTask> qt;
      for (int g = 0; g < nb; ++g)
        qt.push_back(HqrTask{Mm + off[g], V + off[g], ht.Q->as<double>() + off[g], ht.W->as<double>() + ht.w_off[g], n[g], r[g]});
      run_hqr(Prec::F64, qt, sc);
    } else {
      float* Mf = (float*)sc.alloc(NN * 4);
      float* V = (float*)sc.alloc(NN * 4);
      float* Qf = (float*)sc.alloc(NN * 4);
      float* Wf = (float*)sc.alloc(std::max<size_t>(1, ht.w_off[nb]) * 4);
      std::vector<CopyTask> c1, c2, c3;
      std::vector<HqrTask> qt;
      for (int g = 0; g < nb; ++g) {
        c1.push_back(CopyTask{Mm + off[g], Mf + off[g], n[g], r[g], n[g], n[g]});
        qt.push_back(HqrTask{Mf + off[g], V + off[g], Qf + off[g], Wf + ht.w_off[g], n[g], r[g]});
        c2.push_back(CopyTask{Qf + off[g], ht.Q->as<double>() + off[g], n[g], n[g], n[g], n[g]});
        c3.push_back(CopyTask{Wf + ht.w_off[g], ht.W->as<double>() + ht.w_off[g], r[g], r[g], r[g], r[g]});
      }
      run_copy(Prec::F64, Prec::F32, false, c1, maxn, maxn, sc);
      run_hqr(Prec::F32, qt, sc);
      run_copy(Prec::F32, Prec::F64, false, c2, maxn, maxn, sc);
      run_copy(Prec::F32, Prec::F64, false, c3, 256, 256, sc);
    }
    const void* Qw = ht.Q->p;
    const void* Ww = ht.W->p;
    if (W == Prec::F32) {
      ensure(ht.Qw, NN * 4);
      auto Wf = std::make_shared<DBuf>(std::max<size_t>(1, ht.w_off[nb]) * 4);
      std::vector<CopyTask> ct, cw;
      for (int g = 0; g < nb; ++g) {
        ct.push_back(CopyTask{ht.Q->as<double>() + off[g], ht.Qw->as<float>() + off[g], n[g], n[g], n[g], n[g]});
        cw.push_back(CopyTask{ht.W->as<double>() + ht.w_off[g], Wf->as<float>() + ht.w_off[g], r[g], r[g], r[g], r[g]});
      }
      run_copy(Prec::F64, Prec::F32, false, ct, maxn, maxn, sc);
      run_copy(Prec::F64, Prec::F32, false, cw, 256, 256, sc);
      sc.bufs.push_back(Wf);
      Qw = ht.Qw->p;
      Ww = Wf->p;
    }
    auto Qp = [&](int g) -> const char* { return (const char*)Qw + off[g] * ws; };
    auto USp = [&](int g) -> const char* { return (const char*)Qw + (off[g] + (size_t)m[g] * n[g]) * ws; };
    auto Wp = [&](int g) -> const char* { return (const char*)Ww + ht.w_off[g] * ws; };
    // ---------------- parent-level storage (merge target) ---------------
    Height* up = (H + 1 < h.Hmax) ? &h.hs[H + 1] : nullptr;
    std::vector<std::vector<PairRef>> Anext;
    DBufP Anext_buf;
    if (up) {
      up->n.assign(up->nb, 0);
      up->cand.assign(up->nb, {});
      for (int g = 0; g < nb; ++g) {
        int pg = ht.parent[g];
        if (pg < 0) continue;
        up->n[pg] += r[g];
        up->cand[pg].insert(up->cand[pg].end(), ht.sk[g].begin(), ht.sk[g].end());
      }
      // only pairs P <= Q are stored; (Q, P) references the transpose
      size_t tot = 0;
      std::vector<std::vector<size_t>> po(up->nb);
      for (int pg = 0; pg < up->nb; ++pg)
        for (int qg : up->near[pg]) {
          po[pg].push_back(tot);
          if (pg <= qg) tot += (size_t)up->n[pg] * up->n[qg];
        }
      h.exact_bytes += (double)tot * ws;
      bool hit = false;
      if (Apre) {
        hit = true;
        for (int g = 0; g < nb && hit; ++g) hit = r[g] <= rcap[g];
        if (hit) ++h.pred_hits;
        else ++h.pred_misses;
      }
      std::vector<int> lds(up->nb);
      if (hit) {
        // the predicted capacities cover every rank: keep the storage that
        // was allocated before the basis pass (leading dimension = capacity)
        Anext_buf = Apre;
        po = pre_off;
        lds = pre_ld;
      } else {
        Apre.reset();
        if (h.opt.hbm_budget_bytes > 0 && (int64_t)(tot * ws) > h.opt.hbm_budget_bytes)
          throw StatusError(H2_ERR_BUDGET, "level near blocks need " + std::to_string(tot * ws) + " bytes");
        Anext_buf = cached_or_new(std::max<size_t>(1, tot) * ws, s);
        lds = up->n;
      }
      Anext.assign(up->nb, {});
      for (int pg = 0; pg < up->nb; ++pg)
        for (size_t q = 0; q < up->near[pg].size(); ++q) {
          int qg = up->near[pg][q];
          if (pg <= qg) {
            Anext[pg].push_back(PairRef{(char*)Anext_buf->p + po[pg][q] * ws, lds[pg], 0});
          } else {
            const auto& nl = up->near[qg];   // sorted
            size_t qq = std::lower_bound(nl.begin(), nl.end(), pg) - nl.begin();
            Anext[pg].push_back(PairRef{(char*)Anext_buf->p + po[qg][qq] * ws, lds[qg], 1});
          }
        }
    }
    // root setup for problems whose top ULV height is H
    for (size_t p = 0; p < h.probs.size(); ++p) {
      Problem& pb = h.probs[p];
      if (pb.H != H + 1) continue;
      std::vector<int> sizes(pb.t.boxes[pb.t.ltop].size(), 0);
      for (int g = 0; g < nb; ++g)
        if (ht.ref[g].prob == (int)p) sizes[ht.root_slot[g]] += r[g];
      setup_root(pb, sizes);
    }
    // destination of the S^SS block of child pair (g, j): the parent block
    // (or root matrix) at the children's quadrant
    auto dest = [&](int g, int j, int& ld) -> char* {
      int pg = ht.parent[g];
      int rowoff = (ht.ref[g].local % 2) ? r[g - 1] : 0;
      int coloff = (ht.ref[j].local % 2) ? r[j - 1] : 0;
      if (pg >= 0) {
        int pj = ht.parent[j];
        if (pg > pj) return nullptr;
        const auto& nl = up->near[pg];
        int q = (int)(std::lower_bound(nl.begin(), nl.end(), pj) - nl.begin());   // near lists are sorted
        ld = Anext[pg][q].ld;
        return (char*)Anext[pg][q].ptr + ((size_t)rowoff + (size_t)coloff * ld) * ws;
      }
      Root& rt = h.probs[ht.ref[g].prob].root;
      ld = rt.n;
      size_t ro = (size_t)rt.off[ht.root_slot[g]] + rowoff;
      size_t co = (size_t)rt.off[ht.root_slot[j]] + coloff;
      return (char*)rt.A->p + (ro + co * rt.n) * ws;
    };
    // ---------------- 3. projection (eq. rs, eq. ss) -------------------
    prof_tag("proj");
    void* Sw = sc.alloc(NN * ws);
    {
      GemmBatch g1, g2;
      for (int g = 0; g < nb; ++g) {
        int dq = diag_q(g);
        g1.add1((char*)Tmp + so[g] * ws, n[g], n[g], n[g], Ablk[g][dq].ptr, Ablk[g][dq].ld, Qp(g), n[g], n[g]);
        g2.add1((char*)Sw + off[g] * ws, n[g], n[g], n[g], Qp(g), n[g], (char*)Tmp + so[g] * ws, n[g], n[g]);
      }
      g1.run(W, false, false, sc);
      g2.run(W, true, false, sc);
    }
    {
      // near pairs: S^SS_IJ = U^S_I^T A_IJ U^S_J into the parent block, all
      // pairs of a chunk in two launches (V = op(A_IJ) U^S_J, then U^S_I^T V)
      std::vector<PairSlot> prs = near_pairs(
          ht.near,
          [&](int g, int j) {
            int ld;
            return j != g && dest(g, j, ld) != nullptr;   // skip mirrors of stored parent blocks
          },
          [&](int g, int j) { return (size_t)n[g] * r[j] * ws; });
      for (size_t p0 = 0; p0 < prs.size();) {
        const size_t p1 = chunk_pairs(prs, p0, pair_budget);
        char* Vb = (char*)pair_buf(prs[p1 - 1].off + prs[p1 - 1].bytes);
        GemmBatch g1, g2;
        for (size_t q = p0; q < p1; ++q) {
          const PairSlot& pr = prs[q];
          const int g = pr.g, k = pr.k, j = pr.j;
          int ld;
          char* D = dest(g, j, ld);
          char* V = Vb + pr.off;                       // n_g x r_j
          g1.add1(V, n[g], n[g], r[j], Ablk[g][k].ptr, Ablk[g][k].ld, USp(j), n[j], n[j], 1.0, 0.0, nullptr, 0,
                  Ablk[g][k].tr ? 1 : 0);
          g2.add1(D, ld, r[g], r[j], USp(g), n[g], V, n[g], n[g]);
        }
        g1.run(W, false, false, sc);
        g2.run(W, true, false, sc);
        p0 = p1;
      }
      // far pairs at this level: W_I K(sk_I, sk_J) W_J^T, chunked the same way
      std::vector<int> sk_all;
      std::vector<size_t> sko(nb + 1, 0);
      for (int g = 0; g < nb; ++g) {
        sk_all.insert(sk_all.end(), ht.sk[g].begin(), ht.sk[g].end());
        sko[g + 1] = sk_all.size();
      }
      int* dsk = sc.up(sk_all);
      std::vector<PairSlot> fps = near_pairs(
          ht.far,
          [&](int g, int j) {
            int ld;
            return dest(g, j, ld) != nullptr;
          },
          [&](int g, int j) { return 2 * (size_t)r[g] * r[j] * ws; });
      for (size_t p0 = 0; p0 < fps.size();) {
        const size_t p1 = chunk_pairs(fps, p0, pair_budget);
        char* Fb = (char*)pair_buf(fps[p1 - 1].off + fps[p1 - 1].bytes);
        std::vector<AsmTask> at;
        GemmBatch g1, g2;
        int maxc = 0;
        for (size_t q = p0; q < p1; ++q) {
          const PairSlot& pr = fps[q];
          const int g = pr.g, j = pr.j;
          char* Kb = Fb + pr.off;                                 // r_g x r_j
          char* V = Kb + (size_t)r[g] * r[j] * ws;                // r_g x r_j
          at.push_back(AsmTask{Kb, dsk + sko[g], dsk + sko[j], 0, 0, r[g], r[j], r[g]});
          maxc = std::max(maxc, r[j]);
          g1.add1(V, r[g], r[g], r[j], Wp(g), r[g], Kb, r[g], r[g]);
          int ld;
          char* D = dest(g, j, ld);
          g2.add1(D, ld, r[g], r[j], V, r[g], Wp(j), r[j], r[j]);
        }
        if (W == Prec::F32) {   // far pairs: box-relative FP32 coordinates
          validate(at, 4);
          double by = 0.0;
          for (const AsmTask& a : at) by += 4.0 * a.nr * a.nc;
          prof_note(0.0, by);
          launch_assemble_far_f32(sc.up(at), (int)at.size(), maxc, pts, h.kp, sc.s);
        } else {
          run_assemble(W, at, 256, maxc, pts, h.kp, sc);
        }
        g1.run(W, false, false, sc);
        g2.run(W, false, true, sc);
        p0 = p1;
      }
    }
    // ---------------- 4. partial LU of S^RR (eq. lu) -------------------
    prof_tag("elim");
    ensure(ht.S, NN * 8);
    {
      std::vector<CopyTask> ct;
      for (int g = 0; g < nb; ++g)
        ct.push_back(CopyTask{(char*)Sw + off[g] * ws, ht.S->as<double>() + off[g], n[g], n[g], n[g], n[g]});
      run_copy(W, Prec::F64, false, ct, maxn, maxn, sc);
    }
    ht.pv_off.assign(nb + 1, 0);
    ht.lt_off.assign(nb + 1, 0);
    for (int g = 0; g < nb; ++g) {
      ht.pv_off[g + 1] = ht.pv_off[g] + m[g];
      ht.lt_off[g + 1] = ht.lt_off[g] + (size_t)m[g] * r[g];
    }
    ensure(ht.pivRR, std::max<size_t>(1, ht.pv_off[nb]) * 4);
    ensure(ht.Lt, std::max<size_t>(1, ht.lt_off[nb]) * 8);
    int* info = dflags;   // checked once the factorization has been issued
    {
      double* S = ht.S->as<double>();
      std::vector<LuTask> lu;
      std::vector<TrsmTask> trs, tsr;
      std::vector<CopyTask> tr;
      int maxr = 0, maxm = 0;
      for (int g = 0; g < nb; ++g) {
        if (m[g] == 0) continue;
        double* Sg = S + off[g];
        lu.push_back(LuTask{Sg, m[g], m[g], n[g], ht.pivRR->as<int>() + ht.pv_off[g], info, spd ? 1 : 0});
        trs.push_back(TrsmTask{Sg, Sg + (size_t)m[g] * n[g], m[g], r[g], n[g], n[g], ht.pivRR->as<int>() + ht.pv_off[g]});
        // (L^SR)^T = U^-T (S^SR)^T: transpose S^SR (r x m) into Lt (m x r)
        tr.push_back(CopyTask{Sg + m[g], ht.Lt->as<double>() + ht.lt_off[g], m[g], r[g], n[g], m[g]});
        tsr.push_back(TrsmTask{Sg, ht.Lt->as<double>() + ht.lt_off[g], m[g], r[g], n[g], m[g], nullptr});
        maxr = std::max(maxr, r[g]);
        maxm = std::max(maxm, m[g]);
      }
      if (!lu.empty()) {
        run_getrf(Prec::F64, lu, sc);
        run_trsm(Prec::F64, true, true, false, trs, maxr, sc);
        run_copy(Prec::F64, Prec::F64, true, tr, maxm, maxr, sc);
        run_trsm(Prec::F64, true, false, true, tsr, maxr, sc);
        // Schur: S^SS -= (L^SR) U^RS = Lt^T U^RS
        GemmBatch gb;
        for (int g = 0; g < nb; ++g) {
          if (m[g] == 0) continue;
          double* Sg = S + off[g];
          double* SS = Sg + m[g] + (size_t)m[g] * n[g];
          gb.add1(SS, n[g], r[g], r[g], ht.Lt->as<double>() + ht.lt_off[g], m[g], Sg + (size_t)m[g] * n[g], n[g], m[g],
                  -1.0, 1.0);
        }
        gb.run(Prec::F64, true, false, sc);
      }
      // explicit L^-1 P^T and U^-1 of every S^RR LU: the solve sweeps apply
      // them as products instead of sequential triangular solves
      ht.li_off.assign(nb + 1, 0);
      for (int g = 0; g < nb; ++g) ht.li_off[g + 1] = ht.li_off[g] + (size_t)m[g] * m[g];
      ensure(ht.Linv, std::max<size_t>(1, ht.li_off[nb]) * 8);
      ensure(ht.Uinv, std::max<size_t>(1, ht.li_off[nb]) * 8);
      {
        double* I256 = (double*)sc.alloc((size_t)NMAX * NMAX * 8);
        launch_fill_eye(Prec::F64, I256, NMAX, NMAX, s);
        std::vector<CopyTask> ci;
        for (int g = 0; g < nb; ++g) {
          if (m[g] == 0) continue;
          ci.push_back(CopyTask{I256, ht.Linv->as<double>() + ht.li_off[g], m[g], m[g], NMAX, m[g]});
          ci.push_back(CopyTask{I256, ht.Uinv->as<double>() + ht.li_off[g], m[g], m[g], NMAX, m[g]});
        }
        run_copy(Prec::F64, Prec::F64, false, ci, 256, 256, sc);
        if (W == Prec::F64) {
          std::vector<TrsmTask> tl, tu;
          for (int g = 0; g < nb; ++g) {
            if (m[g] == 0) continue;
            tl.push_back(TrsmTask{S + off[g], ht.Linv->as<double>() + ht.li_off[g], m[g], m[g], n[g], m[g],
                                  ht.pivRR->as<int>() + ht.pv_off[g]});
            tu.push_back(TrsmTask{S + off[g], ht.Uinv->as<double>() + ht.li_off[g], m[g], m[g], n[g], m[g], nullptr});
          }
          run_trsm(Prec::F64, true, true, false, tl, maxm, sc);
          run_trsm(Prec::F64, false, false, false, tu, maxm, sc);
        } else {
          // mixed precision: the inverses only precondition, so they are
          // formed in FP32 from FP32 copies of the FP64 LU factors
          const size_t LI = ht.li_off[nb];
          float* Sf = (float*)sc.alloc(NN * 4);
          float* Lf = (float*)sc.alloc(std::max<size_t>(1, LI) * 4);
          float* Uf = (float*)sc.alloc(std::max<size_t>(1, LI) * 4);
          std::vector<CopyTask> c1, c2;
          std::vector<TrsmTask> tl, tu;
          for (int g = 0; g < nb; ++g) {
            if (m[g] == 0) continue;
            c1.push_back(CopyTask{S + off[g], Sf + off[g], m[g], m[g], n[g], n[g]});
            c1.push_back(CopyTask{ht.Linv->as<double>() + ht.li_off[g], Lf + ht.li_off[g], m[g], m[g], m[g], m[g]});
            c1.push_back(CopyTask{ht.Uinv->as<double>() + ht.li_off[g], Uf + ht.li_off[g], m[g], m[g], m[g], m[g]});
            tl.push_back(TrsmTask{Sf + off[g], Lf + ht.li_off[g], m[g], m[g], n[g], m[g], ht.pivRR->as<int>() + ht.pv_off[g]});
            tu.push_back(TrsmTask{Sf + off[g], Uf + ht.li_off[g], m[g], m[g], n[g], m[g], nullptr});
            c2.push_back(CopyTask{Lf + ht.li_off[g], ht.Linv->as<double>() + ht.li_off[g], m[g], m[g], m[g], m[g]});
            c2.push_back(CopyTask{Uf + ht.li_off[g], ht.Uinv->as<double>() + ht.li_off[g], m[g], m[g], m[g], m[g]});
          }
          run_copy(Prec::F64, Prec::F32, false, c1, 256, 256, sc);
          run_trsm(Prec::F32, true, true, false, tl, maxm, sc);
          run_trsm(Prec::F32, false, false, false, tu, maxm, sc);
          run_copy(Prec::F32, Prec::F64, false, c2, 256, 256, sc);
        }
      }
      // S^SS_II -> parent quadrant
      std::vector<CopyTask> cs;
      for (int g = 0; g < nb; ++g) {
        int ld;
        char* D = dest(g, g, ld);
        cs.push_back(CopyTask{S + off[g] + m[g] + (size_t)m[g] * n[g], D, r[g], r[g], n[g], ld});
      }
      run_copy(Prec::F64, W, false, cs, 256, 256, sc);
    }
    // ---------------- 5. next height: T = blockdiag(W_a, W_b) ---------
    prof_tag("merge");
    if (up) {
      std::vector<size_t> to(up->nb + 1, 0);
      for (int pg = 0; pg < up->nb; ++pg) to[pg + 1] = to[pg] + (size_t)up->n[pg] * up->n[pg];
      auto Tn = cached_or_new(std::max<size_t>(1, to[up->nb]) * 8, s);
      H2_CUDA(cudaMemsetAsync(Tn->p, 0, Tn->bytes, s));
      std::vector<CopyTask> ct;
      for (int g = 0; g < nb; ++g) {
        int pg = ht.parent[g];
        if (pg < 0) continue;
        int o = (ht.ref[g].local % 2) ? r[g - 1] : 0;
        ct.push_back(CopyTask{ht.W->as<double>() + ht.w_off[g], Tn->as<double>() + to[pg] + o + (size_t)o * up->n[pg],
                              r[g], r[g], r[g], up->n[pg]});
      }
      run_copy(Prec::F64, Prec::F64, false, ct, 256, 256, sc);
      scratch_cache().give(std::move(Tcur), s);
      Tcur = Tn;
      t_off = to;
      Ablk = std::move(Anext);
      for (DBufP& b : Aown) scratch_cache().give(std::move(b), s);
      Aown.clear();
      Aown.push_back(Anext_buf);
    }
    // level-vector offsets (solve)
    ht.v_off.assign(nb + 1, 0);
    for (int g = 0; g < nb; ++g) ht.v_off[g + 1] = ht.v_off[g] + n[g];
    ht.v_len = ht.v_off[nb];
    ht.y_off.assign(nb + 1, 0);
    for (int g = 0; g < nb; ++g) ht.y_off[g + 1] = ht.y_off[g] + m[g];
    ht.y_len = ht.y_off[nb];
    {
      cudaEvent_t e1;
      H2_CUDA(cudaEventCreate(&e1));
      hev.push_back(e1);
      H2_CUDA(cudaEventRecord(e1, s));
    }
  }
  // roots
  prof_tag("root");
  for (size_t p = 0; p < P; ++p) {
    Root& rt = h.probs[p].root;
    if (rt.n == 0) continue;
    if (W == Prec::F64) {
      Scratch sc(s);
      std::vector<CopyTask> ct{CopyTask{rt.A->p, rt.LU->p, rt.n, rt.n, rt.n, rt.n}};
      run_copy(W, Prec::F64, false, ct, rt.n, rt.n, sc);
      root_factor(h, rt, spd, Prec::F64, rt.LU->p, dflags + 1, droot + 2 * p);
    } else {
      root_factor(h, rt, spd, W, rt.A->p, dflags + 1, droot + 2 * p);
    }
  }
  prof_tag(nullptr);
  // the deferred results (one synchronisation for the whole factorization)
  int hflags[4] = {0, 0, 0, 0};
  std::vector<double> hroot(2 * std::max<size_t>(1, P));
  H2_CUDA(cudaMemcpyAsync(hflags, dflags, 16, cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaMemcpyAsync(hroot.data(), droot, hroot.size() * 8, cudaMemcpyDeviceToHost, s));
  H2_CUDA(cudaStreamSynchronize(s));
  for (size_t p = 0; p < P; ++p) {
    Root& rt = h.probs[p].root;
    rt.A.reset();
    rt.logdet = rt.n ? hroot[2 * p] : 0.0;
    rt.sign = rt.n ? hroot[2 * p + 1] : 1.0;
  }
  for (size_t k = 0; k + 1 < hev.size(); k += 2) {
    float ms = 0.f;
    H2_CUDA(cudaEventElapsedTime(&ms, hev[k], hev[k + 1]));
    h.level_ms.push_back(ms);
  }
  if (W == Prec::F32 && tc_error_flag_read_and_clear(s))
    throw StatusError(H2_ERR_TIMEOUT, "a tensor-core completion wait gave up");
  if (hflags[0])
    throw StatusError(spd ? H2_ERR_NOT_SPD : H2_ERR_SINGULAR,
                      spd ? "non-positive pivot in a redundant-block Cholesky" : "zero pivot in a redundant-block LU");
  if (hflags[1])
    throw StatusError(spd ? H2_ERR_NOT_SPD : H2_ERR_SINGULAR,
                      spd ? "non-positive pivot in the top-level Cholesky" : "zero pivot in the top-level LU");
}

// -------------------------------------------------------------- solve ----
// Plan of x = ULV^-1 b in tree order (N x nrhs, ld = Ntot), FP64 sweeps:
// forward (L z = U^T b), root solve, backward (U y = z, x = V^T y).
static PlanP build_ulv_plan(Handle& h, const double* b, double* x, int nrhs) {
  auto P = std::make_shared<Plan>();
  Plan& pl = *P;
  const int64_t ld = h.Ntot;
  std::vector<double*> c(h.Hmax), xo(h.Hmax), yb(h.Hmax);
  for (int H = 0; H < h.Hmax; ++H) {
    c[H] = pl.work((size_t)h.hs[H].v_len * nrhs);
    xo[H] = pl.work((size_t)h.hs[H].v_len * nrhs);
    yb[H] = pl.work((size_t)std::max<int64_t>(1, h.hs[H].y_len) * nrhs);
  }
  std::vector<double*> rootb(h.probs.size(), nullptr), rootx(h.probs.size(), nullptr);
  for (size_t p = 0; p < h.probs.size(); ++p)
    if (h.probs[p].root.n) {
      rootb[p] = pl.work((size_t)h.probs[p].root.n * nrhs);
      rootx[p] = pl.work((size_t)h.probs[p].root.n * nrhs);
    }
  // problems without ULV heights: root rhs = the whole problem
  {
    std::vector<CopyTask> ct;
    for (size_t p = 0; p < h.probs.size(); ++p)
      if (h.probs[p].H == 0)
        ct.push_back(CopyTask{b + h.probs[p].off, rootb[p], h.probs[p].root.n, nrhs, (int)ld, h.probs[p].root.n});
    pl.copy(Prec::F64, Prec::F64, false, ct, 8192, nrhs);
  }
  // forward sweep
  pl.tag("ulv_fwd");
  for (int H = 0; H < h.Hmax; ++H) {
    Height& ht = h.hs[H];
    const int nb = ht.nb;
    const int64_t lv = ht.v_len;
    GemmBatch g1;
    for (int g = 0; g < nb; ++g) {
      const double* src;
      int64_t lds;
      if (H == 0) {
        const BoxRef& bb = ht.ref[g];
        const Problem& pb = h.probs[bb.prob];
        src = b + pb.off + pb.t.boxes[bb.level][bb.local].s;
        lds = ld;
      } else {
        src = xo[H - 1] + ht.v_off[g];   // gathered into xo[H-1] below, by parent offsets
        lds = ht.v_len;
      }
      g1.add1(c[H] + ht.v_off[g], (int)lv, ht.n[g], nrhs, ht.Q->as<double>() + ht.q_off[g], ht.n[g], src, (int)lds,
              ht.n[g]);
    }
    pl.gemm(Prec::F64, g1, true, false);
    // y_R = (L^-1 P^T) c_R, then c_S -= L^SR y_R
    const int64_t ly = std::max<int64_t>(1, ht.y_len);
    GemmBatch gl, g2;
    for (int g = 0; g < nb; ++g) {
      int m = ht.n[g] - ht.r[g];
      if (m == 0) continue;
      gl.add1(yb[H] + ht.y_off[g], (int)ly, m, nrhs, ht.Linv->as<double>() + ht.li_off[g], m, c[H] + ht.v_off[g],
              (int)lv, m);
      g2.add1(c[H] + ht.v_off[g] + m, (int)lv, ht.r[g], nrhs, ht.Lt->as<double>() + ht.lt_off[g], m,
              yb[H] + ht.y_off[g], (int)ly, m, -1.0, 1.0);
    }
    pl.gemm(Prec::F64, gl, false, false);
    pl.gemm(Prec::F64, g2, true, false);
    // gather skeleton parts into the next height's input (stored in xo[H])
    std::vector<CopyTask> ct;
    for (int g = 0; g < nb; ++g) {
      int m = ht.n[g] - ht.r[g];
      int o = (ht.ref[g].local % 2) ? ht.r[g - 1] : 0;
      if (ht.parent[g] >= 0) {
        const Height& up = h.hs[H + 1];
        ct.push_back(CopyTask{c[H] + ht.v_off[g] + m, xo[H] + up.v_off[ht.parent[g]] + o, ht.r[g], nrhs, (int)lv,
                              (int)up.v_len});
      } else {
        Root& rt = h.probs[ht.ref[g].prob].root;
        ct.push_back(CopyTask{c[H] + ht.v_off[g] + m, rootb[ht.ref[g].prob] + rt.off[ht.root_slot[g]] + o, ht.r[g],
                              nrhs, (int)lv, rt.n});
      }
    }
    if (H + 1 < h.Hmax) {
      // xo[H] is sized by height H; the parent vector is shorter, fits
    }
    pl.copy(Prec::F64, Prec::F64, false, ct, 256, nrhs);
  }
  // root solves
  pl.tag("ulv_root");
  {
    GemmBatch gb;
    for (size_t p = 0; p < h.probs.size(); ++p) {
      Root& rt = h.probs[p].root;
      if (!rt.n) continue;
      gb.add1(rootx[p], rt.n, rt.n, nrhs, rt.inv->p, rt.n, rootb[p], rt.n, rt.n);
    }
    pl.gemm(Prec::F64, gb, false, false);
  }
  {
    std::vector<CopyTask> ct;
    for (size_t p = 0; p < h.probs.size(); ++p)
      if (h.probs[p].H == 0)
        ct.push_back(CopyTask{rootx[p], x + h.probs[p].off, h.probs[p].root.n, nrhs, h.probs[p].root.n, (int)ld});
    pl.copy(Prec::F64, Prec::F64, false, ct, 8192, nrhs);
  }
  // backward sweep
  pl.tag("ulv_bwd");
  for (int H = h.Hmax - 1; H >= 0; --H) {
    Height& ht = h.hs[H];
    const int nb = ht.nb;
    const int64_t lv = ht.v_len;
    std::vector<CopyTask> ct;
    for (int g = 0; g < nb; ++g) {
      int m = ht.n[g] - ht.r[g];
      int o = (ht.ref[g].local % 2) ? ht.r[g - 1] : 0;
      const double* src;
      int lds;
      if (ht.parent[g] >= 0) {
        const Height& up = h.hs[H + 1];
        src = xo[H + 1] + up.v_off[ht.parent[g]] + o;
        lds = (int)up.v_len;
      } else {
        Root& rt = h.probs[ht.ref[g].prob].root;
        src = rootx[ht.ref[g].prob] + rt.off[ht.root_slot[g]] + o;
        lds = rt.n;
      }
      ct.push_back(CopyTask{src, c[H] + ht.v_off[g] + m, ht.r[g], nrhs, lds, (int)lv});
    }
    pl.copy(Prec::F64, Prec::F64, false, ct, 256, nrhs);
    // x_R = U^-1 (y_R - U^RS x_S)
    const int64_t ly = std::max<int64_t>(1, ht.y_len);
    GemmBatch g1, gu;
    for (int g = 0; g < nb; ++g) {
      int m = ht.n[g] - ht.r[g];
      if (m == 0) continue;
      double* Sg = ht.S->as<double>() + ht.q_off[g];
      g1.add1(yb[H] + ht.y_off[g], (int)ly, m, nrhs, Sg + (size_t)m * ht.n[g], ht.n[g], c[H] + ht.v_off[g] + m, (int)lv,
              ht.r[g], -1.0, 1.0);
      gu.add1(c[H] + ht.v_off[g], (int)lv, m, nrhs, ht.Uinv->as<double>() + ht.li_off[g], m, yb[H] + ht.y_off[g],
              (int)ly, m);
    }
    pl.gemm(Prec::F64, g1, false, false);
    pl.gemm(Prec::F64, gu, false, false);
    GemmBatch g2;
    for (int g = 0; g < nb; ++g) {
      double* dst;
      int ldd;
      if (H == 0) {
        const BoxRef& bb = ht.ref[g];
        const Problem& pb = h.probs[bb.prob];
        dst = x + pb.off + pb.t.boxes[bb.level][bb.local].s;
        ldd = (int)ld;
      } else {
        dst = xo[H] + ht.v_off[g];
        ldd = (int)lv;
      }
      g2.add1(dst, ldd, ht.n[g], nrhs, ht.Q->as<double>() + ht.q_off[g], ht.n[g], c[H] + ht.v_off[g], (int)lv, ht.n[g]);
    }
    pl.gemm(Prec::F64, g2, false, false);
  }
  return P;
}


// ------------------------------------------------------ allocation-free --
// Log-determinant without any device allocation, for callers that cannot
// call cudaMalloc at that point: a process whose device memory is owned by
// another allocator or fully reserved, or code that must not trigger a
// synchronising allocation between captured or latency-critical launches.
// The per-block task descriptors and partial results live in this
// file-scope device array (every device that loads the library holds it
// until exit); the host-side name is only a stand-in, so its device
// address is looked up once per device with cudaGetSymbolAddress.
namespace {
constexpr int NOALLOC_MAX_BLOCKS = 16384;   // factored blocks per height
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_MAX_BLOCKS * (sizeof(LuTask) + 2 * sizeof(double));
__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];
void* g_noalloc_ptr[256] = {nullptr};
}  // namespace

}  // namespace h2

// ================================================================= C ABI ==
using namespace h2;

static thread_local std::string g_err;

struct h2_handle_ {
  Handle h;
};

template <class F> static h2_status guard(F&& f) {
  try {
    f();
    return H2_OK;
  } catch (const StatusError& e) {
    g_err = e.what();
    return (h2_status)e.status;
  } catch (const CudaError& e) {
    g_err = e.what();
    return H2_ERR_DEVICE;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return H2_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return H2_ERR_DEVICE;
  }
}

static void check_opts(const h2_kernel* k, const h2_options* o) {
  if (!k || !o) throw StatusError(H2_ERR_ARG, "null kernel or options");
  if (k->kind < 0 || k->kind > 2) throw StatusError(H2_ERR_ARG, "unknown kernel kind");
  if (!(o->eta > 0)) throw StatusError(H2_ERR_ARG, "eta must be > 0");
  if (o->leaf < 1 || o->leaf > 256) throw StatusError(H2_ERR_ARG, "leaf must be in [1, 256]");
  if (o->max_rank < 1 || o->max_rank > 256) throw StatusError(H2_ERR_ARG, "max_rank must be in [1, 256]");
  if (!(o->tol >= 0) || !std::isfinite(o->tol)) throw StatusError(H2_ERR_ARG, "tol must be finite and >= 0");
  if (o->far_s0 < 0 || o->far_smin < 0) throw StatusError(H2_ERR_ARG, "far sample sizes must be >= 0");
  if (o->partition != 0 && o->partition != 1) throw StatusError(H2_ERR_ARG, "partition must be 0 or 1");
}

static void construct_impl(h2_handle_* H, int P, const double* const* points, const int64_t* N,
                           const h2_kernel* kern, const h2_options* opt, void* stream) {
  check_opts(kern, opt);
  Handle& h = H->h;
  h.s = (cudaStream_t)stream;
  h.kp = KParams{kern->kind, kern->delta, kern->kappa, kern->ell, kern->nugget};
  h.opt = *opt;
  double t0 = now_ms();
  h.probs.resize(P);
  int64_t off = 0;
  std::vector<double> host;
  for (int p = 0; p < P; ++p) {
    if (N[p] < 1) throw StatusError(H2_ERR_ARG, "N must be >= 1");
    if (N[p] > (int64_t)1 << 30) throw StatusError(H2_ERR_ARG, "N too large");
    if (!points[p]) throw StatusError(H2_ERR_ARG, "null points");
    host.resize((size_t)N[p] * 3);
    if (is_device_ptr(points[p])) {
      H2_CUDA(cudaMemcpy(host.data(), points[p], host.size() * 8, cudaMemcpyDeviceToHost));
    } else {
      std::memcpy(host.data(), points[p], host.size() * 8);
    }
    for (double v : host)
      if (!std::isfinite(v)) throw StatusError(H2_ERR_NONFINITE, "non-finite coordinate");
    Problem& pb = h.probs[p];
    pb.t = build_tree(host.data(), N[p], opt->leaf, opt->eta, opt->partition);
    pb.off = off;
    pb.H = pb.t.L - pb.t.ltop;
    off += N[p];
  }
  h.Ntot = off;
  if (h.Ntot > ((int64_t)1 << 31) - 1) throw StatusError(H2_ERR_ARG, "total N too large");
  // tree-order points and the permutation
  std::vector<double> xs(h.Ntot), ys(h.Ntot), zs(h.Ntot);
  std::vector<int64_t> perm(h.Ntot);
  for (auto& pb : h.probs) {
    for (int64_t q = 0; q < pb.t.N; ++q) {
      xs[pb.off + q] = pb.t.xt[q];
      ys[pb.off + q] = pb.t.yt[q];
      zs[pb.off + q] = pb.t.zt[q];
      perm[pb.off + q] = pb.off + pb.t.perm[q];
    }
  }
  H2_CUDA(cudaGetDevice(&h.dev));
  h.px.alloc(h.Ntot * 8);
  h.py.alloc(h.Ntot * 8);
  h.pz.alloc(h.Ntot * 8);
  h.perm.alloc(h.Ntot * 8);
  H2_CUDA(cudaMemcpy(h.px.p, xs.data(), h.Ntot * 8, cudaMemcpyHostToDevice));
  H2_CUDA(cudaMemcpy(h.py.p, ys.data(), h.Ntot * 8, cudaMemcpyHostToDevice));
  H2_CUDA(cudaMemcpy(h.pz.p, zs.data(), h.Ntot * 8, cudaMemcpyHostToDevice));
  H2_CUDA(cudaMemcpy(h.perm.p, perm.data(), h.Ntot * 8, cudaMemcpyHostToDevice));
  build_heights(h);
  build_operator(h);
  h.t_construct_ms = now_ms() - t0;
}

extern "C" {

h2_status h2_construct(const double* points, int64_t N, const h2_kernel* kern, const h2_options* opt,
                       void* stream, h2_handle* out) {
  if (!out) {
    g_err = "null output handle";
    return H2_ERR_ARG;
  }
  *out = nullptr;
  auto* H = new h2_handle_();
  h2_status st = guard([&] { construct_impl(H, 1, &points, &N, kern, opt, stream); });
  if (st != H2_OK) {
    delete H;
    return st;
  }
  *out = H;
  return H2_OK;
}

h2_status h2_construct_batched(int32_t P, const double* const* points, const int64_t* N, const h2_kernel* kern,
                               const h2_options* opt, void* stream, h2_handle* out) {
  if (!out || P < 1 || !points || !N) {
    g_err = "invalid batched arguments";
    return H2_ERR_ARG;
  }
  *out = nullptr;
  auto* H = new h2_handle_();
  h2_status st = guard([&] { construct_impl(H, P, points, N, kern, opt, stream); });
  if (st != H2_OK) {
    delete H;
    return st;
  }
  *out = H;
  return H2_OK;
}

h2_status h2_factor(h2_handle H, int32_t precision, int32_t spd) {
  if (!H) {
    g_err = "null handle";
    return H2_ERR_ARG;
  }
  if (precision != H2_FP64 && precision != H2_MIXED) {
    g_err = "unknown precision";
    return H2_ERR_ARG;
  }
  return guard([&] {
    Handle& h = H->h;
    h.factored = false;
    h.plans.clear();
    h.pred_hits = h.pred_misses = 0;
    h.pred_bytes = h.worst_bytes = h.exact_bytes = 0;
    double t0 = now_ms();
    factor(h, precision, spd);
    h.t_factor_ms = now_ms() - t0;
    h.precision = precision;
    h.spd = spd;
    h.factored = true;
  });
}

// Workspaces and plans for nrhs right-hand sides (built on first use; the
// ULV plan is rebuilt after each factorization).
static Handle::SolvePlans& solve_plans(Handle& h, int nrhs, bool need_ulv) {
  auto& sp = h.plans[nrhs];
  if (!sp) {
    sp = std::make_shared<Handle::SolvePlans>();
    sp->nrhs = nrhs;
    auto mk = [&](size_t e) {
      auto b = std::make_shared<DBuf>(std::max<size_t>(e, 2) * 8);
      sp->bufs.push_back(b);
      return b->as<double>();
    };
    size_t NE = (size_t)h.Ntot * nrhs;
    sp->B = mk(NE);
    sp->X = mk(NE);
    sp->R = mk(NE);
    sp->Uin = mk(NE);
    sp->Uout = mk(NE);
    sp->nrm = mk(2 * (size_t)nrhs);
    sp->mv = build_matvec_plan(h, sp->X, sp->R, nrhs);
  }
  if (need_ulv && !sp->ulv) sp->ulv = build_ulv_plan(h, sp->Uin, sp->Uout, nrhs);
  return *sp;
}

// Caller block (host or device, caller order, leading dim ld) -> tree order.
static void to_tree(Handle& h, const double* src, int64_t ld, int nrhs, double* dst_tree, double* stage) {
  const double* d = src;
  if (!is_device_ptr(src)) {
    H2_CUDA(cudaMemcpy2DAsync(stage, (size_t)h.Ntot * 8, src, (size_t)ld * 8, (size_t)h.Ntot * 8, nrhs,
                              cudaMemcpyHostToDevice, h.s));
    d = stage;
    ld = h.Ntot;
  }
  launch_permute_rows(d, ld, dst_tree, h.Ntot, h.perm.as<int64_t>(), h.Ntot, nrhs, false, h.s);
}

static void from_tree(Handle& h, const double* src_tree, double* dst, int64_t ld, int nrhs, double* stage) {
  if (is_device_ptr(dst)) {
    launch_permute_rows(src_tree, h.Ntot, dst, ld, h.perm.as<int64_t>(), h.Ntot, nrhs, true, h.s);
  } else {
    launch_permute_rows(src_tree, h.Ntot, stage, h.Ntot, h.perm.as<int64_t>(), h.Ntot, nrhs, true, h.s);
    H2_CUDA(cudaMemcpy2DAsync(dst, (size_t)ld * 8, stage, (size_t)h.Ntot * 8, (size_t)h.Ntot * 8, nrhs,
                              cudaMemcpyDeviceToHost, h.s));
  }
  H2_CUDA(cudaStreamSynchronize(h.s));
}


// GMRES-based refinement (right preconditioned): FP64 GMRES(m) on the H^2
// operator, ULV factors as the preconditioner, classical Gram-Schmidt applied
// twice, everything on the device except the small Givens / least-squares
// work on the Hessenberg columns (one device-to-host read per Arnoldi step).
static void gmres_solve(Handle& h, Handle::SolvePlans& sp, int nrhs, double target, int max_iter,
                        const std::vector<double>& bn2, std::vector<double>& rel, int& iters, bool& converged) {
  const int64_t N = h.Ntot;
  const size_t blk = (size_t)N * nrhs;
  const int m = std::max(1, std::min(30, max_iter));
  if (!sp.V || sp.m < m) {
    auto mk = [&](size_t e) {
      auto b = std::make_shared<DBuf>(std::max<size_t>(e, 2) * 8);
      sp.bufs.push_back(b);
      return b->as<double>();
    };
    sp.V = mk(blk * (m + 1));
    sp.Xsol = mk(blk);
    sp.hdev = mk((size_t)nrhs * 3 * 32);
    sp.part = mk((size_t)608 * 32);
    sp.ydev = mk((size_t)nrhs * 32);
    sp.m = m;
  }
  cudaStream_t s = h.s;
  std::vector<double> bnorm(nrhs);
  for (int c = 0; c < nrhs; ++c) bnorm[c] = bn2[c] > 0 ? std::sqrt(bn2[c]) : 1.0;
  // x0 = ULV^-1 b
  H2_CUDA(cudaMemcpyAsync(sp.Uin, sp.B, blk * 8, cudaMemcpyDeviceToDevice, s));
  sp.ulv->run(s);
  H2_CUDA(cudaMemcpyAsync(sp.Xsol, sp.Uout, blk * 8, cudaMemcpyDeviceToDevice, s));
  iters = 0;
  converged = false;
  std::vector<double> rn(nrhs), hh((size_t)nrhs * 3 * 32), nrm2(nrhs);
  Scratch sc(s);
  while (true) {
    // R = A x - b, the FP64 H^2 residual
    H2_CUDA(cudaMemcpyAsync(sp.X, sp.Xsol, blk * 8, cudaMemcpyDeviceToDevice, s));
    sp.mv->run(s);
    launch_axpy_cols(sp.R, sp.B, (int)N, nrhs, N, N, -1.0, s);
    launch_colnorm2(sp.R, (int)N, nrhs, N, sp.nrm, s);
    H2_CUDA(cudaMemcpyAsync(rn.data(), sp.nrm, nrhs * 8, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    bool ok = true;
    for (int c = 0; c < nrhs; ++c) {
      rel[c] = std::sqrt(rn[c]) / bnorm[c];
      if (!(rel[c] <= target)) ok = false;
    }
    if (ok) {
      converged = true;
      return;
    }
    if (iters >= max_iter) return;
    // V_0 = R / ||R||, g = -||R|| e_1
    for (int c = 0; c < nrhs; ++c)
      launch_normalize(sp.V + (size_t)c * N, sp.R + (size_t)c * N, N, sp.nrm + c, s);
    std::vector<std::vector<double>> H((size_t)nrhs, std::vector<double>((size_t)(m + 1) * m, 0.0));
    std::vector<std::vector<double>> g((size_t)nrhs, std::vector<double>(m + 1, 0.0));
    std::vector<std::vector<double>> cs((size_t)nrhs, std::vector<double>(m, 0.0)), sn = cs;
    for (int c = 0; c < nrhs; ++c) g[c][0] = -std::sqrt(rn[c]);
    int jend = -1;
    for (int j = 0; j < m && iters < max_iter; ++j) {
      double* Vj = sp.V + (size_t)j * blk;
      H2_CUDA(cudaMemcpyAsync(sp.Uin, Vj, blk * 8, cudaMemcpyDeviceToDevice, s));
      sp.ulv->run(s);                                                     // Z = M^-1 v_j
      H2_CUDA(cudaMemcpyAsync(sp.X, sp.Uout, blk * 8, cudaMemcpyDeviceToDevice, s));
      sp.mv->run(s);                                                      // w = A Z
      ++iters;
      for (int c = 0; c < nrhs; ++c) {
        double* w = sp.R + (size_t)c * N;
        const double* Vc = sp.V + (size_t)c * N;
        for (int pass = 0; pass < 2; ++pass) {
          double* hc = sp.hdev + ((size_t)c * 3 + pass) * 32;
          launch_mdot(Vc, (int64_t)blk, j + 1, w, N, sp.part, hc, s);
          GemmBatch gb;
          gb.add1(w, (int)N, (int)N, 1, Vc, (int)blk, hc, j + 1, j + 1, -1.0, 1.0);
          gb.run(Prec::F64, false, false, sc);
        }
      }
      launch_colnorm2(sp.R, (int)N, nrhs, N, sp.nrm, s);
      for (int c = 0; c < nrhs; ++c)
        launch_normalize(sp.V + (size_t)(j + 1) * blk + (size_t)c * N, sp.R + (size_t)c * N, N, sp.nrm + c, s);
      H2_CUDA(cudaMemcpyAsync(hh.data(), sp.hdev, hh.size() * 8, cudaMemcpyDeviceToHost, s));
      H2_CUDA(cudaMemcpyAsync(nrm2.data(), sp.nrm, nrhs * 8, cudaMemcpyDeviceToHost, s));
      H2_CUDA(cudaStreamSynchronize(s));
      bool all = true;
      for (int c = 0; c < nrhs; ++c) {
        std::vector<double>& Hc = H[c];
        auto Hx = [&](int i, int jj) -> double& { return Hc[(size_t)i + (size_t)jj * (m + 1)]; };
        for (int i = 0; i <= j; ++i) Hx(i, j) = hh[((size_t)c * 3 + 0) * 32 + i] + hh[((size_t)c * 3 + 1) * 32 + i];
        Hx(j + 1, j) = std::sqrt(std::max(0.0, nrm2[c]));
        for (int i = 0; i < j; ++i) {   // previous rotations
          double t = cs[c][i] * Hx(i, j) + sn[c][i] * Hx(i + 1, j);
          Hx(i + 1, j) = -sn[c][i] * Hx(i, j) + cs[c][i] * Hx(i + 1, j);
          Hx(i, j) = t;
        }
        double a0 = Hx(j, j), b0 = Hx(j + 1, j);
        double rr = std::hypot(a0, b0);
        cs[c][j] = rr > 0 ? a0 / rr : 1.0;
        sn[c][j] = rr > 0 ? b0 / rr : 0.0;
        Hx(j, j) = rr;
        Hx(j + 1, j) = 0.0;
        g[c][j + 1] = -sn[c][j] * g[c][j];
        g[c][j] = cs[c][j] * g[c][j];
        if (!(std::fabs(g[c][j + 1]) / bnorm[c] <= 0.5 * target)) all = false;
      }
      jend = j;
      if (all) break;
    }
    if (jend < 0) return;
    // x += M^-1 (V y), y = H^-1 g (upper triangular)
    std::vector<double> y((size_t)nrhs * 32, 0.0);
    for (int c = 0; c < nrhs; ++c) {
      auto Hx = [&](int i, int jj) -> double { return H[c][(size_t)i + (size_t)jj * (m + 1)]; };
      for (int i = jend; i >= 0; --i) {
        double t = g[c][i];
        for (int k = i + 1; k <= jend; ++k) t -= Hx(i, k) * y[(size_t)c * 32 + k];
        y[(size_t)c * 32 + i] = Hx(i, i) != 0.0 ? t / Hx(i, i) : 0.0;
      }
    }
    H2_CUDA(cudaMemcpyAsync(sp.ydev, y.data(), y.size() * 8, cudaMemcpyHostToDevice, s));
    {
      GemmBatch gb;
      for (int c = 0; c < nrhs; ++c)
        gb.add1(sp.Uin + (size_t)c * N, (int)N, (int)N, 1, sp.V + (size_t)c * N, (int)blk, sp.ydev + (size_t)c * 32,
                jend + 1, jend + 1);
      gb.run(Prec::F64, false, false, sc);
    }
    sp.ulv->run(s);
    launch_axpy_cols(sp.Xsol, sp.Uout, (int)N, nrhs, N, N, 1.0, s);
  }
}

h2_status h2_matvec(h2_handle H, const double* x, double* y, int32_t nrhs, int64_t ld) {
  if (!H || !x || !y || nrhs < 1 || ld < H->h.Ntot) {
    g_err = "invalid matvec arguments";
    return H2_ERR_ARG;
  }
  return guard([&] {
    Handle& h = H->h;
    auto& sp = solve_plans(h, nrhs, false);
    to_tree(h, x, ld, nrhs, sp.X, sp.Uin);
    sp.mv->run(h.s);
    from_tree(h, sp.R, y, ld, nrhs, sp.Uin);
  });
}

h2_status h2_solve(h2_handle H, const double* b, double* x, int32_t nrhs, int64_t ld, double target,
                   int32_t max_iter, double* achieved, int32_t* iters) {
  if (!H || !b || !x || nrhs < 1 || ld < H->h.Ntot || max_iter < 0) {
    g_err = "invalid solve arguments";
    return H2_ERR_ARG;
  }
  if (!H->h.factored) {
    g_err = "h2_solve before h2_factor";
    return H2_ERR_STATE;
  }
  bool converged = true;
  h2_status st = guard([&] {
    Handle& h = H->h;
    const int64_t N = h.Ntot;
    const size_t bytes = (size_t)N * nrhs * 8;
    auto& sp = solve_plans(h, nrhs, true);
    to_tree(h, b, ld, nrhs, sp.B, sp.Uin);
    launch_colnorm2(sp.B, (int)N, nrhs, N, sp.nrm, h.s);
    std::vector<double> bn(nrhs);
    H2_CUDA(cudaMemcpyAsync(bn.data(), sp.nrm, nrhs * 8, cudaMemcpyDeviceToHost, h.s));
    H2_CUDA(cudaStreamSynchronize(h.s));
    for (double v : bn)
      if (!std::isfinite(v)) throw StatusError(H2_ERR_NONFINITE, "non-finite right-hand side");
    std::vector<double> rel(nrhs, 0.0);
    const char* mode = getenv("H2_REFINE");
    const bool use_gmres = nrhs <= 8 && !(mode && std::string(mode) == "stationary") && !h.per_problem;
    // squared column norms per problem segment (tree-order rows [off, off + N))
    // when every problem is checked on its own, else over the whole column
    const size_t nseg = h.per_problem ? h.probs.size() : 1;
    std::vector<double> bseg(nseg * nrhs), rseg(nseg * nrhs);
    auto seg_norms = [&](const double* V, std::vector<double>& out) {
      if (nseg == 1) {
        launch_colnorm2(V, (int)N, nrhs, N, sp.nrm, h.s);
        H2_CUDA(cudaMemcpyAsync(out.data(), sp.nrm, nrhs * 8, cudaMemcpyDeviceToHost, h.s));
      } else {
        ensure(h.segnrm, nseg * nrhs * 8);
        double* d = h.segnrm->as<double>();
        for (size_t q = 0; q < nseg; ++q)
          launch_colnorm2(V + h.probs[q].off, (int)h.probs[q].t.N, nrhs, N, d + q * nrhs, h.s);
        H2_CUDA(cudaMemcpyAsync(out.data(), d, nseg * nrhs * 8, cudaMemcpyDeviceToHost, h.s));
      }
      H2_CUDA(cudaStreamSynchronize(h.s));
    };
    if (nseg > 1) seg_norms(sp.B, bseg);
    if (use_gmres) {
      int it = 0;
      bool conv = false;
      gmres_solve(h, sp, nrhs, target, max_iter, bn, rel, it, conv);
      converged = conv;
      from_tree(h, sp.Xsol, x, ld, nrhs, sp.Uin);
      if (achieved)
        for (int c = 0; c < nrhs; ++c) achieved[c] = rel[c];
      if (iters) *iters = it;
      return;
    }
    // stationary refinement: x0 = ULV^-1 b, x <- x - ULV^-1 (A x - b)
    H2_CUDA(cudaMemcpyAsync(sp.Uin, sp.B, bytes, cudaMemcpyDeviceToDevice, h.s));
    sp.ulv->run(h.s);
    H2_CUDA(cudaMemcpyAsync(sp.X, sp.Uout, bytes, cudaMemcpyDeviceToDevice, h.s));
    int it = 0;
    if (nseg == 1) bseg = bn;
    while (true) {
      sp.mv->run(h.s);                                               // R = A_H2 X
      launch_axpy_cols(sp.R, sp.B, (int)N, nrhs, N, N, -1.0, h.s);   // R = A X - b
      seg_norms(sp.R, rseg);
      bool ok = true;
      std::fill(rel.begin(), rel.end(), 0.0);
      h.last_rel.assign(nseg * nrhs, 0.0);
      for (size_t q = 0; q < nseg; ++q)
        for (int c = 0; c < nrhs; ++c) {
          const double bq = bseg[q * nrhs + c];
          const double rq = bq > 0 ? std::sqrt(rseg[q * nrhs + c]) / std::sqrt(bq) : std::sqrt(rseg[q * nrhs + c]);
          h.last_rel[q * nrhs + c] = rq;
          rel[c] = std::max(rel[c], rq);
          if (!(rq <= target)) ok = false;
        }
      if (ok || it >= max_iter) {
        converged = ok;
        break;
      }
      // X <- X - ULV^-1 (A X - b)
      H2_CUDA(cudaMemcpyAsync(sp.Uin, sp.R, bytes, cudaMemcpyDeviceToDevice, h.s));
      sp.ulv->run(h.s);
      launch_axpy_cols(sp.X, sp.Uout, (int)N, nrhs, N, N, -1.0, h.s);
      ++it;
    }
    from_tree(h, sp.X, x, ld, nrhs, sp.Uin);
    if (achieved)
      for (int c = 0; c < nrhs; ++c) achieved[c] = rel[c];
    if (iters) *iters = it;
  });
  if (st == H2_OK && !converged) {
    g_err = "refinement did not reach the target residual";
    return H2_ERR_NOT_CONVERGED;
  }
  return st;
}

h2_status h2_solve_batched(h2_handle H, const double* const* b, double* const* x, const int32_t* nrhs,
                           const int64_t* ld, double target, int32_t max_iter, double* achieved, int32_t* iters) {
  if (!H || !b || !x || !nrhs || !ld || max_iter < 0) {
    g_err = "invalid batched solve arguments";
    return H2_ERR_ARG;
  }
  if (!H->h.factored) {
    g_err = "h2_solve_batched before h2_factor";
    return H2_ERR_STATE;
  }
  Handle& h = H->h;
  const size_t P = h.probs.size();
  int nmax = 0;
  for (size_t p = 0; p < P; ++p) {
    const int64_t Np = h.probs[p].t.N;
    if (!b[p] || !x[p] || nrhs[p] < 1 || ld[p] < Np) {
      g_err = "invalid batched solve arguments (problem " + std::to_string(p) + ")";
      return H2_ERR_ARG;
    }
    nmax = std::max(nmax, (int)nrhs[p]);
  }
  std::vector<double> ach((size_t)nmax, 0.0);
  int it = 0;
  h2_status st = guard([&] {
    // stack the problems' columns (rows by problem, caller order), zero-padded
    // to the largest count: a zero column is solved exactly at no extra sweep
    const size_t bytes = (size_t)h.Ntot * nmax * 8;
    ensure(h.bstage, bytes);
    ensure(h.xstage, bytes);
    double* B = h.bstage->as<double>();
    H2_CUDA(cudaMemsetAsync(B, 0, bytes, h.s));
    for (size_t p = 0; p < P; ++p) {
      const int64_t Np = h.probs[p].t.N;
      H2_CUDA(cudaMemcpy2DAsync(B + h.probs[p].off, (size_t)h.Ntot * 8, b[p], (size_t)ld[p] * 8, (size_t)Np * 8,
                                nrhs[p], cudaMemcpyDefault, h.s));
    }
  });
  if (st != H2_OK) return st;
  h.per_problem = true;
  const h2_status sst = h2_solve(H, h.bstage->as<double>(), h.xstage->as<double>(), nmax, h.Ntot, target, max_iter,
                                 ach.data(), &it);
  h.per_problem = false;
  if (sst != H2_OK && sst != H2_ERR_NOT_CONVERGED) return sst;
  st = guard([&] {
    const double* X = h.xstage->as<double>();
    for (size_t p = 0; p < P; ++p) {
      const int64_t Np = h.probs[p].t.N;
      H2_CUDA(cudaMemcpy2DAsync(x[p], (size_t)ld[p] * 8, X + h.probs[p].off, (size_t)h.Ntot * 8, (size_t)Np * 8,
                                nrhs[p], cudaMemcpyDefault, h.s));
    }
    H2_CUDA(cudaStreamSynchronize(h.s));
  });
  if (st != H2_OK) return st;
  if (achieved)   // per problem: the largest relative residual over its own columns
    for (size_t p = 0; p < P; ++p) {
      double a = 0.0;
      for (int c = 0; c < nrhs[p]; ++c)
        a = std::max(a, h.last_rel.size() == P * (size_t)nmax ? h.last_rel[p * nmax + c] : ach[c]);
      achieved[p] = a;
    }
  if (iters) *iters = it;
  if (sst == H2_ERR_NOT_CONVERGED) g_err = "refinement did not reach the target residual";
  return sst;
}

h2_status h2_logdet(h2_handle H, double* log_abs_det, int32_t* sign) {
  if (!H || !log_abs_det) {
    g_err = "invalid logdet arguments";
    return H2_ERR_ARG;
  }
  if (!H->h.factored) {
    g_err = "h2_logdet before h2_factor";
    return H2_ERR_STATE;
  }
  return guard([&] {
    Handle& h = H->h;
    Scratch sc(h.s);
    std::vector<double> ld(h.probs.size(), 0.0), sg(h.probs.size(), 1.0);
    for (int Hh = 0; Hh < h.Hmax; ++Hh) {
      Height& ht = h.hs[Hh];
      std::vector<LuTask> lt;
      std::vector<int> who;
      for (int g = 0; g < ht.nb; ++g) {
        int m = ht.n[g] - ht.r[g];
        if (m == 0) continue;
        lt.push_back(LuTask{ht.S->as<double>() + ht.q_off[g], m, m, ht.n[g], ht.pivRR->as<int>() + ht.pv_off[g], nullptr, 0});
        who.push_back(ht.ref[g].prob);
      }
      if (lt.empty()) continue;
      double* o = (double*)sc.alloc(lt.size() * 16);
      launch_logdet_lu(sc.up(lt), (int)lt.size(), o, o + lt.size(), false, h.s);
      std::vector<double> ho(lt.size() * 2);
      H2_CUDA(cudaMemcpyAsync(ho.data(), o, ho.size() * 8, cudaMemcpyDeviceToHost, h.s));
      H2_CUDA(cudaStreamSynchronize(h.s));
      for (size_t i = 0; i < lt.size(); ++i) {
        ld[who[i]] += ho[i];
        sg[who[i]] *= ho[lt.size() + i];
      }
    }
    for (size_t p = 0; p < h.probs.size(); ++p) {
      ld[p] += h.probs[p].root.logdet;
      sg[p] *= h.probs[p].root.sign;
      log_abs_det[p] = ld[p];
      if (sign) sign[p] = sg[p] < 0 ? -1 : 1;
    }
  });
}


h2_status h2_logdet_noalloc(h2_handle H, double* log_abs_det, int32_t* sign) {
  if (!H || !log_abs_det) {
    g_err = "invalid logdet arguments";
    return H2_ERR_ARG;
  }
  if (!H->h.factored) {
    g_err = "h2_logdet_noalloc before h2_factor";
    return H2_ERR_STATE;
  }
  return guard([&] {
    Handle& h = H->h;
    // The scratch array used is the one on the handle's device (where its
    // factors and stream live), made current for the duration of the call
    // when the caller's current device is another one.
    const int dev = h.dev;
    if (dev < 0 || dev >= 256) throw StatusError(H2_ERR_ARG, "device index out of range");
    int cur = 0;
    H2_CUDA(cudaGetDevice(&cur));
    struct Restore {
      int prev, now;
      ~Restore() {
        if (prev != now) (void)cudaSetDevice(prev);
      }
    } restore{cur, dev};
    if (cur != dev) H2_CUDA(cudaSetDevice(dev));
    if (!g_noalloc_ptr[dev]) {
      // first call on this device: resolve the scratch array's device address
      // (the host-side name is only a stand-in), with that device current
      void* p = nullptr;
      H2_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_ptr[dev] = p;
    }
    LuTask* d_tasks = reinterpret_cast<LuTask*>(g_noalloc_ptr[dev]);
    double* d_out = reinterpret_cast<double*>(reinterpret_cast<char*>(g_noalloc_ptr[dev]) +
                                              (size_t)NOALLOC_MAX_BLOCKS * sizeof(LuTask));
    const size_t P = h.probs.size();
    for (size_t p = 0; p < P; ++p) {
      log_abs_det[p] = h.probs[p].root.logdet;
      if (sign) sign[p] = h.probs[p].root.sign < 0 ? -1 : 1;
    }
    std::vector<LuTask> lt;
    std::vector<int> who;
    std::vector<double> ho;
    for (int Hh = 0; Hh < h.Hmax; ++Hh) {
      Height& ht = h.hs[Hh];
      lt.clear();
      who.clear();
      for (int g = 0; g < ht.nb; ++g) {
        int m = ht.n[g] - ht.r[g];
        if (m == 0) continue;
        lt.push_back(LuTask{ht.S->as<double>() + ht.q_off[g], m, m, ht.n[g], ht.pivRR->as<int>() + ht.pv_off[g], nullptr, 0});
        who.push_back(ht.ref[g].prob);
      }
      if (lt.empty()) continue;
      if (lt.size() > (size_t)NOALLOC_MAX_BLOCKS)
        throw StatusError(H2_ERR_ARG, "h2_logdet_noalloc: more than 16384 factored blocks at one height");
      const int nblk = (int)lt.size();
      H2_CUDA(cudaMemcpyAsync(d_tasks, lt.data(), lt.size() * sizeof(LuTask), cudaMemcpyHostToDevice, h.s));
      launch_logdet_lu(d_tasks, nblk, d_out, d_out + nblk, false, h.s);
      ho.resize(2 * (size_t)nblk);
      H2_CUDA(cudaMemcpyAsync(ho.data(), d_out, ho.size() * sizeof(double), cudaMemcpyDeviceToHost, h.s));
      H2_CUDA(cudaStreamSynchronize(h.s));
      for (int i = 0; i < nblk; ++i) {
        log_abs_det[who[i]] += ho[i];
        if (sign && ho[nblk + i] < 0) sign[who[i]] = -sign[who[i]];
      }
    }
  });
}

h2_status h2_stats(h2_handle H, char* json, size_t cap) {
  if (!H || !json || cap == 0) {
    g_err = "invalid stats arguments";
    return H2_ERR_ARG;
  }
  return guard([&] {
    Handle& h = H->h;
    std::ostringstream o;
    o << "{\"N\":" << h.Ntot << ",\"problems\":" << h.probs.size() << ",\"heights\":" << h.Hmax
      << ",\"construct_ms\":" << h.t_construct_ms << ",\"factor_ms\":" << h.t_factor_ms
      << ",\"basis_route\":\"" << (h.factored ? h.basis_route : "none")
      << "\",\"tol_basis\":" << h.tol_basis << ",\"levels\":[";
    for (int H2i = 0; H2i < h.Hmax; ++H2i) {
      const Height& ht = h.hs[H2i];
      double rs = 0, rmax = 0, ro = 0, nearc = 0, farc = 0;
      for (int g = 0; g < ht.nb; ++g) {
        if (!ht.r.empty()) {
          rs += ht.r[g];
          rmax = std::max(rmax, (double)ht.r[g]);
        }
        if (!ht.r_op.empty()) ro += ht.r_op[g];
        nearc += ht.near[g].size();
        farc += ht.far[g].size();
      }
      if (H2i) o << ",";
      o << "{\"height\":" << H2i << ",\"boxes\":" << ht.nb << ",\"rank_mean\":" << (ht.nb ? rs / ht.nb : 0)
        << ",\"rank_max\":" << rmax << ",\"op_rank_mean\":" << (ht.nb ? ro / ht.nb : 0)
        << ",\"near_mean\":" << (ht.nb ? nearc / ht.nb : 0) << ",\"far_mean\":" << (ht.nb ? farc / ht.nb : 0);
      if ((size_t)H2i < h.level_ms.size()) o << ",\"factor_ms\":" << h.level_ms[H2i];
      o << "}";
    }
    o << "],\"roots\":[";
    for (size_t p = 0; p < h.probs.size(); ++p) o << (p ? "," : "") << h.probs[p].root.n;
    o << "],\"predictor\":{\"attached\":" << (h.predictor ? 1 : 0) << ",\"hits\":" << h.pred_hits
      << ",\"misses\":" << h.pred_misses << ",\"presized_bytes\":" << h.pred_bytes
      << ",\"worstcase_bytes\":" << h.worst_bytes << ",\"exact_bytes\":" << h.exact_bytes << "}";
    o << ",\"autotune\":" << autotune_report();
    o << ",\"launches\":" << prof().total_launches << ",\"kernels\":{";
    prof().resolve();
    bool first = true;
    for (auto& kv : prof().stats) {
      o << (first ? "" : ",") << "\"" << kv.first << "\":{\"launches\":" << kv.second.launches
        << ",\"ms\":" << kv.second.ms << ",\"flops\":" << kv.second.flops << ",\"bytes\":" << kv.second.bytes
        << "}";
      first = false;
    }
    o << "}}";
    std::string sj = o.str();
    size_t n = std::min(cap - 1, sj.size());
    std::memcpy(json, sj.data(), n);
    json[n] = 0;
  });
}

h2_status h2_box_features(h2_handle H, int32_t height, float* features, int32_t* ranks, int32_t* nboxes) {
  if (!H || height < 0 || height >= H->h.Hmax) {
    g_err = "invalid h2_box_features arguments";
    return H2_ERR_ARG;
  }
  return guard([&] {
    Handle& h = H->h;
    const Height& ht = h.hs[height];
    if (nboxes) *nboxes = ht.nb;
    if (features) {
      std::vector<float> F;
      height_features(h, height, F);
      std::memcpy(features, F.data(), F.size() * 4);
    }
    if (ranks) {
      if (!h.factored) throw StatusError(H2_ERR_STATE, "ranks need h2_factor first");
      for (int g = 0; g < ht.nb; ++g) ranks[g] = ht.r[g];
    }
  });
}

h2_status h2_set_rank_predictor(h2_handle H, h2_mlp m, double margin) {
  if (!H || !(margin >= 0)) {
    g_err = "invalid h2_set_rank_predictor arguments";
    return H2_ERR_ARG;
  }
  H->h.predictor = m ? reinterpret_cast<const Mlp*>(m) : nullptr;
  H->h.pred_margin = margin;
  return H2_OK;
}

h2_status h2_profile(int32_t enable, int32_t reset) {
  return guard([&] {
    if (reset) prof().reset();
    prof().timing = enable != 0;
  });
}

const char* h2_last_error(void) { return g_err.c_str(); }

void h2_destroy(h2_handle H) {
  delete H;
  h2::scratch_cache_release();
}

}  // extern "C"
