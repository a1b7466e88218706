// Per-kernel launch counting and optional CUDA-event timing.  The caller of
// a launch wrapper may note the algorithmic flops and bytes of the next
// launch; with timing enabled each launch is bracketed by events on its own
// stream and the durations are resolved when statistics are read.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

namespace h2 {

struct KStat {
  long long launches = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

struct Prof {
  bool timing = false;
  std::map<std::string, KStat> stats;
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double next_flops = 0.0, next_bytes = 0.0;
  std::string tag;                 // call-site tag appended to kernel names
  long long total_launches = 0;
  void resolve();
  void reset();
};

Prof& prof();
void prof_note(double flops, double bytes);
void prof_tag(const char* tag);   // nullptr clears
// Add flops to the statistics of kernel `base` under the current tag (work
// known only after the launch, e.g. rank-dependent).
void prof_add(const char* base, double flops);

struct ProfScope {
  std::string name;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(const char* n, cudaStream_t st);
  ~ProfScope();
};

}  // namespace h2
