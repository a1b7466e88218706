#include "h2_prof.h"

namespace h2 {

Prof& prof() {
  static Prof p;
  return p;
}

void prof_note(double flops, double bytes) {
  prof().next_flops += flops;
  prof().next_bytes += bytes;
}

void prof_tag(const char* tag) { prof().tag = tag ? tag : ""; }

void prof_add(const char* base, double flops) {
  std::string name(base);
  if (!prof().tag.empty()) name += "@" + prof().tag;
  auto it = prof().stats.find(name);
  if (it != prof().stats.end()) it->second.flops += flops;
}

void Prof::resolve() {
  for (auto& q : pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess)
      stats[q.name].ms += ms;
    cudaEventDestroy(q.a);
    cudaEventDestroy(q.b);
  }
  pending.clear();
  (void)cudaGetLastError();
}

void Prof::reset() {
  resolve();
  stats.clear();
  total_launches = 0;
}

ProfScope::ProfScope(const char* n, cudaStream_t st) : name(n), s(st) {
  Prof& p = prof();
  if (!p.tag.empty()) name += "@" + p.tag;
  KStat& k = p.stats[name];
  k.launches += 1;
  k.flops += p.next_flops;
  k.bytes += p.next_bytes;
  p.next_flops = p.next_bytes = 0.0;
  p.total_launches += 1;
  if (p.timing) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
  }
}

ProfScope::~ProfScope() {
  if (a) {
    cudaEventRecord(b, s);
    prof().pending.push_back(Prof::Pending{name, a, b});
  }
}

}  // namespace h2
