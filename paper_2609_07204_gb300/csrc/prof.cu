// prof.cu -- per-kernel CUDA-event timing used by the optional profile mode.
#include <vector>

#include "kernels.h"

namespace mc {

struct ProfRec {
  int cat;
  long long units;
  cudaEvent_t a, b;
};

struct Profiler {
  std::vector<ProfRec> recs;
  std::vector<cudaEvent_t> pool;
  double ms[P_NCAT] = {};
  long long launches[P_NCAT] = {};
  long long units[P_NCAT] = {};
};

thread_local Profiler* tl_prof = nullptr;

static const char* kNames[P_NCAT] = {"degree", "lp_sweep", "lp_bound", "pr_marks",
                                     "capforest_passes", "capforest_seq", "union_find", "emit",
                                     "sort_hist", "sort_pass", "build_csr", "tile_rows",
                                     "witness", "other", "contract_rows", "batch_warp"};

const char* prof_name(int cat) { return (cat >= 0 && cat < P_NCAT) ? kNames[cat] : "?"; }

static cudaEvent_t take(Profiler* p) {
  if (!p->pool.empty()) {
    cudaEvent_t e = p->pool.back();
    p->pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

ProfScope::ProfScope(int c, long long u, cudaStream_t st) : cat(c), units(u), s(st), idx(-1) {
  Profiler* p = tl_prof;
  if (!p) return;
  ProfRec r{c, u, take(p), take(p)};
  cudaEventRecord(r.a, s);
  p->recs.push_back(r);
  idx = (int)p->recs.size() - 1;
}

ProfScope::~ProfScope() {
  Profiler* p = tl_prof;
  if (!p || idx < 0) return;
  cudaEventRecord(p->recs[idx].b, s);
}

Profiler* prof_create() { return new Profiler(); }

void prof_destroy(Profiler* p) {
  if (!p) return;
  for (auto& r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto e : p->pool) cudaEventDestroy(e);
  delete p;
}

// Resolve recorded events (the stream must have been synchronised).
void prof_flush(Profiler* p) {
  if (!p) return;
  for (auto& r : p->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      p->ms[r.cat] += ms;
      p->launches[r.cat] += 1;
      p->units[r.cat] += r.units;
    }
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->recs.clear();
  cudaGetLastError();
}

void prof_read(const Profiler* p, int cat, double* ms, long long* launches, long long* units) {
  *ms = p->ms[cat];
  *launches = p->launches[cat];
  *units = p->units[cat];
}

void prof_reset(Profiler* p) {
  for (int i = 0; i < P_NCAT; ++i) { p->ms[i] = 0; p->launches[i] = 0; p->units[i] = 0; }
}

}  // namespace mc
