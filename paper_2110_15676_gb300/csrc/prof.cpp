// Per-kernel device timing of the library's launches (diagnostics only).
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "afc_internal.h"

namespace afc {

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  struct Rec { const char* name; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::map<std::string, std::pair<double, int64_t>> agg;

  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  // fold recorded pairs into the totals (synchronises with the recorded events)
  void drain() {
    for (auto& r : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        auto& a = agg[r.name];
        a.first += ms;
        a.second += 1;
      }
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
};

cudaEvent_t prof_start(afc_problem_s* p) {
  p->launches++;
  if (!p->prof || !p->prof->on) return nullptr;
  cudaEvent_t e = p->prof->get();
  if (e) cudaEventRecord(e, p->stream);
  return e;
}

void prof_stop(afc_problem_s* p, const char* name, cudaEvent_t start) {
  if (!start || !p->prof) return;
  cudaEvent_t e = p->prof->get();
  if (!e) return;
  cudaEventRecord(e, p->stream);
  p->prof->pending.push_back({name, start, e});
  if (p->prof->pending.size() >= 100000) p->prof->drain();
}

bool prof_set_enabled(afc_problem_s* p, bool on) {
  if (!p->prof) return false;
  const bool was = p->prof->on;
  p->prof->on = on;
  return was;
}

void prof_free(afc_problem_s* p) {
  if (!p->prof) return;
  p->prof->drain();
  for (auto e : p->prof->pool) cudaEventDestroy(e);
  delete p->prof;
  p->prof = nullptr;
}

}  // namespace afc

using namespace afc;

extern "C" int afc_profile(afc_problem p, int mode) {
  if (!p) return AFC_E_INVALID;
  if (!p->prof) p->prof = new Profiler();
  p->prof->drain();
  if (mode) p->prof->agg.clear();
  p->prof->on = mode != 0;
  return AFC_OK;
}

extern "C" int afc_profile_read(afc_problem p, int cap, char* names, double* total_ms, int64_t* launches, int* n,
                                int64_t* all_launches) {
  if (!p) return AFC_E_INVALID;
  if (all_launches) *all_launches = p->launches;
  if (n) *n = 0;
  if (!p->prof) return AFC_OK;
  p->prof->drain();
  int k = 0;
  for (auto& kv : p->prof->agg) {
    if (k >= cap) break;
    if (names) {
      std::strncpy(names + 48 * k, kv.first.c_str(), 47);
      names[48 * k + 47] = 0;
    }
    if (total_ms) total_ms[k] = kv.second.first;
    if (launches) launches[k] = kv.second.second;
    ++k;
  }
  if (n) *n = k;
  return AFC_OK;
}
