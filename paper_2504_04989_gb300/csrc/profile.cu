// profile.cu -- optional per-stage timing with CUDA events on the launching
// stream.  While enabled, every pipeline stage records an event pair around
// its kernels; tsvd_profile_end() synchronises and sums the elapsed times per
// stage name.  The state is process-global and not thread safe: it is a
// diagnostic for benchmarks, off by default.
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace tsvd {

struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
static bool g_on = false;
static unsigned long long g_launches = 0;

void count_launch() { __atomic_add_fetch(&g_launches, 1ULL, __ATOMIC_RELAXED); }
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_pool;

static cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

StageTimer::StageTimer(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
  if (!g_on) return;
  a_ = get_event();
  cudaEventRecord((cudaEvent_t)a_, s_);
}

StageTimer::~StageTimer() {
  if (!g_on || !a_) return;
  cudaEvent_t b = get_event();
  cudaEventRecord(b, s_);
  g_recs.push_back(Rec{name_, (cudaEvent_t)a_, b});
}

}  // namespace tsvd

using namespace tsvd;

extern "C" int tsvd_profile_begin(void) {
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_on = true;
  return TSVD_OK;
}

extern "C" int tsvd_profile_end(tsvd_stage_time* out, int max_out, int* n_out) {
  g_on = false;
  if (n_out) *n_out = 0;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int> cnt;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return TSVD_ERR_CUDA;
    float t = 0;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return TSVD_ERR_CUDA;
    size_t k = 0;
    while (k < names.size() && names[k] != r.name) ++k;
    if (k == names.size()) {
      names.push_back(r.name);
      ms.push_back(0);
      cnt.push_back(0);
    }
    ms[k] += t;
    cnt[k] += 1;
  }
  int n = 0;
  for (size_t k = 0; k < names.size() && n < max_out; ++k, ++n) {
    if (!out) break;
    memset(out[n].name, 0, sizeof(out[n].name));
    strncpy(out[n].name, names[k].c_str(), sizeof(out[n].name) - 1);
    out[n].ms = ms[k];
    out[n].count = cnt[k];
  }
  if (n_out) *n_out = out ? n : (int)names.size();
  return TSVD_OK;
}

extern "C" unsigned long long tsvd_launch_count(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
