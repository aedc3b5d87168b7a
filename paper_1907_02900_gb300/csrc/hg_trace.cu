// Per-kernel tracing: when enabled, every kernel launch of the library is
// bracketed by CUDA events on its own stream; hg_profile_read() sums the
// elapsed times per kernel name.  Disabled (the default) it costs one branch.
#include <cstring>
#include <mutex>
#include <vector>

#include "hg_trace.h"

namespace hg {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_enabled() { return g_on; }

ProfScope::ProfScope(const char* name, cudaStream_t st) : name_(name), st_(st), a_(nullptr) {
  if (!g_on) return;
  // launches recorded into a CUDA graph are timed as a whole by the caller
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = take_event();
  cudaEventRecord(a_, st_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = take_event();
  cudaEventRecord(b, st_);
  g_recs.push_back(Rec{name_, a_, b});
}

}  // namespace hg

using namespace hg;

extern "C" {

void hg_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
}

void hg_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
}

int hg_profile_read(int max_entries, const char** names, double* total_ms, uint64_t* launches) {
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<const char*> keys;
  std::vector<double> ms;
  std::vector<uint64_t> cnt;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return -1;
    size_t k = 0;
    while (k < keys.size() && std::strcmp(keys[k], r.name) != 0) ++k;
    if (k == keys.size()) {
      keys.push_back(r.name);
      ms.push_back(0.0);
      cnt.push_back(0);
    }
    ms[k] += t;
    cnt[k] += 1;
  }
  const int n = (int)keys.size();
  for (int i = 0; i < n && i < max_entries; ++i) {
    if (names) names[i] = keys[i];
    if (total_ms) total_ms[i] = ms[i];
    if (launches) launches[i] = cnt[i];
  }
  return n;
}

}  // extern "C"
