// Kernel-launch tracing scope (see hg_trace.cu).
#pragma once

#include <cuda_runtime.h>

namespace hg {

bool prof_enabled();

// Records a CUDA event on `st` at construction and another at destruction
// when tracing is on; the pair is attributed to `name`.
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  cudaEvent_t a_;
};

}  // namespace hg

#define HG_TRACE_CAT2(a, b) a##b
#define HG_TRACE_CAT(a, b) HG_TRACE_CAT2(a, b)
// Scope guard around one launch: HG_TRACE("k_hist", stream);
#define HG_TRACE(name, st) ::hg::ProfScope HG_TRACE_CAT(hg_trace_scope_, __LINE__)(name, st)
