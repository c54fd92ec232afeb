// Tracing: per-kernel launch counts, algorithmic bytes/flops and (optionally) CUDA-event durations.
#include <algorithm>

#include "snac_impl.h"

namespace snac {

static const char* const kKernelNames[K_COUNT] = {
    "field3d", "reduce", "fix_mean", "shift", "forward_transform", "backward_update", "smooth",
    "restrict", "prolong", "coarse_solve", "mode_resid", "mode_reduce", "mode_apply", "fused_down", "fused_up",
    "bottom", "field3d_ff", "onchip", "fwd_onchip"};

static cudaEvent_t take_event(snac_plan* P) {
  if (!P->event_pool.empty()) {
    cudaEvent_t e = P->event_pool.back();
    P->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

LaunchScope::LaunchScope(snac_plan* P, int kind, double bytes, double flops, cudaStream_t s)
    : P_(P), kind_(kind), s_(s) {
  KernelStat& k = P->kstats[kind];
  ++k.launches;
  k.bytes += bytes;
  k.flops += flops;
  if (P->profiling) {
    b_ = take_event(P);
    if (b_) cudaEventRecord(b_, s_);
  }
}

LaunchScope::~LaunchScope() {
  if (!b_) return;
  cudaEvent_t e = take_event(P_);
  if (!e) {
    P_->event_pool.push_back(b_);
    return;
  }
  cudaEventRecord(e, s_);
  P_->pending.push_back({kind_, b_, e});
}

void profile_resolve(snac_plan* P) {
  for (const PendingEvent& pe : P->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) P->kstats[pe.kind].ms += ms;
    else cudaGetLastError();
    P->event_pool.push_back(pe.a);
    P->event_pool.push_back(pe.b);
  }
  P->pending.clear();
}

void profile_release(snac_plan* P) {
  for (const PendingEvent& pe : P->pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  P->pending.clear();
  for (cudaEvent_t e : P->event_pool) cudaEventDestroy(e);
  P->event_pool.clear();
}

}  // namespace snac

extern "C" {

int snac_plan_set_profiling(snac_plan* plan, int32_t enable) {
  if (!plan) return SNAC_ERR_INVALID_ARG;
  plan->profiling = enable != 0;
  return SNAC_OK;
}

int snac_plan_kernel_stats(const snac_plan* plan, snac_kernel_stat* h_out, int32_t n, int32_t* count) {
  if (!plan || (n > 0 && !h_out)) return SNAC_ERR_INVALID_ARG;
  if (count) *count = snac::K_COUNT;
  for (int k = 0; k < std::min<int>(n, snac::K_COUNT); ++k) {
    const snac::KernelStat& s = plan->kstats[k];
    h_out[k] = snac_kernel_stat{snac::kKernelNames[k], s.launches, s.ms, s.bytes, s.flops};
  }
  return SNAC_OK;
}

int snac_plan_reset_stats(snac_plan* plan) {
  if (!plan) return SNAC_ERR_INVALID_ARG;
  for (auto& s : plan->kstats) s = snac::KernelStat{};
  return SNAC_OK;
}

}  // extern "C"
