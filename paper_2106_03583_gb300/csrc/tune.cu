// Schedule autotuning (include/snac.h, snac_autotune): coordinate descent over the multigrid
// schedule options, each candidate timed by complete solves of the caller's right-hand side.
// Host code; the solves are the library's own (snac_plan_create / snac_poisson_solve).
#include <cmath>
#include <vector>

#include "snac_impl.h"

namespace {

snac_options defaults() {
  const snac_plan d;  // the plan's member defaults
  snac_options o{};
  o.precision = d.precision;
  o.nu1 = d.nu1;
  o.nu2 = d.nu2;
  o.max_outer = d.max_outer;
  o.max_cycles = d.max_cycles;
  o.max_coarse = d.max_coarse;
  o.fused = d.fused;
  o.inner_reduction = d.inner_reduction;
  o.shift = d.shift;
  o.bottom_cells = d.bottom_cells;
  return o;
}

bool same(const snac_options& a, const snac_options& b) {
  return a.precision == b.precision && a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.max_outer == b.max_outer &&
         a.max_cycles == b.max_cycles && a.max_coarse == b.max_coarse && a.fused == b.fused &&
         a.inner_reduction == b.inner_reduction && a.shift == b.shift && a.onchip == b.onchip &&
         a.bottom_cells == b.bottom_cells;
}

struct Trial {
  int nblocks;
  const snac_block* blocks;
  int homog;
  const double* d_rhs;
  double* d_p;
  size_t bytes;
  double tol;
  cudaStream_t s;
  cudaEvent_t e0, e1;
};

// Mean time of `reps` solves from p = 0 with options o, after one untimed solve; +inf if the plan
// cannot be built or a solve does not reach tol.
double time_options(const Trial& t, const snac_options& o, int reps) {
  snac_plan* pl = nullptr;
  if (snac_plan_create(&pl, t.nblocks, t.blocks, t.homog, &o) != SNAC_OK) return INFINITY;
  double ms = INFINITY;
  bool ok = cudaMemsetAsync(t.d_p, 0, t.bytes, t.s) == cudaSuccess &&
            snac_poisson_solve(pl, t.d_rhs, t.d_p, t.tol, t.s) == SNAC_OK;
  if (ok) {
    float total = 0.0f;
    for (int r = 0; r < reps && ok; ++r) {
      ok = cudaMemsetAsync(t.d_p, 0, t.bytes, t.s) == cudaSuccess && cudaEventRecord(t.e0, t.s) == cudaSuccess &&
           snac_poisson_solve(pl, t.d_rhs, t.d_p, t.tol, t.s) == SNAC_OK && cudaEventRecord(t.e1, t.s) == cudaSuccess &&
           cudaEventSynchronize(t.e1) == cudaSuccess;
      float one = 0.0f;
      if (ok && cudaEventElapsedTime(&one, t.e0, t.e1) == cudaSuccess) total += one;
    }
    if (ok) ms = total / reps;
  }
  cudaGetLastError();
  snac_plan_destroy(pl);
  return ms;
}

}  // namespace

extern "C" int snac_autotune(int32_t nblocks, const snac_block* blocks, int32_t homog_axis, const snac_options* base,
                             const double* d_rhs, double tol, snac_options* best, snac_tune_report* report,
                             void* stream) {
  if (!blocks || nblocks < 1 || !d_rhs || !best || !(tol > 0.0) || !std::isfinite(tol)) return SNAC_ERR_INVALID_ARG;
  if (base && (base->mode_begin != 0 || base->mode_end != 0)) return SNAC_ERR_INVALID_ARG;  // whole solves only
  int st = snac::check_layout(nblocks, blocks, homog_axis);
  if (st) return st;
  const snac_options b0 = base ? *base : defaults();
  long long n3 = 0;
  for (int b = 0; b < nblocks; ++b) {
    long long c = 1;
    for (int a = 0; a < 3; ++a) c *= blocks[b].hi[a] - blocks[b].lo[a] + 1;
    n3 += c;
  }
  Trial t{nblocks, blocks, homog_axis, d_rhs, nullptr, (size_t)n3 * sizeof(double), tol, (cudaStream_t)stream,
          nullptr, nullptr};
  if (cudaMalloc((void**)&t.d_p, t.bytes) != cudaSuccess) {
    cudaGetLastError();
    return SNAC_ERR_OOM;
  }
  if (cudaEventCreate(&t.e0) != cudaSuccess || cudaEventCreate(&t.e1) != cudaSuccess) {
    cudaGetLastError();
    if (t.e0) cudaEventDestroy(t.e0);
    cudaFree(t.d_p);
    return SNAC_ERR_CUDA;
  }
  const int reps = 2;
  int trials = 1;
  const double base_ms = time_options(t, b0, reps);
  snac_options cur = b0;
  double cur_ms = base_ms;
  auto consider = [&](const snac_options& cand) {
    if (same(cand, cur)) return;
    const double ms = time_options(t, cand, reps);
    ++trials;
    if (ms < cur_ms) {
      cur = cand;
      cur_ms = ms;
    }
  };
  // one pass of coordinate descent, in the order of the largest expected effect
  const int nus[4][2] = {{2, 2}, {2, 1}, {1, 2}, {1, 1}};
  {
    const snac_options start = cur;
    for (const auto& nu : nus) {
      snac_options c = start;
      c.nu1 = nu[0];
      c.nu2 = nu[1];
      consider(c);
    }
  }
  {
    const snac_options start = cur;
    for (int mc : {16, 64, 256}) {
      snac_options c = start;
      c.max_coarse = mc;
      consider(c);
    }
  }
  {
    // where the whole solve of a wavenumber fits in one CTA: on chip (device-side convergence, one
    // launch per step) or level by level (grids over all wavenumbers, host-checked rounds)
    const snac_options start = cur;
    for (int oc : {0, -1}) {
      snac_options c = start;
      c.onchip = oc;
      consider(c);
    }
  }
  {
    // where the coarse levels move into one CTA's shared memory per wavenumber: a smaller top
    // level means more, lighter CTAs for the bottom launch and one more level on the grid-wide path
    const snac_options start = cur;
    for (int bc : {0, 2048, 512}) {
      snac_options c = start;
      c.bottom_cells = bc;
      consider(c);
    }
  }
  if (b0.precision == SNAC_MIXED) {
    const snac_options start = cur;
    for (double eta : {1e-4, 3e-5, 1e-5, 3e-4, 1e-3}) {
      snac_options c = start;
      c.inner_reduction = eta;
      consider(c);
    }
    const snac_options start2 = cur;
    for (int fz : {-1, 0}) {
      snac_options c = start2;
      c.fused = fz;
      consider(c);
    }
  }
  cudaEventDestroy(t.e0);
  cudaEventDestroy(t.e1);
  cudaFree(t.d_p);
  if (!std::isfinite(cur_ms)) return SNAC_ERR_NOT_CONVERGED;  // no candidate reached tol
  *best = cur;
  if (report) *report = snac_tune_report{trials, same(cur, b0) ? 0 : 1, base_ms, cur_ms};
  return SNAC_OK;
}
