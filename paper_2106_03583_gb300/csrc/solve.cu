// The solve: Algorithm 1 (Sec. 2) inside an FP64 defect-correction loop, plus the stage entry points.
//
//   repeat:  r = f - A p                     (FP64, 3-D, Eq. 8)         stop when ||r|| <= tol ||f||
//            r_hat = F r                     (Table 1, along z)
//            for every wavenumber q:  V-cycles on (A_xy + lambda_q/dz^2) e_q = r_hat_q   (Eq. 9)
//                                     until its own share of the residual target is met
//            p += F^-1 e_hat                 (FP64 update)
//
// The per-wavenumber stopping rule: with the Parseval weights w_q of the transform
// (||x||^2 = sum_q w_q ||x_hat_q||^2), the 3-D residual after the update is the inverse transform of
// the per-mode residuals, so w_q ||r_q||^2 <= target^2 / n_z for every q gives ||r_new|| <= target.
// Modes with a large |lambda_q| meet it in fewer cycles (Sec. 3.3 and App. B); each cycle only runs
// the modes still active. A mode whose residual stops falling (the floating-point floor of the inner
// precision) is retired as well; the outer loop then takes another defect-correction step.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "snac_impl.h"

namespace snac {
void set_error(const std::string& s);
}

namespace {
using namespace snac;

int cuda_fail(cudaError_t e, const char* where) {
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  return SNAC_ERR_CUDA;
}

#define CK(call)                                   \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int check_plan(snac_plan* P) {
  if (!P) return SNAC_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device) {
    set_error("the current CUDA device is not the plan's device");
    return SNAC_ERR_INVALID_ARG;
  }
  return SNAC_OK;
}

// Calls on 3-D fields: not on a wavenumber-range plan, which holds a slab of the mode space only.
int check_plan3d(snac_plan* P) {
  int st = check_plan(P);
  if (st) return st;
  if (P->ranged) {
    set_error("a wavenumber-range plan has no 3-D field: use the pencil calls");
    return SNAC_ERR_INVALID_ARG;
  }
  return SNAC_OK;
}

int set_active_all(snac_plan* P, cudaStream_t s) {
  for (int q = 0; q < P->nz; ++q) P->h_active[q] = q;
  CK(launch_from_host(P->dh_active, P->d_active, P->nz, s));
  return SNAC_OK;
}

// V-cycles of every mode until its share of `target` is met, it stagnates, or max_cycles.
// One V-cycle round of the active modes and their norms. Without profiling the round is replayed from
// a CUDA graph captured (on the plan's private stream) the first time this number of modes is active;
// the graph's kernels read the active list from device memory, which the caller updates before.
// skip_first0: the cycle's first colour-0 half-sweep at level 0 was done by the last norm check.
cudaError_t run_round(snac_plan* P, int nact, bool norms, cudaStream_t s, int* replayed, bool skip_first0) {
  if (!P->graphs || P->profiling) {
    cudaError_t e = launch_vcycle(P, nact, s, skip_first0);
    return e != cudaSuccess || !norms ? e : launch_mode_norms(P, nact, true, s);
  }
  const int key = 2 * nact + (skip_first0 ? 1 : 0);
  auto it = P->round_graphs.find(key);
  if (it == P->round_graphs.end()) {
    snac_plan::RoundGraph rg;
    KernelStat before[K_COUNT];
    for (int k = 0; k < K_COUNT; ++k) before[k] = P->kstats[k];
    cudaError_t e = cudaSuccess;
    if (!P->capture_stream) e = cudaStreamCreateWithFlags(&P->capture_stream, cudaStreamNonBlocking);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(P->capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t el = launch_vcycle(P, nact, P->capture_stream, skip_first0);
      if (el == cudaSuccess && norms) el = launch_mode_norms(P, nact, true, P->capture_stream);
      e = cudaStreamEndCapture(P->capture_stream, &g);
      if (el != cudaSuccess) e = el;
    }
    for (int k = 0; k < K_COUNT; ++k) {  // counted once at capture; added again at every replay
      rg.delta[k].launches = P->kstats[k].launches - before[k].launches;
      rg.delta[k].bytes = P->kstats[k].bytes - before[k].bytes;
      rg.delta[k].flops = P->kstats[k].flops - before[k].flops;
      P->kstats[k] = before[k];
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&rg.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {  // capture not possible here: launch the kernels directly from now on
      cudaGetLastError();
      P->graphs = false;
      return run_round(P, nact, norms, s, replayed, skip_first0);
    }
    it = P->round_graphs.emplace(key, rg).first;
  }
  for (int k = 0; k < K_COUNT; ++k) {
    P->kstats[k].launches += it->second.delta[k].launches;
    P->kstats[k].bytes += it->second.delta[k].bytes;
    P->kstats[k].flops += it->second.delta[k].flops;
  }
  ++*replayed;
  return cudaGraphLaunch(it->second.exec, s);
}

// The on-chip path's results: per-mode cycles and final norms from the mapped host arrays.
int onchip_results(snac_plan* P, int* cycles_out) {
  int total = 0;
  for (int q = 0; q < P->nz; ++q) {
    cycles_out[q] = P->h_cycles[q];
    total += cycles_out[q];
    if (!std::isfinite(P->h_mode_norm2[q])) return SNAC_ERR_NONFINITE;
  }
  P->info.total_cycles += total;
  return SNAC_OK;
}

// The level-by-level wavenumber solves of one plan as a state machine, so that several plans can
// run them in lock-step: each round's launches of all of them go out together and one stream
// synchronisation serves every plan that reads norms back in that round. A single plan is a set of
// one (the same launches and synchronisations as a dedicated loop).
struct ModeRun {
  snac_plan* P = nullptr;
  cudaStream_t s = nullptr;  // the stream of this plan's launches
  double target = 0.0;
  int* cycles = nullptr;
  int st = SNAC_OK;
  bool done = false;
  // state between rounds
  std::vector<double> thr2, prev;  // prev: norm^2 at the mode's last check
  std::vector<int> list, prev_cycle, next_check;
  std::vector<char> checked;
  bool predictive = false, sweep_checks = false, red_done = false, list_changed = true, pending = false;
  int c = 0, total = 0;

  int fail(int status) {
    st = status;
    done = true;
    return status;
  }

  // norms of the zero iterate (the right-hand side), which the same pass sets to zero
  int begin(cudaStream_t s) {
    if (set_active_all(P, s)) return fail(SNAC_ERR_CUDA);
    cudaError_t e = launch_mode_norms(P, P->nz, false, s, nullptr, true);
    if (e == cudaSuccess) e = launch_to_host(P->d_mode_norm2, P->dh_mode_norm2, P->nz, s);
    return e == cudaSuccess ? SNAC_OK : fail(cuda_fail(e, "mode norms"));
  }

  // after a synchronisation
  void begin_read() {
    profile_resolve(P);
    const int nz = P->nz;
    thr2.assign(nz, 0.0);
    prev.assign(nz, 0.0);
    prev_cycle.assign(nz, 0);
    next_check.assign(nz, 1);
    checked.assign(nz, 0);
    list.clear();
    for (int q = 0; q < nz; ++q) {
      thr2[q] = target * target / (P->nzt * P->pweight[q]);
      prev[q] = P->h_mode_norm2[q];
      cycles[q] = 0;
      if (!std::isfinite(prev[q])) {
        fail(SNAC_ERR_NONFINITE);
        return;
      }
      if (prev[q] > thr2[q]) list.push_back(q);
    }
    // Where the level-0 norms need a pass of their own (the fused up kernel gives them for free), a
    // mode is checked only when its observed per-cycle reduction says it should have reached its
    // share, at most 3 cycles after its last check; rounds without a check need no synchronisation.
    // A mode stops only at a check, so at worst it runs one cycle more than needed.
    predictive = !P->lev[0].fused;
    // scaled FP64 plans take the norms of a check from the next cycle's first colour-0 half-sweep at
    // level 0 (done for every active mode), so the check costs no pass of its own
    sweep_checks = predictive && P->scaled_f && P->nu1 >= 1;
    done = list.empty();
  }

  // One V-cycle round of the active modes and, if some mode is due a check, its norms on their way
  // to the host (pending: read them after the next synchronisation).
  int round(cudaStream_t s) {
    pending = false;
    if (done) return SNAC_OK;
    if (c >= P->max_cycles || list.empty()) {
      done = true;
      return SNAC_OK;
    }
    const int nact = (int)list.size();
    cudaError_t e = cudaSuccess;
    if (list_changed) {  // the previous upload has completed: every list change follows a synchronisation
      std::copy(list.begin(), list.end(), P->h_active);
      e = launch_from_host(P->dh_active, P->d_active, nact, s);
      list_changed = false;
    }
    if (e == cudaSuccess) e = run_round(P, nact, !predictive, s, &P->info.graph_rounds, red_done);
    if (e != cudaSuccess) return fail(cuda_fail(e, "V-cycle round"));
    red_done = false;
    ++c;
    int ncheck = 0;
    for (int q : list) {
      ++cycles[q];
      ++total;
      checked[q] = !predictive || cycles[q] >= next_check[q];
      if (checked[q]) P->h_check[ncheck++] = q;
    }
    if (ncheck == 0) return SNAC_OK;
    if (predictive) {
      e = launch_from_host(P->dh_check, P->d_check, ncheck, s);
      if (e == cudaSuccess) {
        if (sweep_checks) {
          e = launch_check_sweep(P, nact, ncheck, s);
          red_done = true;  // for every mode that stays active
        } else {
          e = launch_mode_norms(P, ncheck, true, s, P->d_check);
        }
      }
    }
    if (e == cudaSuccess) e = launch_to_host(P->d_mode_norm2, P->dh_mode_norm2, P->nz, s);
    if (e != cudaSuccess) return fail(cuda_fail(e, "mode norms"));
    pending = true;
    return SNAC_OK;
  }

  // after a synchronisation, when a round left norms pending
  void read() {
    if (!pending || done) return;
    pending = false;
    profile_resolve(P);
    const double stag2 = 0.6 * 0.6;  // a cycle that reduces the norm less than 0.6x: the precision floor
    std::vector<int> next;
    for (int q : list) {
      if (!checked[q]) {
        next.push_back(q);
        continue;
      }
      const double r2 = P->h_mode_norm2[q];
      if (!std::isfinite(r2)) {
        fail(SNAC_ERR_NONFINITE);
        return;
      }
      const int dc = cycles[q] - prev_cycle[q];
      const bool ok = r2 <= thr2[q] || r2 > std::pow(stag2, dc) * prev[q];
      if (!ok && predictive) {
        const double rho2 = std::pow(r2 / prev[q], 1.0 / dc);  // per-cycle factor of the norm^2, < 1
        const double need = std::log(thr2[q] / r2) / std::log(rho2);
        next_check[q] = cycles[q] + std::max(1, std::min(3, (int)std::ceil(need - 0.25)));
      }
      prev[q] = r2;
      prev_cycle[q] = cycles[q];
      if (!ok) next.push_back(q);
    }
    list_changed = next.size() != list.size();
    list.swap(next);
  }

  void finish() { P->info.total_cycles += total; }
};

// V-cycles of every mode of every plan until its share of the plan's target is met, it stagnates,
// or max_cycles; the plans in lock-step, each on its own stream (r->s). `wait` makes the host wait
// for every stream the runs use. Each run's status in its st.
template <typename Wait>
void mode_solves_many(const std::vector<ModeRun*>& runs, Wait&& wait) {
  auto sync = [&]() -> bool {
    const cudaError_t e = wait();
    if (e == cudaSuccess) return true;
    const int st = cuda_fail(e, "cudaStreamSynchronize");
    for (ModeRun* r : runs)
      if (!r->done) r->fail(st);
    return false;
  };
  for (ModeRun* r : runs) r->begin(r->s);
  if (!sync()) return;
  for (ModeRun* r : runs)
    if (!r->done) r->begin_read();
  for (;;) {
    bool active = false, pending = false;
    for (ModeRun* r : runs) {
      r->round(r->s);
      active = active || !r->done;
      pending = pending || r->pending;
    }
    if (!active) break;
    if (!pending) continue;
    if (!sync()) return;
    for (ModeRun* r : runs) r->read();
  }
  for (ModeRun* r : runs)
    if (r->st == SNAC_OK) r->finish();
}

int mode_solves(snac_plan* P, double target, cudaStream_t s, int* cycles_out) {
  if (P->onchip) {  // every wavenumber's whole solve in one CTA; convergence decided on the device
    const int st = set_active_all(P, s);
    if (st) return st;
    CK(launch_onchip(P, P->nz, target, s));
    CK(cudaStreamSynchronize(s));
    profile_resolve(P);
    return onchip_results(P, cycles_out);
  }
  ModeRun r;
  r.P = P;
  r.s = s;
  r.target = target;
  r.cycles = cycles_out;
  mode_solves_many({&r}, [&] { return cudaStreamSynchronize(s); });
  return r.st;
}

int read_sums(snac_plan* P, cudaStream_t s, int n = 4) {
  CK(launch_to_host(P->d_sums, P->dh_sums, n, s));
  CK(cudaStreamSynchronize(s));
    profile_resolve(P);
  return SNAC_OK;
}

// One problem's solve as a sequence of steps, so that several problems can run in lock-step: their
// launches of one phase go out together, one stream synchronisation serves all of them, and the
// on-chip wavenumber solves of all of them share one persistent launch. A single solve is a batch of
// one (the same steps, the same synchronisations as a dedicated loop would have).
struct Job {
  snac_plan* P = nullptr;
  const double* f = nullptr;
  double* p = nullptr;
  double tol = 0.0;
  int st = SNAC_OK;
  bool finished = false;
  bool p_zero = false, updated = false, aim_final = false, r32 = false, ff = false, redo = false;
  bool fused = false;  // this step's forward transform runs inside the on-chip launch
  FusedInput fin{};
  double fshift = 0.0, fn = 0.0, fn_pre = 0.0, prev_rel = INFINITY, rn = 0.0, target = 0.0;
  int k = 0;
  std::vector<int> cyc;
  void finish(int status) {
    st = status;
    finished = true;
    P->info.status = status;
  }
};

// Mixed plans compute the residual of an intermediate defect-correction step in float-float
// arithmetic (written in FP32, the precision the FP32 transform reads); the FP64 pass decides
// convergence: it runs after a correction that aimed at the tolerance itself, and whenever the
// float-float residual comes within 2x of the tolerance. (The float-float error, a few units of
// 2^-47 of |f| + |A||p| per cell, is about 1e-11 ||f|| on the 2.7e8-cell channel: it steers an
// intermediate correction well enough, but a convergence decision near tol takes the FP64 pass.)

// pre-pass: statistics of f, and whether the initial guess is zero (then r = f - fshift at k = 0
// and the first residual pass is not needed)
cudaError_t job_begin(Job& J, cudaStream_t s) {
  snac_plan* P = J.P;
  P->info = snac_solve_info{};
  P->info.levels = (int)P->lev.size();
  P->info.n_modes = P->nz;
  std::fill(P->mode_cycles.begin(), P->mode_cycles.end(), 0);
  J.cyc.assign(P->nz, 0);
  cudaError_t e = launch_prepass(P, J.f, J.p, s);
  if (e == cudaSuccess) e = launch_to_host(P->d_sums, P->dh_sums, SUM_NONZERO + 1, s);
  return e;
}

void job_begin_read(Job& J) {
  snac_plan* P = J.P;
  profile_resolve(P);
  J.p_zero = P->h_sums[SUM_NONZERO] == 0.0;
  const double f2 = P->h_sums[2], sum_f = P->h_sums[3];
  if (!std::isfinite(f2)) return J.finish(SNAC_ERR_NONFINITE);
  if (P->singular) {
    const double vf = P->h_sums[0], vaf = P->h_sums[1];
    if (!std::isfinite(vf) || !std::isfinite(vaf)) return J.finish(SNAC_ERR_NONFINITE);
    if (std::fabs(vf) > 1e-12 * vaf) {
      set_error("singular problem: the volume-weighted sum of the right-hand side is not zero");
      return J.finish(SNAC_ERR_INCOMPATIBLE_RHS);
    }
    J.fshift = vf / P->vol_total;
    P->info.removed_mean = J.fshift;
  }
  // ||f - fshift||^2 = ||f||^2 - fshift (2 sum f - N fshift)
  J.fn_pre = std::sqrt(std::max(0.0, f2 - J.fshift * (2.0 * sum_f - (double)P->n3 * J.fshift)));
}

// The residual pass of step k (none for k = 0 from a zero guess): launched, read after a sync.
cudaError_t job_resid_launch(Job& J, cudaStream_t s) {
  snac_plan* P = J.P;
  J.r32 = J.ff = J.redo = false;
  if (J.k == 0 && J.p_zero) {
    J.fn = J.rn = J.fn_pre;
    return P->singular ? launch_fill(P->d_sums + 2, 1, 0.0, s) : cudaSuccess;  // sum V p = 0
  }
  // ||f|| is needed once; sum V p only for singular problems (zero-mean update). In FP64 plans
  // only for the caller's initial guess: an update leaves sum V p = 0 to rounding (the mean fix
  // solves for it), so later passes take it as 0 (their partials carry 0 in that slot). Mixed
  // plans measure it every time: the FP32 transform of the correction leaves a drift that the
  // next mean fix removes.
  const bool need_vp = P->singular && (J.k == 0 || P->precision != SNAC_FP64);
  cudaError_t e;
  if (P->precision == SNAC_MIXED && J.k > 0 && !J.aim_final) {
    J.ff = true;
    e = launch_field3d_ff(P, J.f, J.p, reinterpret_cast<float*>(P->d_r3), J.fshift, J.fn / std::sqrt((double)P->n3),
                          false, need_vp, s);
  } else {
    e = launch_field3d(P, 0, J.f, J.p, P->d_r3, J.fshift, J.k == 0, need_vp, s);
  }
  if (e == cudaSuccess) e = launch_to_host(P->d_sums, P->dh_sums, 4, s);
  return e;
}

// After the sync: read the pass. A float-float pass within 2x of the tolerance launches the FP64
// pass instead (J.redo: read again after another sync).
cudaError_t job_resid_read(Job& J, cudaStream_t s) {
  snac_plan* P = J.P;
  profile_resolve(P);
  if (J.k == 0 && J.p_zero) return cudaSuccess;
  if (J.ff && !J.redo) {
    J.rn = std::sqrt(P->h_sums[0]);
    J.r32 = !(J.rn <= 2.0 * J.tol * J.fn);  // (NaN stays: reported by the decision)
    if (J.r32) return cudaSuccess;
    J.redo = true;
    const bool need_vp = P->singular;
    cudaError_t e = launch_field3d(P, 0, J.f, J.p, P->d_r3, J.fshift, false, need_vp, s);
    if (e == cudaSuccess) e = launch_to_host(P->d_sums, P->dh_sums, 4, s);
    return e;
  }
  if (J.k == 0) J.fn = std::sqrt(P->h_sums[1]);
  J.rn = std::sqrt(P->h_sums[0]);
  J.redo = false;
  return cudaSuccess;
}

// Convergence decision of step k; on continuing, the forward transform of the residual.
int job_decide(Job& J, cudaStream_t s) {
  snac_plan* P = J.P;
  int st;
  const double rn = J.rn, fn = J.fn;
  if (!std::isfinite(rn) || !std::isfinite(fn)) {
    J.finish(SNAC_ERR_NONFINITE);
    return SNAC_OK;
  }
  P->info.rhs_norm = fn;
  P->info.outer_iters = J.k;
  if (fn == 0.0) {  // zero right-hand side: p = 0
    CK(cudaMemsetAsync(J.p, 0, (size_t)P->n3 * sizeof(double), s));
    CK(cudaStreamSynchronize(s));
    profile_resolve(P);
    P->info.rel_res = 0.0;
    J.finish(SNAC_OK);
    return SNAC_OK;
  }
  const double rel = rn / fn;
  P->info.rel_res = rel;
  const bool done = rel <= J.tol;
  // a correction that did not lower the residual: the inner solve has reached the floating-point
  // floor of the outer residual (or diverged); more steps would not help
  const bool stalled = J.updated && rel >= J.prev_rel;
  const bool give_up = !done && (J.k >= P->max_outer || stalled);
  if (done || give_up) {
    if (P->singular && !J.updated) {  // the initial guess was kept: return its zero-mean shift
      CK(launch_shift(P, J.p, P->d_sums + 3, s));
      CK(cudaStreamSynchronize(s));
      profile_resolve(P);
    }
    if (stalled) {
      // return the better iterate: take the last correction back (its modes are still in the
      // level-0 iterate) and report the residual of what is returned, re-evaluated
      CK(launch_backward_update(P, P->lev[0].d_u, J.p, s, true));
      CK(launch_field3d(P, 0, J.f, J.p, P->d_r3, J.fshift, false, false, s));
      if ((st = read_sums(P, s))) return st;
      P->info.rel_res = std::sqrt(P->h_sums[0]) / fn;
    }
    J.finish(done ? SNAC_OK : SNAC_ERR_NOT_CONVERGED);
    return SNAC_OK;
  }
  J.prev_rel = rel;
  // target of this defect-correction step: the tolerance (with a factor 2 of margin); in mixed
  // plans a reduction by inner_reduction while that is still above the tolerance -- once it is not,
  // the step aims at the tolerance itself (an FP32 solve reaches it from there), which saves a step
  J.target = 0.5 * J.tol * fn;
  if (P->precision == SNAC_MIXED && P->inner_reduction * rn > J.tol * fn) J.target = P->inner_reduction * rn;
  J.aim_final = J.target <= 0.5 * J.tol * fn;
  J.fused = fused_ready(P);
  if (J.fused) {  // the forward transform goes into the same launch as the wavenumber solves
    if (J.k == 0 && J.p_zero) J.fin = FusedInput{J.f, false, J.fshift};
    else J.fin = FusedInput{P->d_r3, J.r32, 0.0};
    return SNAC_OK;
  }
  if (J.k == 0 && J.p_zero) CK(launch_forward(P, J.f, P->lev[0].d_f, J.fshift, P->scaled_f, s));
  else if (J.r32) CK(launch_forward_f32(P, reinterpret_cast<const float*>(P->d_r3), P->lev[0].d_f, s));
  else CK(launch_forward(P, P->d_r3, P->lev[0].d_f, 0.0, P->scaled_f, s));
  return SNAC_OK;
}

// After the wavenumber solves: record their cycles, fix the mean, update p.
cudaError_t job_update(Job& J, cudaStream_t s) {
  snac_plan* P = J.P;
  for (int q = 0; q < P->nz; ++q) {
    P->mode_cycles[q] = J.cyc[q];
    P->info.max_mode_cycles = std::max(P->info.max_mode_cycles, J.cyc[q]);
  }
  cudaError_t e = cudaSuccess;
  if (P->singular) e = launch_fix_mean(P, P->lev[0].d_u, s);
  if (e == cudaSuccess) e = launch_backward_update(P, P->lev[0].d_u, J.p, s);
  J.updated = true;
  ++J.k;
  return e;
}

int job_cuda(Job& J, cudaError_t e, const char* where) {
  if (e != cudaSuccess) J.finish(cuda_fail(e, where));
  return J.st;
}

// Run the jobs to completion on stream s (all plans on the current device).
// Several problems at once: each problem's own launches go to one of a few side streams, forked
// from the caller's stream at the start and joined back into it before every synchronisation and
// before a launch on the caller's stream that reads their results, so that the kernels of
// different problems can run at the same time. Without side streams everything runs on `main`.
struct SideStreams {
  cudaStream_t main;
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev;  // one per side stream, then the fork event
  SideStreams(cudaStream_t s, int n) : main(s) {
    for (int k = 0; k < n; ++k) {
      cudaStream_t t = nullptr;
      cudaEvent_t e = nullptr;
      if (cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (t) cudaStreamDestroy(t);
        break;
      }
      side.push_back(t);
      ev.push_back(e);
    }
    cudaEvent_t f = nullptr;
    if (!side.empty() && cudaEventCreateWithFlags(&f, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release();
    }
    if (f) ev.push_back(f);
  }
  ~SideStreams() { release(); }
  void release() {
    for (cudaStream_t t : side) cudaStreamDestroy(t);
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    side.clear();
    ev.clear();
  }
  cudaStream_t of(size_t k) const { return side.empty() ? main : side[k % side.size()]; }
  cudaError_t fork() {
    if (side.empty()) return cudaSuccess;
    cudaError_t e = cudaEventRecord(ev.back(), main);
    for (size_t k = 0; k < side.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(side[k], ev.back(), 0);
    return e;
  }
  cudaError_t join() {
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < side.size() && e == cudaSuccess; ++k) {
      e = cudaEventRecord(ev[k], side[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(main, ev[k], 0);
    }
    return e;
  }
};

int run_jobs(std::vector<Job>& jobs, cudaStream_t s) {
  SideStreams ss(s, jobs.size() > 1 ? (int)std::min<size_t>(16, jobs.size()) : 0);
  auto js = [&](const Job& J) { return ss.of((size_t)(&J - jobs.data())); };
  auto sync = [&]() -> cudaError_t {
    const cudaError_t e = ss.join();
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);
  };
  cudaError_t e = ss.fork();  // the caller's earlier work on s (f, p) comes first
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamWaitEvent");
  for (Job& J : jobs) job_cuda(J, job_begin(J, js(J)), "pre-pass");
  e = sync();
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
  for (Job& J : jobs)
    if (!J.finished) job_begin_read(J);
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  int sms = jobs.empty() ? 152 : jobs[0].P->sms;
  int status = SNAC_OK;
  for (;;) {
    bool any = false;
    for (Job& J : jobs) any = any || !J.finished;
    if (!any) break;
    for (Job& J : jobs)
      if (!J.finished) job_cuda(J, job_resid_launch(J, js(J)), "residual");
    if ((e = sync()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamSynchronize"); break; }
    bool redo = false;
    for (Job& J : jobs)
      if (!J.finished && job_cuda(J, job_resid_read(J, js(J)), "residual") == SNAC_OK) redo = redo || J.redo;
    if (redo) {
      if ((e = sync()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamSynchronize"); break; }
      for (Job& J : jobs)
        if (!J.finished && J.redo) job_cuda(J, job_resid_read(J, js(J)), "residual");
    }
    for (Job& J : jobs)
      if (!J.finished) {
        const int st = job_decide(J, js(J));
        if (st) J.finish(st);
      }
    // the forward transforms of the on-chip plans come before their solves on s
    if ((e = ss.join()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamWaitEvent"); break; }
    // the wavenumber solves: on-chip plans together (one persistent launch per precision), the
    // others level by level
    std::vector<Job*> chip[2], fusedj[2];
    for (Job& J : jobs)
      if (!J.finished && J.P->onchip) (J.fused ? fusedj : chip)[J.P->precision == SNAC_FP64 ? 0 : 1].push_back(&J);
    // forward transform + on-chip solves in one persistent launch per precision (bounded waits)
    for (int g = 0; g < 2; ++g) {
      if (fusedj[g].empty()) continue;
      if (fusedj[g].size() == 1) {
        Job& J = *fusedj[g][0];
        job_cuda(J, launch_fwd_onchip(J.P, J.fin.in3, J.fin.in_f32, J.fin.shift0, J.target, WAIT_LIMIT_S, 0, s),
                 "forward transform and on-chip wavenumber solves");
        continue;
      }
      std::vector<snac_plan*> plans;
      std::vector<FusedInput> ins;
      std::vector<double> targets;
      int nitems = 0;
      for (Job* J : fusedj[g]) {
        plans.push_back(J->P);
        ins.push_back(J->fin);
        targets.push_back(J->target);
        nitems += J->P->nz + (int)(J->P->precision == SNAC_FP64 ? J->P->chunks64.size() : J->P->chunks32.size());
      }
      const size_t need = fwd_onchip_batch_scratch((int)plans.size(), nitems);
      if (need > scratch_bytes) {
        if (scratch) cudaFreeAsync(scratch, s);
        scratch = nullptr;
        scratch_bytes = 0;
        if ((e = cudaMallocAsync(&scratch, need, s)) != cudaSuccess) { status = cuda_fail(e, "cudaMallocAsync"); break; }
        scratch_bytes = need;
      }
      e = launch_fwd_onchip_batch(plans.data(), ins.data(), targets.data(), (int)plans.size(), WAIT_LIMIT_S, scratch,
                                  sms, s);
      if (e != cudaSuccess)
        for (Job* J : fusedj[g]) job_cuda(*J, e, "forward transform and on-chip wavenumber solves");
      // the next group reuses the scratch only after this launch has read it
      if (g == 0 && !fusedj[1].empty() && (e = sync()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamSynchronize"); break; }
    }
    if (status) break;
    for (int g = 0; g < 2; ++g) {
      if (chip[g].empty()) continue;
      if (chip[g].size() == 1) {
        Job& J = *chip[g][0];
        job_cuda(J, set_active_all(J.P, s) == SNAC_OK ? launch_onchip(J.P, J.P->nz, J.target, s) : cudaErrorUnknown,
                 "on-chip wavenumber solves");
        continue;
      }
      std::vector<snac_plan*> plans;
      std::vector<double> targets;
      std::vector<int2> items;
      for (Job* J : chip[g]) {
        const int idx = (int)plans.size();
        plans.push_back(J->P);
        targets.push_back(J->target);
        for (int q = 0; q < J->P->nz; ++q) items.push_back(make_int2(idx, q));
      }
      const size_t need = onchip_batch_scratch((int)plans.size(), (int)items.size());
      if (need > scratch_bytes || !fusedj[0].empty() || !fusedj[1].empty()) {
        if (scratch && (e = sync()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamSynchronize"); break; }
        if (scratch) cudaFreeAsync(scratch, s);
        scratch = nullptr;
        scratch_bytes = 0;
        if ((e = cudaMallocAsync(&scratch, need, s)) != cudaSuccess) { status = cuda_fail(e, "cudaMallocAsync"); break; }
        scratch_bytes = need;
      }
      e = launch_onchip_batch(plans.data(), targets.data(), (int)plans.size(), items.data(), (int)items.size(), scratch,
                              sms, s);
      if (e != cudaSuccess)
        for (Job* J : chip[g]) job_cuda(*J, e, "on-chip wavenumber solves");
    }
    if (status) break;
    {  // the level-by-level plans' wavenumber solves, in lock-step with one another
      std::vector<ModeRun> runs;
      std::vector<Job*> owners;
      for (Job& J : jobs)
        if (!J.finished && !J.P->onchip) {
          ModeRun r;
          r.P = J.P;
          r.s = js(J);
          r.target = J.target;
          r.cycles = J.cyc.data();
          runs.push_back(std::move(r));
          owners.push_back(&J);
        }
      if (!runs.empty()) {
        std::vector<ModeRun*> ptrs;
        for (ModeRun& r : runs) ptrs.push_back(&r);
        mode_solves_many(ptrs, sync);
        for (size_t k = 0; k < runs.size(); ++k)
          if (runs[k].st) owners[k]->finish(runs[k].st);
      }
    }
    if (!chip[0].empty() || !chip[1].empty() || !fusedj[0].empty() || !fusedj[1].empty()) {
      if ((e = sync()) != cudaSuccess) { status = cuda_fail(e, "cudaStreamSynchronize"); break; }
      for (int g = 0; g < 2; ++g) {
        for (Job* J : chip[g])
          if (!J->finished) {
            profile_resolve(J->P);
            const int st = onchip_results(J->P, J->cyc.data());
            if (st) J->finish(st);
          }
        for (Job* J : fusedj[g])
          if (!J->finished) {
            profile_resolve(J->P);
            if (*J->P->h_wait) {
              set_error("a device-side wait gave up (transform chunks not counted within the limit)");
              J->finish(SNAC_ERR_TIMEOUT);
              continue;
            }
            const int st = onchip_results(J->P, J->cyc.data());
            if (st) J->finish(st);
          }
      }
    }
    for (Job& J : jobs)
      if (!J.finished) job_cuda(J, job_update(J, js(J)), "update");
  }
  if (scratch) cudaFreeAsync(scratch, s);
  const cudaError_t ef = sync();  // every problem's last launches are complete on return
  if (ef != cudaSuccess && status == SNAC_OK) status = cuda_fail(ef, "cudaStreamSynchronize");
  return status;
}

int run_solve(snac_plan* P, const double* f, double* p, double tol, cudaStream_t s) {
  std::vector<Job> jobs(1);
  jobs[0].P = P;
  jobs[0].f = f;
  jobs[0].p = p;
  jobs[0].tol = tol;
  const int st = run_jobs(jobs, s);
  return st ? st : jobs[0].st;
}

}  // namespace

extern "C" {

int snac_poisson_solve(snac_plan* plan, const double* d_rhs, double* d_p, double tol, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_rhs || !d_p || !(tol > 0.0) || !std::isfinite(tol)) return SNAC_ERR_INVALID_ARG;
  st = run_solve(plan, d_rhs, d_p, tol, (cudaStream_t)stream);
  plan->info.status = st;
  return st;
}

int snac_poisson_solve_batch(int32_t n, snac_plan* const* plans, const double* const* d_rhs, double* const* d_p,
                             double tol, int32_t* h_status, void* stream) {
  if (n < 1 || !plans || !d_rhs || !d_p || !h_status || !(tol > 0.0) || !std::isfinite(tol)) return SNAC_ERR_INVALID_ARG;
  std::vector<Job> jobs(n);
  for (int k = 0; k < n; ++k) {
    int st = check_plan3d(plans[k]);
    if (st) return st;
    if (!d_rhs[k] || !d_p[k]) return SNAC_ERR_INVALID_ARG;
    for (int j = 0; j < k; ++j)
      if (plans[j] == plans[k]) {
        set_error("a plan appears twice in one batch");
        return SNAC_ERR_INVALID_ARG;
      }
    jobs[k].P = plans[k];
    jobs[k].f = d_rhs[k];
    jobs[k].p = d_p[k];
    jobs[k].tol = tol;
  }
  const int st = run_jobs(jobs, (cudaStream_t)stream);
  int worst = st;
  for (int k = 0; k < n; ++k) {
    h_status[k] = st ? st : jobs[k].st;
    plans[k]->info.status = h_status[k];
    if (!worst && h_status[k]) worst = h_status[k];
  }
  return worst;
}

int snac_test_wait_timeout(snac_plan* plan, double wait_seconds, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!fused_ready(plan) || !(wait_seconds > 0.0) || wait_seconds > WAIT_LIMIT_S) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  // the wavenumber solves wait for one transform chunk more than the launch has: nothing ever
  // completes the count, every wait runs out and the launch must come back with the status set
  CK(launch_fwd_onchip(plan, plan->d_r3, false, 0.0, 1.0, wait_seconds, 1, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return *plan->h_wait ? SNAC_ERR_TIMEOUT : SNAC_OK;
}

int snac_apply_operator(snac_plan* plan, const double* d_p, double* d_out, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_p || !d_out) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_field3d(plan, 1, nullptr, d_p, d_out, 0.0, false, false, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_residual(snac_plan* plan, const double* d_rhs, const double* d_p, double* d_r, double* h_norms, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_rhs || !d_p || !d_r || !h_norms) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_field3d(plan, 0, d_rhs, d_p, d_r, 0.0, true, false, s));
  if ((st = read_sums(plan, s))) return st;
  h_norms[0] = plan->h_sums[0];
  h_norms[1] = plan->h_sums[1];
  return SNAC_OK;
}

int snac_residual_ff(snac_plan* plan, const double* d_rhs, const double* d_p, float* d_r, double* h_norms,
                     void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_rhs || !d_p || !d_r || !h_norms) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_field3d_ff(plan, d_rhs, d_p, d_r, 0.0, 1.0, true, false, s));
  if ((st = read_sums(plan, s))) return st;
  h_norms[0] = plan->h_sums[0];
  h_norms[1] = plan->h_sums[1];
  return SNAC_OK;
}

int snac_forward_transform(snac_plan* plan, const double* d_in, void* d_modes, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_in || !d_modes) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_forward(plan, d_in, d_modes, 0.0, false, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_backward_update(snac_plan* plan, const void* d_modes, double* d_p, void* stream) {
  int st = check_plan3d(plan);
  if (st) return st;
  if (!d_modes || !d_p) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_backward_update(plan, d_modes, d_p, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_mode_solve(snac_plan* plan, const void* d_rhs, void* d_sol, double target, void* stream) {
  int st = check_plan(plan);
  if (st) return st;
  if (!d_rhs || !d_sol || !(target >= 0.0) || !std::isfinite(target)) return SNAC_ERR_INVALID_ARG;
  snac_plan* P = plan;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)P->nz * P->lev[0].ncell * plan_inner_size(P);
  // the right-hand side into the level-0 buffer, in the order the cycles read it
  if (P->scaled_f) CK(launch_to_split(P, (const double*)d_rhs, (double*)P->lev[0].d_f, s));
  else CK(cudaMemcpyAsync(P->lev[0].d_f, d_rhs, bytes, cudaMemcpyDeviceToDevice, s));
  P->info = snac_solve_info{};
  P->info.levels = (int)P->lev.size();
  P->info.n_modes = P->nz;
  std::vector<int> cyc(P->nz);
  if ((st = mode_solves(P, target, s, cyc.data()))) {
    P->info.status = st;
    return st;
  }
  for (int q = 0; q < P->nz; ++q) {
    P->mode_cycles[q] = cyc[q];
    P->info.max_mode_cycles = std::max(P->info.max_mode_cycles, cyc[q]);
  }
  CK(cudaMemcpyAsync(d_sol, P->lev[0].d_u, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(P);
  return SNAC_OK;
}

int snac_mode_fix_mean(snac_plan* plan, void* d_sol, double sum_vp, void* stream) {
  int st = check_plan(plan);
  if (st) return st;
  if (!d_sol || !std::isfinite(sum_vp)) return SNAC_ERR_INVALID_ARG;
  if (!plan->singular || plan->q0 != 0) return SNAC_OK;
  cudaStream_t s = (cudaStream_t)stream;
  CK(launch_fill(plan->d_sums + 2, 1, sum_vp, s));  // sum V p of the current p (all ranks)
  CK(launch_fix_mean(plan, d_sol, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_mode_operator(snac_plan* plan, const void* d_u, void* d_out, void* stream) {
  int st = check_plan(plan);
  if (st) return st;
  if (!d_u || !d_out) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = set_active_all(plan, s))) return st;
  CK(launch_mode_operator(plan, d_u, d_out, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

int snac_mode_vcycles(snac_plan* plan, const void* d_f, void* d_u, int32_t ncycles, void* stream) {
  int st = check_plan(plan);
  if (st) return st;
  if (!d_f || !d_u || ncycles < 0) return SNAC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)plan->nz * plan->lev[0].ncell * plan_inner_size(plan);
  if (plan->scaled_f) CK(launch_to_split(plan, (const double*)d_f, (double*)plan->lev[0].d_f, s));
  else CK(cudaMemcpyAsync(plan->lev[0].d_f, d_f, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(plan->lev[0].d_u, d_u, bytes, cudaMemcpyDeviceToDevice, s));
  if ((st = set_active_all(plan, s))) return st;
  // the zero-iterate norms put the right-hand side into the form the cycles read (scaled plans)
  if (plan->scaled_f) CK(launch_mode_norms(plan, plan->nz, false, s));
  for (int c = 0; c < ncycles; ++c) CK(launch_vcycle(plan, plan->nz, s));
  CK(cudaMemcpyAsync(d_u, plan->lev[0].d_u, bytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaStreamSynchronize(s));
  profile_resolve(plan);
  return SNAC_OK;
}

}  // extern "C"
