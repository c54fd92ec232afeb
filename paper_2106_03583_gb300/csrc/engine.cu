// Serving engine (include/snac_engine.h): admission under a device-memory budget, a cache of
// resident plans, worker threads that each drive their own CUDA stream, and continuous batching of
// small problems. Host code only; every step of a solve runs in the library's kernels through
// snac_plan_create / snac_poisson_solve / snac_poisson_solve_batch.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "snac_engine.h"
#include "snac_impl.h"

namespace snac {
void set_error(const std::string& s);
}

namespace {

using Clock = std::chrono::steady_clock;
const Clock::time_point g_epoch = Clock::now();

double now_s() { return std::chrono::duration<double>(Clock::now() - g_epoch).count(); }

struct PlanSlot {
  std::string key;
  snac_plan* plan = nullptr;
  uint64_t bytes = 0;
  bool busy = false;
  uint64_t last_use = 0;
};

enum class State { Queued, Ready, Running, Done };

struct Request {
  int64_t ticket = 0;
  std::vector<std::vector<double>> dx;  // copies of the cell widths, 3 per block
  std::vector<snac_block> blocks;       // h_dx pointing into dx
  int32_t homog_axis = 2;
  bool has_opt = false;
  snac_options opt{};
  const double* h_rhs = nullptr;
  double* h_p = nullptr;
  double tol = 0.0;
  long long n3 = 0;
  std::string key;
  uint64_t buf_bytes = 0;      // device copies of f and p
  uint64_t plan_estimate = 0;  // reservation while its plan is built
  uint64_t tune_bytes = 0;     // the autotuner's scratch field, while it runs
  bool tune = false;           // this request runs the autotuner
  // progress
  State state = State::Queued;
  PlanSlot* slot = nullptr;
  bool build_plan = false;
  int status = SNAC_OK;
  snac_solve_info info{};
  snac_request_times times{};
};

template <typename T>
void put(std::string& k, const T& v) {
  k.append(reinterpret_cast<const char*>(&v), sizeof(T));
}

// Identity of a problem: everything snac_plan_create reads.
std::string problem_key(const Request& r) {
  std::string k;
  put(k, r.homog_axis);
  put(k, (int32_t)r.blocks.size());
  for (size_t b = 0; b < r.blocks.size(); ++b) {
    const snac_block& s = r.blocks[b];
    for (int a = 0; a < 3; ++a) {
      put(k, s.lo[a]);
      put(k, s.hi[a]);
      for (int sd = 0; sd < 2; ++sd) {
        put(k, s.bc[a][sd]);
        put(k, s.nbr[a][sd]);
      }
      k.append(reinterpret_cast<const char*>(r.dx[3 * b + a].data()), r.dx[3 * b + a].size() * sizeof(double));
    }
  }
  put(k, (int32_t)r.has_opt);
  if (r.has_opt) {
    put(k, r.opt.precision);
    put(k, r.opt.nu1);
    put(k, r.opt.nu2);
    put(k, r.opt.max_outer);
    put(k, r.opt.max_cycles);
    put(k, r.opt.max_coarse);
    put(k, r.opt.fused);
    put(k, r.opt.inner_reduction);
    put(k, r.opt.shift);
    put(k, r.opt.onchip);
    put(k, r.opt.bottom_cells);
  }
  return k;
}

// Device bytes of a plan before it exists: the level hierarchy (u, f and, FP64, the inverse
// diagonals, x 4/3 over levels; FP32 fused levels add a second iterate), the residual field and the
// small tables, rounded up. Replaced by the plan's own count once it is built.
uint64_t plan_estimate(long long n3, bool fp64) {
  const double per_cell = fp64 ? 64.0 : 40.0;
  return (uint64_t)(per_cell * (double)n3) + (64ull << 20);
}

}  // namespace

struct snac_engine {
  int device = 0;
  snac_engine_options opt{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;  // waiting for admission, arrival order
  std::deque<Request*> ready;  // admitted, waiting for a worker
  std::map<int64_t, Request*> tickets;
  std::list<PlanSlot*> plans;
  std::map<std::string, snac_options> tuned;  // problem key -> chosen schedule (autotune)
  std::map<std::string, int> building;        // problem key -> plans being built
  uint64_t used = 0, peak = 0, use_clock = 0;
  int running = 0;
  int64_t completed = 0, built = 0, evicted = 0, next_ticket = 1;
  bool stopping = false;
  std::vector<std::thread> threads;

  void account(int64_t delta) {
    used = (uint64_t)((int64_t)used + delta);
    peak = std::max(peak, used);
  }

  // Idle plans beyond the cache size, least recently used first (caller holds mu).
  void trim_cache(std::vector<snac_plan*>& dead) {
    int idle = 0;
    for (PlanSlot* s : plans) idle += s->busy ? 0 : 1;
    while (idle > opt.max_cached_plans && evict_one(nullptr, dead)) --idle;
  }

  // Release the least recently used idle plan other than `keep` (caller holds mu).
  bool evict_one(const PlanSlot* keep, std::vector<snac_plan*>& dead) {
    auto victim = plans.end();
    for (auto it = plans.begin(); it != plans.end(); ++it)
      if (!(*it)->busy && *it != keep && (victim == plans.end() || (*it)->last_use < (*victim)->last_use)) victim = it;
    if (victim == plans.end()) return false;
    dead.push_back((*victim)->plan);
    account(-(int64_t)(*victim)->bytes);
    delete *victim;
    plans.erase(victim);
    ++evicted;
    return true;
  }

  // Admit waiting requests, first fit in arrival order (caller holds mu).
  void admit(std::vector<snac_plan*>& dead) {
    for (auto it = queue.begin(); it != queue.end();) {
      Request* r = *it;
      PlanSlot* idle = nullptr;
      int have = 0;  // plans of this problem, resident or being built
      for (PlanSlot* s : plans) {
        if (s->key != r->key) continue;
        ++have;
        if (!s->busy && (!idle || s->last_use > idle->last_use)) idle = s;
      }
      auto bit = building.find(r->key);
      if (bit != building.end()) have += bit->second;
      if (!idle && have >= opt.workers) {  // enough plans of this problem: wait for one of them
        ++it;
        continue;
      }
      r->tune = !idle && opt.autotune && tuned.find(r->key) == tuned.end();
      const uint64_t need = r->buf_bytes + (idle ? 0 : r->plan_estimate) + (r->tune ? r->tune_bytes : 0);
      while (used + need > opt.hbm_budget && evict_one(idle, dead)) {
      }
      if (used + need > opt.hbm_budget) {
        ++it;
        continue;
      }
      account((int64_t)need);
      if (idle) {
        idle->busy = true;
        r->slot = idle;
      } else {
        r->build_plan = true;
        ++building[r->key];
      }
      r->state = State::Ready;
      r->times.t_admit = now_s();
      ready.push_back(r);
      it = queue.erase(it);
      cv_work.notify_one();
    }
  }

  // A request that may share a batched solve: its cached plan is resident and solves on chip
  // (caller holds mu).
  static bool mergeable(const Request* r) {
    return r->slot && !r->build_plan && !r->tune && r->slot->plan->onchip;
  }

  // Take the next ready request and, if it is mergeable, the ready requests that can join it
  // (caller holds mu).
  void take(std::vector<Request*>& group) {
    Request* r = ready.front();
    ready.pop_front();
    group.push_back(r);
    if (!mergeable(r)) return;
    for (auto it = ready.begin(); it != ready.end() && (int)group.size() < opt.max_group;) {
      if (mergeable(*it) && (*it)->tol == r->tol) {
        group.push_back(*it);
        it = ready.erase(it);
      } else {
        ++it;
      }
    }
  }

  void worker(int id);
  int run(Request* r, cudaStream_t s);
  void run_group(const std::vector<Request*>& g, cudaStream_t s, std::vector<int>& st);
};

namespace {

void destroy_plans(const std::vector<snac_plan*>& dead) {
  for (snac_plan* p : dead) snac_plan_destroy(p);
}

}  // namespace

// One request on stream s: build its plan if needed, copy f in, solve from zero, copy p out.
int snac_engine::run(Request* r, cudaStream_t s) {
  int st = SNAC_OK;
  const size_t nb = (size_t)r->n3 * sizeof(double);
  double *d_f = nullptr, *d_p = nullptr;
  if (cudaMallocAsync((void**)&d_f, nb, s) != cudaSuccess || cudaMallocAsync((void**)&d_p, nb, s) != cudaSuccess) {
    cudaGetLastError();
    if (d_f) cudaFreeAsync(d_f, s);
    cudaStreamSynchronize(s);
    std::lock_guard<std::mutex> lk(mu);
    if (r->build_plan) {
      account(-(int64_t)r->plan_estimate);
      if (--building[r->key] == 0) building.erase(r->key);
    }
    if (r->tune) account(-(int64_t)r->tune_bytes);
    return SNAC_ERR_OOM;
  }
  cudaError_t ce = cudaMemcpyAsync(d_f, r->h_rhs, nb, cudaMemcpyHostToDevice, s);
  bool ok = ce == cudaSuccess;
  if (!ok) snac::set_error(std::string("engine: copy of the right-hand side: ") + cudaGetErrorString(ce));
  if (r->build_plan) {
    snac_options use = r->has_opt ? r->opt : snac_options{};
    bool have_opt = r->has_opt;
    if (r->tune && ok) {  // choose the schedule on this request's right-hand side
      snac_options chosen{};
      if (snac_autotune((int32_t)r->blocks.size(), r->blocks.data(), r->homog_axis, r->has_opt ? &r->opt : nullptr,
                        d_f, r->tol, &chosen, nullptr, s) == SNAC_OK) {
        use = chosen;
        have_opt = true;
        std::lock_guard<std::mutex> lk(mu);
        tuned[r->key] = chosen;
      }
      r->times.tuned = 1;
    } else {
      std::lock_guard<std::mutex> lk(mu);
      auto it = tuned.find(r->key);
      if (it != tuned.end()) {
        use = it->second;
        have_opt = true;
      }
    }
    snac_plan* pl = nullptr;
    st = snac_plan_create(&pl, (int32_t)r->blocks.size(), r->blocks.data(), r->homog_axis, have_opt ? &use : nullptr);
    size_t bytes = 0;
    if (st == SNAC_OK) snac_plan_workspace_bytes(pl, &bytes);
    std::lock_guard<std::mutex> lk(mu);
    account(-(int64_t)r->plan_estimate);
    if (r->tune) account(-(int64_t)r->tune_bytes);
    if (--building[r->key] == 0) building.erase(r->key);
    PlanSlot* slot = st == SNAC_OK ? new (std::nothrow) PlanSlot{r->key, pl, (uint64_t)bytes, true, 0} : nullptr;
    if (st == SNAC_OK && !slot) {
      snac_plan_destroy(pl);
      st = SNAC_ERR_OOM;
    }
    if (st != SNAC_OK) {
      cudaFreeAsync(d_f, s);
      cudaFreeAsync(d_p, s);
      cudaStreamSynchronize(s);
      return st;
    }
    account((int64_t)bytes);
    plans.push_back(slot);
    r->slot = slot;
    ++built;
  }
  r->times.plan_reused = r->build_plan ? 0 : 1;
  if (ok && (ce = cudaMemsetAsync(d_p, 0, nb, s)) != cudaSuccess) {
    ok = false;
    snac::set_error(std::string("engine: zeroing the solution: ") + cudaGetErrorString(ce));
  }
  if (ok) {
    st = snac_poisson_solve(r->slot->plan, d_f, d_p, r->tol, s);
    snac_plan_info(r->slot->plan, &r->info);
    if ((st == SNAC_OK || st == SNAC_ERR_NOT_CONVERGED) &&
        (ce = cudaMemcpyAsync(r->h_p, d_p, nb, cudaMemcpyDeviceToHost, s)) != cudaSuccess) {
      st = SNAC_ERR_CUDA;
      snac::set_error(std::string("engine: copy of the solution: ") + cudaGetErrorString(ce));
    }
  } else {
    st = SNAC_ERR_CUDA;
  }
  cudaFreeAsync(d_f, s);
  cudaFreeAsync(d_p, s);
  if ((ce = cudaStreamSynchronize(s)) != cudaSuccess && st == SNAC_OK) {
    st = SNAC_ERR_CUDA;
    snac::set_error(std::string("engine: stream synchronisation: ") + cudaGetErrorString(ce));
  }
  return st;
}

// Requests of resident on-chip plans on stream s, solved together by snac_poisson_solve_batch:
// one device block holds every right-hand side and solution, each copied in and out on its own.
void snac_engine::run_group(const std::vector<Request*>& g, cudaStream_t s, std::vector<int>& st) {
  const size_t n = g.size();
  std::vector<size_t> off(n + 1, 0);
  for (size_t k = 0; k < n; ++k) {  // 256-byte aligned field pairs (f, p)
    const size_t nb = ((size_t)g[k]->n3 * sizeof(double) + 255) / 256 * 256;
    off[k + 1] = off[k] + 2 * nb;
  }
  st.assign(n, SNAC_ERR_CUDA);
  char* base = nullptr;
  cudaError_t ce = cudaMallocAsync((void**)&base, off[n], s);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    st.assign(n, SNAC_ERR_OOM);
    snac::set_error("engine: device buffers of a batched group could not be allocated");
    return;
  }
  std::vector<snac_plan*> plans(n);
  std::vector<const double*> fs(n);
  std::vector<double*> ps(n);
  bool ok = true;
  for (size_t k = 0; k < n && ok; ++k) {
    const size_t nb = (size_t)g[k]->n3 * sizeof(double);
    plans[k] = g[k]->slot->plan;
    double* f = reinterpret_cast<double*>(base + off[k]);
    ps[k] = reinterpret_cast<double*>(base + off[k] + (off[k + 1] - off[k]) / 2);
    fs[k] = f;
    if ((ce = cudaMemcpyAsync(f, g[k]->h_rhs, nb, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (ce = cudaMemsetAsync(ps[k], 0, nb, s)) != cudaSuccess) {
      ok = false;
      snac::set_error(std::string("engine: copies into a batched group: ") + cudaGetErrorString(ce));
    }
  }
  if (ok) {
    std::vector<int32_t> hs(n, INT32_MIN);
    const int rc = snac_poisson_solve_batch((int32_t)n, plans.data(), fs.data(), ps.data(), g[0]->tol, hs.data(), s);
    for (size_t k = 0; k < n; ++k) {
      st[k] = hs[k] == INT32_MIN ? (rc ? rc : SNAC_ERR_CUDA) : hs[k];  // rejected before it ran: its status
      snac_plan_info(plans[k], &g[k]->info);
      if ((st[k] == SNAC_OK || st[k] == SNAC_ERR_NOT_CONVERGED) &&
          (ce = cudaMemcpyAsync(g[k]->h_p, ps[k], (size_t)g[k]->n3 * sizeof(double), cudaMemcpyDeviceToHost, s)) !=
              cudaSuccess) {
        st[k] = SNAC_ERR_CUDA;
        snac::set_error(std::string("engine: copy of a solution: ") + cudaGetErrorString(ce));
      }
    }
  }
  cudaFreeAsync(base, s);
  if ((ce = cudaStreamSynchronize(s)) != cudaSuccess) {
    snac::set_error(std::string("engine: stream synchronisation: ") + cudaGetErrorString(ce));
    for (int& x : st)
      if (x == SNAC_OK) x = SNAC_ERR_CUDA;
  }
}

void snac_engine::worker(int id) {
  cudaSetDevice(device);
  cudaStream_t s = nullptr;
  cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  std::vector<Request*> g;
  std::vector<int> st;
  for (;;) {
    g.clear();
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stopping || !ready.empty(); });
      if (ready.empty()) break;
      take(g);
      for (Request* r : g) r->state = State::Running;
      running += (int)g.size();
    }
    const double t0 = now_s();
    for (Request* r : g) {
      r->times.t_start = t0;
      r->times.worker = id;
      r->times.group = (int32_t)g.size();
    }
    snac::set_error("");
    st.assign(g.size(), SNAC_ERR_CUDA);
    if (!s) {  // this worker has no stream: release what the admission reserved for a plan build
      std::lock_guard<std::mutex> lk(mu);
      for (Request* r : g) {
        if (r->build_plan) {
          account(-(int64_t)r->plan_estimate);
          if (--building[r->key] == 0) building.erase(r->key);
        }
        if (r->tune) account(-(int64_t)r->tune_bytes);
      }
      snac::set_error("engine: the worker's CUDA stream could not be created");
    } else if (g.size() == 1) {
      st[0] = run(g[0], s);
    } else {
      run_group(g, s, st);
      for (Request* r : g) r->times.plan_reused = 1;
    }
    const double t1 = now_s();
    for (size_t k = 0; k < g.size(); ++k) {
      g[k]->times.t_done = t1;
      if (st[k] != SNAC_OK) {  // the detail this worker thread recorded (plan creation, solve or copies)
        std::strncpy(g[k]->times.error, snac_last_error_message(), sizeof(g[k]->times.error) - 1);
        g[k]->times.error[sizeof(g[k]->times.error) - 1] = '\0';
      }
    }
    std::vector<snac_plan*> dead;
    {
      std::lock_guard<std::mutex> lk(mu);
      for (size_t k = 0; k < g.size(); ++k) {
        Request* r = g[k];
        account(-(int64_t)r->buf_bytes);
        if (r->slot) {
          r->slot->busy = false;
          r->slot->last_use = ++use_clock;
        }
        r->status = st[k];
        r->info.status = st[k];
        r->state = State::Done;
        --running;
        ++completed;
      }
      trim_cache(dead);
      admit(dead);
    }
    cv_done.notify_all();
    destroy_plans(dead);
  }
  if (s) cudaStreamDestroy(s);
}

extern "C" {

double snac_engine_clock(void) { return now_s(); }

int snac_engine_create(snac_engine** out, const snac_engine_options* opt) {
  if (!out) return SNAC_ERR_INVALID_ARG;
  *out = nullptr;
  snac_engine_options o{4, 64, 150000000000ull, 0, 16};
  if (opt) o = *opt;
  if (o.workers < 1 || o.workers > 64 || o.max_cached_plans < 0 || o.max_cached_plans > 4096 || o.hbm_budget == 0 ||
      (o.autotune != 0 && o.autotune != 1) || o.max_group < 1 || o.max_group > 256)
    return SNAC_ERR_INVALID_ARG;
  snac_engine* e = new (std::nothrow) snac_engine();
  if (!e) return SNAC_ERR_OOM;
  e->opt = o;
  if (cudaGetDevice(&e->device) != cudaSuccess) {
    cudaGetLastError();
    delete e;
    return SNAC_ERR_CUDA;
  }
  try {
    for (int w = 0; w < o.workers; ++w) e->threads.emplace_back(&snac_engine::worker, e, w);
  } catch (...) {
    {
      std::lock_guard<std::mutex> lk(e->mu);
      e->stopping = true;
    }
    e->cv_work.notify_all();
    for (std::thread& t : e->threads) t.join();
    delete e;
    return SNAC_ERR_OOM;
  }
  *out = e;
  return SNAC_OK;
}

int snac_engine_submit(snac_engine* e, int32_t nblocks, const snac_block* blocks, int32_t homog_axis,
                       const snac_options* opt, const double* h_rhs, double* h_p, double tol, int64_t* ticket) {
  if (!e || !blocks || nblocks < 1 || !h_rhs || !h_p || !ticket || !(tol > 0.0) || !std::isfinite(tol))
    return SNAC_ERR_INVALID_ARG;
  if (opt && (opt->mode_begin != 0 || opt->mode_end != 0)) return SNAC_ERR_INVALID_ARG;  // whole solves only
  int st = snac::check_layout(nblocks, blocks, homog_axis);
  if (st) return st;
  Request* r = new (std::nothrow) Request();
  if (!r) return SNAC_ERR_OOM;
  r->homog_axis = homog_axis;
  r->has_opt = opt != nullptr;
  if (opt) r->opt = *opt;
  r->h_rhs = h_rhs;
  r->h_p = h_p;
  r->tol = tol;
  r->blocks.assign(blocks, blocks + nblocks);
  r->dx.resize(3 * (size_t)nblocks);
  long long n3 = 0;
  for (int b = 0; b < nblocks; ++b) {
    long long cells = 1;
    for (int a = 0; a < 3; ++a) {
      const long long n = blocks[b].hi[a] - blocks[b].lo[a] + 1;
      r->dx[3 * b + a].assign(blocks[b].h_dx[a], blocks[b].h_dx[a] + n);
      r->blocks[b].h_dx[a] = r->dx[3 * b + a].data();
      cells *= n;
    }
    n3 += cells;
  }
  r->n3 = n3;
  r->key = problem_key(*r);
  r->buf_bytes = 16ull * (uint64_t)n3;
  r->plan_estimate = plan_estimate(n3, !(opt && opt->precision == SNAC_MIXED));
  r->tune_bytes = e->opt.autotune ? 8ull * (uint64_t)n3 : 0;
  if (r->buf_bytes + r->plan_estimate + r->tune_bytes > e->opt.hbm_budget) {
    delete r;
    return SNAC_ERR_OOM;
  }
  std::vector<snac_plan*> dead;
  {
    std::lock_guard<std::mutex> lk(e->mu);
    if (e->stopping) {
      delete r;
      return SNAC_ERR_INVALID_ARG;
    }
    r->ticket = e->next_ticket++;
    r->times.t_submit = now_s();
    e->tickets[r->ticket] = r;
    e->queue.push_back(r);
    e->admit(dead);
    *ticket = r->ticket;
  }
  destroy_plans(dead);
  return SNAC_OK;
}

int snac_engine_wait(snac_engine* e, int64_t ticket, snac_solve_info* info, snac_request_times* times) {
  if (!e) return SNAC_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(e->mu);
  auto it = e->tickets.find(ticket);
  if (it == e->tickets.end()) return SNAC_ERR_INVALID_ARG;
  Request* r = it->second;
  e->cv_done.wait(lk, [&] { return r->state == State::Done; });
  if (info) *info = r->info;
  if (times) *times = r->times;
  const int st = r->status;
  e->tickets.erase(it);
  delete r;
  return st;
}

int snac_engine_get_stats(snac_engine* e, snac_engine_stats* st) {
  if (!e || !st) return SNAC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(e->mu);
  st->bytes_in_use = e->used;
  st->bytes_peak = e->peak;
  st->plans_cached = (int32_t)e->plans.size();
  st->queued = (int32_t)e->queue.size();
  st->running = (int32_t)(e->ready.size() + e->running);
  st->completed = e->completed;
  st->plans_built = e->built;
  st->plans_evicted = e->evicted;
  return SNAC_OK;
}

int snac_engine_destroy(snac_engine* e) {
  if (!e) return SNAC_OK;
  {
    std::unique_lock<std::mutex> lk(e->mu);
    e->cv_done.wait(lk, [&] { return e->queue.empty() && e->ready.empty() && e->running == 0; });
    e->stopping = true;
  }
  e->cv_work.notify_all();
  for (std::thread& t : e->threads) t.join();
  for (PlanSlot* s : e->plans) {
    snac_plan_destroy(s->plan);
    delete s;
  }
  for (auto& kv : e->tickets) delete kv.second;
  delete e;
  return SNAC_OK;
}

}  // extern "C"
