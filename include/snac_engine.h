/*
 * snac_engine.h -- a serving engine for the Poisson solves of snac.h: requests for problems of
 * different grids, boundary conditions and precisions arrive at any time, are admitted under a
 * device-memory budget, and run concurrently on the GPU.
 *
 * The paper solves one problem per time step (Algorithm 1 inside its Navier-Stokes solver) and has
 * no counterpart of this engine; it is the serving form of the same solve. Each request runs exactly
 * the computation of snac_plan_create + snac_poisson_solve on its own problem (same kernels, same
 * fixed-order reductions), so its result does not depend on which other requests share the GPU.
 *
 * Model
 * -----
 *  Workers.   `workers` host threads, each with its own non-blocking CUDA stream on the device that
 *             was current when the engine was created. A worker takes an admitted request, copies its
 *             right-hand side to the device, solves from a zero initial guess, copies the solution
 *             back and releases the request's memory. Requests on different workers overlap on the
 *             GPU.
 *  Merging.   Small problems are batched as they arrive (continuous batching): a worker that takes a
 *             request whose cached plan solves its wavenumbers on chip (snac_options.onchip) also
 *             takes the other admitted requests of that kind with the same tolerance, up to
 *             `max_group` in all, and solves them together with snac_poisson_solve_batch -- one
 *             persistent launch per step serves every wavenumber of every request in the group. A
 *             request that needs a plan built, or the autotuner, runs alone. The batched solve
 *             gives each problem the result it gets alone (bitwise), so merging changes timing only.
 *  Plans.     Plans are cached by problem (blocks, spacings, boundary conditions, homogeneous axis,
 *             options) and reused by later requests of the same problem: the level hierarchy,
 *             coefficients, shifts, twiddles and coarse factors stay resident. A cached plan serves one
 *             request at a time; a concurrent request of the same problem gets its own plan, up to
 *             `workers` plans per problem, after which it waits for one of them.
 *             Idle plans are evicted least-recently-used when the cache holds more than
 *             `max_cached_plans` or when their memory is needed to admit a request.
 *  Admission. The engine accounts every device byte it holds: cached plans (idle or busy), plans being
 *             built (at an estimate until built, then at their size), and the device copies of each
 *             running request's right-hand side and solution (16 bytes per cell). A waiting request is
 *             admitted when its bytes fit in `hbm_budget` (after evicting idle plans); the queue is
 *             scanned in arrival order and the first request that fits is admitted (first fit), so a
 *             small request is not held behind a large one. A request that can never fit is refused
 *             at submission (SNAC_ERR_OOM).
 *  Tuning.    With autotune, a problem's first request also times candidate schedules
 *             (snac_autotune) before its solve; the tuner's scratch field (8 bytes per cell) is
 *             counted in that request's admission. Results stay those of snac_poisson_solve with the
 *             chosen options.
 *  Times.     Each request records, on the engine's monotonic clock (seconds): submission, admission,
 *             start on a worker, and completion (solution on the host).
 *
 * Ownership: the engine copies the block descriptions (including the cell-width arrays) at
 * submission. h_rhs must stay valid and unchanged, and h_p writable, until snac_engine_wait has
 * returned for that ticket. Calls on one engine may come from any host thread.
 *
 * Errors: as in snac.h. A failed solve is reported by snac_engine_wait with its status; the engine
 * stays usable.
 */
#ifndef SNAC_ENGINE_H
#define SNAC_ENGINE_H

#include <stddef.h>
#include <stdint.h>

#include "snac.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snac_engine snac_engine;

typedef struct {
  int32_t workers;          /* worker threads / CUDA streams, 1..64 (4)                                  */
  int32_t max_cached_plans; /* idle plans kept resident, 0..4096 (64)                                     */
  uint64_t hbm_budget;      /* device bytes the engine may hold (150e9); must cover the largest request  */
  int32_t autotune;         /* 1: the first request of each problem runs snac_autotune on its own
                               right-hand side (from its submitted options) and later requests of that
                               problem reuse the chosen schedule; 0: options as submitted (0)         */
  int32_t max_group;        /* most requests one worker solves together (Merging), 1..256; 1 = never
                               merge (16)                                                              */
} snac_engine_options;

typedef struct {
  double t_submit, t_admit, t_start, t_done; /* engine clock, seconds                                 */
  int32_t worker;                            /* worker that ran the request                           */
  int32_t plan_reused;                       /* 1 if a cached plan served it, 0 if one was built      */
  int32_t tuned;                             /* 1 if this request ran the autotuner                   */
  int32_t group;                             /* requests in the batched solve that ran it (1: alone)  */
  char error[160];                           /* detail of a failed request (empty if it succeeded)    */
} snac_request_times;

typedef struct {
  uint64_t bytes_in_use;    /* accounted device bytes now                                             */
  uint64_t bytes_peak;      /* largest accounted total so far                                         */
  int32_t plans_cached;     /* plans resident (idle + busy)                                           */
  int32_t queued;           /* requests waiting for admission                                         */
  int32_t running;          /* requests admitted and not yet complete                                 */
  int64_t completed;        /* requests completed (successfully or not)                               */
  int64_t plans_built;      /* plans created so far                                                   */
  int64_t plans_evicted;    /* plans released by the cache                                            */
} snac_engine_stats;

/* Create an engine on the current CUDA device (NULL options = the defaults shown above).
 * SNAC_ERR_INVALID_ARG for a field outside its range. */
int snac_engine_create(snac_engine **out, const snac_engine_options *opt);

/* Submit one solve of A p = f to ||f - A p|| <= tol ||f|| (snac_poisson_solve) from p = 0.
 * blocks/homog_axis/opt as in snac_plan_create; h_rhs: host float64 field in the layout of snac.h;
 * h_p: host float64 field that receives the solution. *ticket identifies the request.
 * SNAC_ERR_INVALID_ARG for bad arguments, SNAC_ERR_LAYOUT for an invalid block layout,
 * SNAC_ERR_OOM if the request alone exceeds the budget. */
int snac_engine_submit(snac_engine *e, int32_t nblocks, const snac_block *blocks, int32_t homog_axis,
                       const snac_options *opt, const double *h_rhs, double *h_p, double tol, int64_t *ticket);

/* Block until the request is complete; return its solve status (and release the ticket). info and
 * times may be NULL. SNAC_ERR_INVALID_ARG for an unknown ticket. */
int snac_engine_wait(snac_engine *e, int64_t ticket, snac_solve_info *info, snac_request_times *times);

/* Counters of the engine (any time). */
int snac_engine_get_stats(snac_engine *e, snac_engine_stats *st);

/* Seconds on the engine clock (steady, shared by all engines of the process). */
double snac_engine_clock(void);

/* Wait for every submitted request, stop the workers, release every plan. NULL is accepted.
 * Tickets not waited for are dropped. */
int snac_engine_destroy(snac_engine *e);

#ifdef __cplusplus
}
#endif

#endif /* SNAC_ENGINE_H */
