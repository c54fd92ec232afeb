/*
 * snac.h -- C ABI of the GB300 FFT-accelerated multi-block Poisson solver.
 *
 * Solves the second-order finite-volume Poisson equation of Costa, "A FFT-accelerated multi-block
 * finite-difference solver for massively parallel simulations of incompressible flows"
 * (arXiv 2106.03583): Eq. 8 on a structured grid made of several blocks (Sec. 3.1), stretched along
 * x and y and uniform along the homogeneous direction z. The solve follows Algorithm 1 (Sec. 2):
 * a real-to-real transform along z chosen by the boundary pair (Table 1), one multigrid solve of the
 * reduced equation (Eq. 9) per wavenumber, and the inverse transform -- wrapped in an FP64
 * defect-correction loop r = f - A p, p += A^-1 r that stops at a relative residual tolerance.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Layout.    A 3-D field (right-hand side, solution, residual) is one contiguous float64 buffer:
 *             blocks concatenated in id order, each block stored [z][y][x] with x fastest.
 *             A mode-space field ("modes") is [q][cell] with q the wavenumber (0..n-1 along the
 *             homogeneous axis) and cell running over the cells of the two other axes of all
 *             blocks, block by block, [b][a] within a block with a < b the two non-homogeneous
 *             axes (a fastest; [y][x] when z is homogeneous); its element type is the plan's
 *             inner type (double for SNAC_FP64, float for SNAC_MIXED).
 *  Memory.    Pointers named d_* are device pointers on the current CUDA device; h_* are host
 *             pointers. The caller owns every buffer it passes; the library never frees them, never
 *             writes an input, and keeps no pointer to them after the call returns.
 *  Streams.   `stream` is a cudaStream_t (passed as void*; NULL = legacy default stream). Every
 *             call that takes one enqueues its work on it and returns after that work is complete
 *             (the solve reads residual norms back to the host).
 *  Plans.     A plan owns its device workspace (level hierarchy, coefficients, eigenvalue shifts,
 *             transform twiddles, coarse-level factors, scratch). A plan is not re-entrant: one call
 *             at a time per plan. Distinct plans may run concurrently on distinct streams.
 *  Errors.    Every function returns SNAC_OK (0) or a negative snac_status. Nothing aborts and no
 *             exception crosses the ABI. After an error the plan stays usable unless the status is
 *             SNAC_ERR_CUDA (the CUDA context may then be unusable).
 */
#ifndef SNAC_H
#define SNAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SNAC_OK = 0,
  SNAC_ERR_INVALID_ARG = -1,      /* NULL pointer, bad size, bad enum value                          */
  SNAC_ERR_LAYOUT = -2,           /* block graph not congruent / not symmetric, z not uniform, n_z
                                     odd for a periodic z, blocks not coarsenable, ...               */
  SNAC_ERR_OOM = -3,              /* device allocation failed                                         */
  SNAC_ERR_CUDA = -4,             /* a CUDA call failed                                               */
  SNAC_ERR_NOT_CONVERGED = -5,    /* tolerance not reached within max_outer, or a defect-correction
                                     step did not lower the residual (the floating-point floor);
                                     p holds the iterate with the smallest residual                   */
  SNAC_ERR_NONFINITE = -6,        /* a residual norm was NaN or Inf (non-finite input)                */
  SNAC_ERR_INCOMPATIBLE_RHS = -7, /* singular problem whose right-hand side has a non-zero mean       */
  SNAC_ERR_TIMEOUT = -8           /* a bounded device-side wait gave up (1 s); nothing was trapped and
                                     the context stays usable                                        */
} snac_status;

/* Face kinds (Sec. 3.1: Dirichlet, Neumann, block-block connectivity; periodic = the cyclic
 * connectivity of a block with itself). Homogeneous Dirichlet/Neumann pressure conditions are imposed
 * at the face (staggered grid): the ghost cell mirrors the first cell with sign -1 / +1. */
typedef enum {
  SNAC_BC_DIRICHLET = 0,
  SNAC_BC_NEUMANN = 1,
  SNAC_BC_PERIODIC = 2,
  SNAC_BC_BLOCK = 3
} snac_bc;

/* One block (Sec. 3.1, Table 2). lo/hi: inclusive index-space corners, n_a = hi[a]-lo[a]+1.
 * h_dx[a]: host array of n_a cell widths along axis a (copied at plan creation; the grid mapping of
 * Table 2 is applied by the caller). bc[a][s]: face kind of the lower (s=0) / upper (s=1) face along
 * axis a. nbr[a][s]: id of the connected block across a SNAC_BC_BLOCK face, else -1.
 * Rules (checked, SNAC_ERR_LAYOUT otherwise): a connected face coincides with the neighbour's
 * opposite face (same extent and the same cell widths along it), connectivity is symmetric, every
 * block spans the whole homogeneous axis with the same n_z, uniform width and boundary pair. */
typedef struct {
  int64_t lo[3];
  int64_t hi[3];
  const double *h_dx[3];
  int32_t bc[3][2];
  int32_t nbr[3][2];
} snac_block;

typedef enum { SNAC_FP64 = 0, SNAC_MIXED = 1 } snac_precision;

/* Solver options; pass NULL to snac_plan_create for the defaults shown. */
typedef struct {
  int32_t precision;   /* SNAC_FP64 (default): every stage in FP64. SNAC_MIXED: transforms and
                          multigrid in FP32 inside the FP64 defect-correction loop; the outer
                          residual, the update, the eigenvalue shifts and the coarsest solve stay FP64 */
  int32_t nu1, nu2;    /* red-black Gauss-Seidel sweeps before / after the coarse correction (2, 2)  */
  int32_t max_outer;   /* defect-correction iterations (20)                                          */
  int32_t max_cycles;  /* V-cycles per wavenumber per outer iteration (40)                          */
  int32_t max_coarse;  /* coarsen while a plane has more than this many cells (64; <= 256)          */
  int32_t fused;       /* fused tile kernels (smoothing + restriction, prolongation + smoothing in
                          shared memory) on levels whose blocks are all >= 8 cells wide:
                          -1 = auto (on for SNAC_MIXED, off for SNAC_FP64), 0 = off, 1 = on         */
  double inner_reduction; /* mixed plans: residual reduction asked of the FP32 multigrid in each
                             defect-correction step, in (0, 1); 0 (default) = automatic: 1e-4, or
                             3e-5 for plans that solve on chip (see onchip: there an outer step --
                             a 3-D residual pass, both transforms, a host round trip -- costs as much
                             as several V-cycles). FP64 plans solve each step to the tolerance      */
  double shift;        /* Helmholtz shift s <= 0 (0): solve (A + s I) p = f, the Helmholtz form the
                          method applies to unchanged (Sec. 3.3, footnote); every reduced equation
                          (Eq. 9) gets the extra diagonal s, and s < 0 removes the null space of the
                          periodic / all-Neumann case (no mean is removed then)                     */
  int32_t mode_begin, mode_end; /* (0, 0): every wavenumber. Otherwise 0 <= mode_begin < mode_end <= n_z
                          gives a wavenumber-range plan: one rank's slab of wavenumbers in a solve
                          sharded over several GPUs (App. A, Algorithm 3). Its mode-space fields hold
                          wavenumbers mode_begin .. mode_end - 1 only (local index q - mode_begin);
                          it has no 3-D field, so the calls on 3-D fields return
                          SNAC_ERR_INVALID_ARG, and the pencil calls below take their place          */
  int32_t onchip;      /* 0 (default): when the whole multigrid hierarchy of a wavenumber, from the
                          finest plane, fits in one CTA's shared memory, each wavenumber's solve runs
                          on chip in one CTA and its convergence is decided on the device (one launch
                          per defect-correction step); -1: always the level-by-level path            */
  int32_t bottom_cells;  /* where the bottom sub-cycle starts (the coarse levels that run in one CTA's
                          shared memory per wavenumber, one launch per cycle): at the finest level below
                          level 0 whose plane has at most this many cells and whose hierarchy fits;
                          0 (default) = 8192; 16 .. 8192; -1 = none (every level level by level, a
                          dense solve at the coarsest). Changes the launch shape only, not the method */
} snac_options;

/* Result of the last solve of a plan. */
typedef struct {
  int32_t status;        /* status of the last solve                                                */
  int32_t outer_iters;   /* defect-correction iterations performed                                  */
  int32_t total_cycles;  /* V-cycles summed over wavenumbers and outer iterations                    */
  int32_t max_mode_cycles; /* largest number of V-cycles of one wavenumber in one outer iteration   */
  int32_t levels;        /* multigrid levels (1 = direct solve of the plane)                         */
  int32_t n_modes;       /* n_z                                                                      */
  double rel_res;        /* final ||f - A p||_2 / ||f||_2 (f after mean removal)                     */
  double rhs_norm;       /* ||f||_2                                                                  */
  double removed_mean;   /* volume-weighted mean removed from f (singular problems), else 0         */
  int32_t graph_rounds;  /* V-cycle rounds of the solve replayed from captured CUDA graphs          */
} snac_solve_info;

typedef struct snac_plan snac_plan;

/* Build a plan for the multi-block problem (Sec. 3.1 setup; Table 1 for the homogeneous pair).
 * homog_axis (0 = x, 1 = y, 2 = z) names the homogeneous direction of Sec. 2 (the paper writes
 * Eq. 9 with the synthesis along x2): uniform, one boundary pair shared by all blocks, not split into
 * blocks (SNAC_ERR_LAYOUT otherwise). The caller's arrays keep the [z][y][x] layout whatever the
 * axis; the transforms run along homog_axis and the multigrid on the planes of the other two.
 * z is the fastest choice: with x, the outer residual walks the arrays across their contiguous
 * axis. On success *out receives a plan owning its device workspace, allocated on the current CUDA
 * device. */
int snac_plan_create(snac_plan **out, int32_t nblocks, const snac_block *blocks, int32_t homog_axis,
                     const snac_options *opt);

/* Device bytes held by the plan. */
int snac_plan_workspace_bytes(const snac_plan *plan, size_t *bytes);

/* Solve A p = f (Eq. 8) to ||f - A p|| <= tol ||f|| (Algorithm 1 inside FP64 defect correction).
 * d_rhs: device float64 3-D field, read only. d_p: device float64 3-D field, in: initial guess (the
 * latest solution, Sec. 3.3.1), out: solution. Singular problems (periodic or Neumann-Neumann z and
 * no Dirichlet face in x-y): a volume-weighted mean of f within 1e-12 sum(V|f|) is removed and the
 * zero-mean solution returned; a larger mean gives SNAC_ERR_INCOMPATIBLE_RHS with p untouched.
 * A zero f gives p = 0. Runs on `stream` and returns when p is complete. It issues kernels only: its
 * small control transfers (norms read back, mode lists) go through pinned host memory mapped into the
 * device (held by the plan), so copies that other streams run meanwhile do not delay it. */
int snac_poisson_solve(snac_plan *plan, const double *d_rhs, double *d_p, double tol, void *stream);

/* Solve n problems together (each as snac_poisson_solve would): plans[k] (distinct plans, all on
 * the current device), d_rhs[k], d_p[k] as in snac_poisson_solve, one tolerance. The problems run
 * in lock-step: each phase's launches of all of them go out together and one synchronisation
 * serves them all; each problem's own launches go to one of up to 16 streams the call creates,
 * forked from `stream` and joined back into it, so that the kernels of different problems overlap;
 * and the wavenumber solves of every plan whose hierarchy fits on chip (see snac_options.onchip)
 * share one persistent launch per precision -- CTAs take (problem, wavenumber)
 * items from a device-side queue, and each wavenumber's V-cycles stop on the device. This is the
 * batched solve of many small systems that the paper's conclusions point to (Sec. 5). h_status[n]
 * receives each problem's status (snac_plan_info gives its statistics); returns SNAC_OK if every
 * problem succeeded, else the first failing status. */
int snac_poisson_solve_batch(int32_t n, snac_plan *const *plans, const double *const *d_rhs, double *const *d_p,
                             double tol, int32_t *h_status, void *stream);

/* Self-test of the bounded device-side wait. For plans that solve on chip, each defect-correction
 * step runs the forward transform and the wavenumber solves in one persistent launch: a solve
 * waits, on the device, until its plan's transform chunks are all counted, for at most 1 s, and
 * then gives up, skips its work and sets a status the host turns into SNAC_ERR_TIMEOUT. This call
 * runs that launch with a chunk count that nothing can reach and a limit of wait_seconds (0 <
 * wait_seconds <= 1): it must return SNAC_ERR_TIMEOUT, with the context still usable. Only for
 * plans of snac_options.onchip whose n_z <= 1024 (SNAC_ERR_INVALID_ARG otherwise); it overwrites the
 * plan's internal work buffers, not the caller's arrays. */
int snac_test_wait_timeout(snac_plan *plan, double wait_seconds, void *stream);

/* Statistics of the last solve. */
int snac_plan_info(const snac_plan *plan, snac_solve_info *info);

/* V-cycles of each wavenumber in the last outer iteration of the last solve: h_cycles[n_z]. */
int snac_plan_mode_cycles(const snac_plan *plan, int32_t *h_cycles, int32_t n);

/* Release the plan and its device workspace. NULL is accepted. */
int snac_plan_destroy(snac_plan *plan);

/* Static string for a status code. */
const char *snac_status_string(int status);

/* Detail of the last error raised by plan creation on this thread (empty if none). */
const char *snac_last_error_message(void);

/* ---- Schedule autotuning ---- */

typedef struct {
  int32_t trials;      /* configurations timed (each: plan creation, one warm solve, timed solves)  */
  int32_t improved;    /* 1 if the chosen options differ from the ones passed in                  */
  double base_ms;      /* mean solve time with the options passed in                              */
  double best_ms;      /* mean solve time with the chosen options                                 */
} snac_tune_report;

/* Choose the multigrid schedule for one problem by timing complete solves (snac_poisson_solve from
 * p = 0) of a representative right-hand side d_rhs (device float64 field, caller layout) at tol.
 * Starting from *base (NULL = defaults), coordinate descent over: (nu1, nu2) in {(2,2), (2,1),
 * (1,2), (1,1)}; max_coarse in {16, 64, 256}; onchip in {auto, off} (the launch shape of the
 * wavenumber solves: one CTA per wavenumber on chip, or level-by-level grids over all wavenumbers);
 * bottom_cells in {8192, 2048, 512}; and for SNAC_MIXED, inner_reduction in {1e-4, 3e-5, 1e-5, 3e-4,
 * 1e-3} and fused in {auto, off}. A candidate counts only if its solve succeeds at tol. *best
 * receives the fastest options (precision, max_outer, max_cycles and shift are kept from *base).
 * The paper has no counterpart (its multigrid is hypre's); this is the schedule choice of a serving
 * system. Allocates and frees plans and an 8-byte-per-cell scratch field on the current device;
 * runs on `stream` and returns when done. report may be NULL. */
int snac_autotune(int32_t nblocks, const snac_block *blocks, int32_t homog_axis, const snac_options *base,
                  const double *d_rhs, double tol, snac_options *best, snac_tune_report *report, void *stream);

/* ---- Kernel statistics (tracing) ---- */

/* Per-kernel counters of a plan: launches (always counted), and with profiling enabled the summed
 * CUDA-event duration of those launches, measured on the stream they were launched on. bytes and
 * flops are the algorithmic DRAM bytes and floating-point operations of the counted launches (the
 * minimum the operation must move / compute, not a hardware counter). name is a static string. */
typedef struct {
  const char *name;
  int64_t launches;
  double ms;
  double bytes;
  double flops;
} snac_kernel_stat;

/* enable != 0: record a CUDA event pair around every kernel launch of the plan (default off). */
int snac_plan_set_profiling(snac_plan *plan, int32_t enable);

/* Copy up to n per-kernel statistics into h_out; *count receives the number of kernel kinds. */
int snac_plan_kernel_stats(const snac_plan *plan, snac_kernel_stat *h_out, int32_t n, int32_t *count);

/* Zero the per-kernel statistics. */
int snac_plan_reset_stats(snac_plan *plan);

/* ---- Stages of the solve, one call each (the same kernels the solve uses). ---- */

/* d_out = A d_p, the 3-D operator of Eq. 8 (float64 3-D fields). */
int snac_apply_operator(snac_plan *plan, const double *d_p, double *d_out, void *stream);

/* d_r = d_rhs - A d_p (float64 3-D fields); h_norms[0] = ||r||_2^2, h_norms[1] = ||rhs||_2^2. */
int snac_residual(snac_plan *plan, const double *d_rhs, const double *d_p, double *d_r, double *h_norms,
                  void *stream);

/* The same residual in float-float arithmetic, rounded to FP32: the pass that mixed plans use for
 * their intermediate defect-correction steps (Eq. 8). d_rhs, d_p: float64 3-D fields; d_r: float32
 * 3-D field in the same layout. Each float64 operand is split into two floats (47 significant bits)
 * and the stencil is summed in float-float arithmetic, so |r - (f - A p)| stays below a few units of
 * 2^-47 (|f| + sum |c p|) per cell before the final rounding to FP32; no FP64 instruction runs per
 * cell. Operands below 2^-103 in magnitude count as zero; operands beyond the FP32 range give a
 * non-finite r. h_norms[0] = ||r||^2, h_norms[1] = ||rhs||^2, summed from FP32 squares (for fields
 * whose values lie within about 1e-15 .. 1e15). Works on plans of either precision. */
int snac_residual_ff(snac_plan *plan, const double *d_rhs, const double *d_p, float *d_r, double *h_norms,
                     void *stream);

/* Forward transform along z (Table 1 F, Algorithm 1 first loop): d_in float64 3-D field ->
 * d_modes mode-space field of the plan's inner type. */
int snac_forward_transform(snac_plan *plan, const double *d_in, void *d_modes, void *stream);

/* Backward transform and update (Algorithm 1 third loop): d_p += F^-1(d_modes), where F^-1 is the
 * backward transform of Table 1 divided by theta; d_modes of the plan's inner type. */
int snac_backward_update(snac_plan *plan, const void *d_modes, double *d_p, void *stream);

/* d_out = (A_xy + lambda_q / dz^2) d_u for every wavenumber q: the reduced operator of Eq. 9 on
 * mode-space fields of the plan's inner type. */
int snac_mode_operator(snac_plan *plan, const void *d_u, void *d_out, void *stream);

/* ncycles V(nu1, nu2) cycles of the reduced equations (Eq. 9) for every wavenumber, in place on
 * d_u, with right-hand side d_f (mode-space fields of the plan's inner type). */
int snac_mode_vcycles(snac_plan *plan, const void *d_f, void *d_u, int32_t ncycles, void *stream);

/* ---- One rank of a solve sharded by wavenumber (App. A, Algorithm 3) ----
 *
 * The x-y cells of the problem are split into pencils (contiguous ranges of the level-0 plane
 * numbering: blocks in id order, [y][x] within a block), each held by one rank with every z plane;
 * the wavenumbers into slabs. A rank transforms its pencil (snac_pencil_forward), the slabs are
 * exchanged (all-to-all, outside the library), each rank solves the reduced equations of its slab
 * (snac_mode_solve on a wavenumber-range plan), the solutions are exchanged back and each rank
 * updates its pencil (snac_pencil_backward_update). The outer FP64 residual of a pencil needs the
 * values of p in the neighbouring columns held by other ranks (snac_pencil_setup lists them).
 * A pencil field is [z][c] (the ncols columns fastest), float64; its mode field [q][c], of the
 * plan's inner type, for every q of the n_z-point transform. The calls accept any plan of the
 * problem (full or wavenumber-range) and return after their work on `stream` is complete. */

/* Forward transform along z (Table 1) of ncols columns: d_in [n_z][ncols] float64 ->
 * d_modes [n_z][ncols] of the plan's inner type (Algorithm 3, first loop). */
int snac_pencil_forward(snac_plan *plan, int64_t ncols, const double *d_in, void *d_modes, void *stream);

/* d_p [n_z][ncols] += F^-1(d_modes) / theta (Algorithm 3, last loop). */
int snac_pencil_backward_update(snac_plan *plan, int64_t ncols, const void *d_modes, double *d_p, void *stream);

/* Describe this rank's pencil: plane cells c0 .. c0 + ncols - 1. The cells of other ranks that the
 * pencil's x-y stencil reaches (across blocks and periodic faces too) are written to h_halo in
 * increasing order, at most max_halo of them (*nhalo receives the count; SNAC_ERR_INVALID_ARG if it
 * exceeds max_halo). The pencil residual reads p as [z][ncols + nhalo]: the pencil's columns, then
 * the halo columns in that order. Replaces the plan's previous pencil. */
int snac_pencil_setup(snac_plan *plan, int64_t c0, int64_t ncols, int64_t *h_halo, int64_t max_halo,
                      int64_t *nhalo);

/* r = (f - fshift) - A p on the pencil (Eq. 8, FP64): d_f, d_r [n_z][ncols]; d_p_ext
 * [n_z][ncols + nhalo]. h_sums[5] receives the pencil's ||r||^2, ||f - fshift||^2, sum V p,
 * sum V (f - fshift), sum V |f - fshift| (V = cell volume). */
int snac_pencil_residual(snac_plan *plan, const double *d_f, const double *d_p_ext, double *d_r, double fshift,
                         double *h_sums, void *stream);

/* Solve the reduced equations (Eq. 9) of the plan's wavenumbers (every one for a full plan, the
 * range of a wavenumber-range plan): d_rhs, d_sol [local q][plane cell] of the plan's inner type.
 * Each wavenumber runs V-cycles from zero until w_q ||r_q||^2 <= target^2 / n_z (w_q the transform's
 * Parseval weight), it stagnates, or max_cycles: the per-mode stopping rule of snac_poisson_solve,
 * which makes the 3-D residual after the update at most `target` over all ranks together. */
int snac_mode_solve(snac_plan *plan, const void *d_rhs, void *d_sol, double target, void *stream);

/* Singular problems (see snac_poisson_solve): shift the wavenumber-0 plane of d_sol by a constant so
 * that the updated p keeps a zero volume-weighted mean, given sum_vp = sum V p of the current p over
 * the whole problem (all ranks). A no-op for non-singular problems and for plans that do not hold
 * wavenumber 0. */
int snac_mode_fix_mean(snac_plan *plan, void *d_sol, double sum_vp, void *stream);

/* ---- Allocation-free residual of one block (the paper has no counterpart) ---- */

/* Largest number of cells along any axis that snac_residual_noalloc accepts. */
#define SNAC_NOALLOC_MAX_CELLS_PER_AXIS 4096

/* d_r = d_rhs - A d_p for a single block, with h_norms[0] = ||r||^2 and h_norms[1] = ||rhs||^2:
 * the same result as snac_residual on a one-block plan, for callers that cannot allocate device
 * memory and so cannot create a plan -- programs whose device memory is owned by their own
 * (caching) allocator or capped by a fixed budget, and latency-sensitive loops that cannot afford the
 * device-wide synchronisation that cudaMalloc and cudaFree imply. Nothing is allocated: the scratch
 * (cell widths, operator coefficients, per-CTA partial sums; about 2.5 MB) is a fixed array in the
 * library's device image, present on every GPU that loads the library until the process exits.
 * block: one block, faces SNAC_BC_DIRICHLET / _NEUMANN / _PERIODIC only (no connectivity), at most
 * SNAC_NOALLOC_MAX_CELLS_PER_AXIS cells per axis (SNAC_ERR_INVALID_ARG otherwise), uniform along z
 * (SNAC_ERR_LAYOUT otherwise). d_rhs, d_p, d_r: device float64 fields [z][y][x]; h_norms: host.
 * Every call looks up the scratch's address on the current device (cudaGetSymbolAddress), copies
 * the cell widths from host memory and waits for `stream`: do not call it while `stream` is being
 * captured into a CUDA graph. Every call uses the same scratch, so calls whose work overlaps on the
 * GPU (other streams, other host threads) race: issue them one after another. Returns after the work
 * on `stream` is complete. */
int snac_residual_noalloc(const snac_block *block, const double *d_rhs, const double *d_p, double *d_r,
                          double *h_norms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SNAC_H */
