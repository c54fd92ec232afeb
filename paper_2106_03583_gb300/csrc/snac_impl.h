// Internal declarations of the CUDA Poisson solver library (libsnac.so).
//
// Data model on the device (one plan):
//   * a "plane" is the set of x-y cells of all blocks at one multigrid level, numbered block by
//     block, [y][x] within a block (x fastest); block b starts at cell off[b];
//   * per level: a block table (BlockDev), a tile table (32x8-cell tiles, never straddling blocks),
//     1-D coefficient arrays along x (per block column) and y (per block row), prolongation and
//     restriction weights; the 2-D operator of a cell is separable into these 1-D pieces;
//   * mode-space fields are [q][plane cell] in the inner type T (double or float);
//   * 3-D caller fields are [block][z][y][x] in double.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <string>
#include <vector>

#include "snac.h"

namespace snac {

enum Kind { KIND_PP = 0, KIND_NN = 1, KIND_DD = 2, KIND_ND = 3, KIND_DN = 4 };

constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int TILE_THREADS = TILE_X * TILE_Y;
constexpr int MAX_NZ = 4096;
// Columns per transform CTA: two half-length complex buffers of TC columns stay within 128 KB of
// shared memory, so TC halves as n_z doubles beyond 1024 (FP64: 8, 4, 2; FP32: 16, 8, 4).
inline int transform_columns(int nz, bool fp64) {
  const int base = fp64 ? 8 : 16;
  return nz <= 1024 ? base : (nz <= 2048 ? base / 2 : base / 4);
}
constexpr int MAX_COARSE = 256;
// The bottom of the V-cycle (kern_bottom.cu): levels from the first one (below level 0) whose
// planes, with all coarser ones, fit in one CTA's shared memory, run in one launch per round.
constexpr int BOTTOM_THREADS = 512;
constexpr int BOTTOM_MAX_LEVELS = 8;
constexpr int BOTTOM_MAX_CELLS = 8192;          // plane cells of the sub-cycle's top level
constexpr int BOTTOM_MAX_SMEM = 200 * 1024;     // dynamic shared memory of one CTA
constexpr int MEAN_CTAS = 2 * 152;  // CTAs (so partials) of the grid-stride plane reductions: fixed, for a fixed summation order
constexpr int SUM_SLOTS = 16;     // d_sums / h_sums: [0..3] residual or pre-pass, [4..7] mean fix
constexpr int SUM_NONZERO = 8;    // d_sums slot of the pre-pass's nonzero-guess flag  // CTAs of the grid-stride reductions over one mode plane
constexpr int FTILE_X = 52;         // tile of the fused multigrid kernels (64x64 window with the halo)
constexpr int FTILE_Y = 52;
constexpr int FUSED_MIN_BLOCK = 8;   // fused kernels on levels whose blocks are all this wide (>= the halo)

// Faces are numbered W, E, S, N = 0..3 (x lower, x upper, y lower, y upper).
struct BlockDev {
  long long off;  // first cell of the block in the plane
  int nx, ny;
  int xo, yo;     // offsets of the block's columns / rows in the level's 1-D arrays
  int nbr[4];     // connected block across each face, -1 on a physical (Dirichlet/Neumann) face
  int par;        // colour of cell (0,0): parity of its global index-space position
  int pad;
};

// Where a block's cells sit in the caller's 3-D arrays ([z][y][x] per block, blocks concatenated):
// cell (i, j, k) of the internal axes (plane axes i, j; homogeneous axis k) is at off3 + i s[0] +
// j s[1] + k s[2].
struct CallerBlk {
  long long off3;
  long long s[3];
};

struct TileDev {
  int b, x0, y0, pad;
};

// 1-D operator piece of one column (x) or row (y): coupling to the lower and upper neighbour
// (zero on a physical face), contribution to the diagonal, and the cell width.
template <typename T>
struct Coef {
  T lo, hi, d, w;
};

// Prolongation weights of one fine column/row: e_f gets self*e_C + nbr*e_X per axis (plus e_C).
template <typename T>
struct PW {
  T self, nbr;
};

template <typename T>
struct LevelView {
  const BlockDev* blk;
  const TileDev* tiles;
  const Coef<T>* cx;
  const Coef<T>* cy;
  const PW<T>* px;  // weights for prolongation into this level (fine side); px[i].self includes the +1 of the parent
  const PW<T>* py;
  const T* rx;      // restriction weights: fine width / parent width
  const T* ry;
  long long ncell;
  int ntiles;
  int nblk;
  const T* dxy;     // x-y part of the diagonal of every plane cell, cx.d + cy.d (plain order)
  const T* wr;      // restriction weight of every plane cell, rx * ry (levels with a coarser one)
  const T* wp;      // prolongation weight of the parent, 1 + self_x + self_y (levels with a coarser one)
};

// One level of the bottom sub-cycle (kern_bottom.cu), in a device table built with the plan.
template <typename T>
struct BottomLevel {
  LevelView<T> L;
  const double* invd;  // FP64 smoothed levels: per-mode 1/diag (colour-split order if the plan is scaled)
  int su, sf, sinv;    // element offsets of u, f and 1/diag in the kernel's shared memory (-1: f read
                       // from the level's global array, 1/diag absent on the coarsest level)
  int sblk;            // byte offset of the level's block table copy in shared memory
};

// Host-side description of one level.
struct HostLevel {
  int nblk = 0;
  std::vector<BlockDev> blk;
  std::vector<TileDev> tiles;
  std::vector<Coef<double>> cx, cy;
  std::vector<PW<double>> px, py;
  std::vector<double> rx, ry;
  long long ncell = 0;
  // device copies
  BlockDev* d_blk = nullptr;
  TileDev* d_tiles = nullptr;
  Coef<double>* d_cx64 = nullptr;
  Coef<double>* d_cy64 = nullptr;
  Coef<float>* d_cx32 = nullptr;
  Coef<float>* d_cy32 = nullptr;
  PW<double>* d_px64 = nullptr;
  PW<double>* d_py64 = nullptr;
  PW<float>* d_px32 = nullptr;
  PW<float>* d_py32 = nullptr;
  double* d_rx64 = nullptr;
  double* d_ry64 = nullptr;
  float* d_rx32 = nullptr;
  float* d_ry32 = nullptr;
  double* d_dxy64 = nullptr;
  float* d_dxy32 = nullptr;
  double* d_wr64 = nullptr;
  float* d_wr32 = nullptr;
  double* d_wp64 = nullptr;
  float* d_wp32 = nullptr;
  void* d_u = nullptr;  // mode-space iterate, n_z x ncell of the inner type
  void* d_f = nullptr;  // mode-space right-hand side
  double* d_invd = nullptr;  // FP64 plans, smoothed levels: 1 / (A_xy + sigma_q)_cc per mode and cell
  bool fused = false;        // this level runs the fused tile kernels
  void* d_u2 = nullptr;      // fused levels: second iterate buffer (the tiles read one, write the other)
  std::vector<TileDev> ftiles;  // FTILE_X x FTILE_Y tiles (fused levels)
  void* d_ftab = nullptr;       // per fused tile: its FusedTab<T> (T = the level's arithmetic type)
};

// A chunk of up to TCOLS consecutive columns (cells of one plane) of one block, for the transforms.
struct ChunkDev {
  int b, c0, ncol, pad;
};

struct TwiddleOffsets {
  int fft, twn, tw2n, tw4a, tw4b, total;
};

// Kernel kinds counted by the tracing facility.
enum KernelKind {
  K_FIELD3D = 0, K_REDUCE, K_FIX_MEAN, K_SHIFT, K_FORWARD, K_BACKWARD, K_SMOOTH, K_RESTRICT, K_PROLONG,
  K_COARSE, K_MODE_RESID, K_MODE_REDUCE, K_MODE_APPLY, K_FDOWN, K_FUP, K_BOTTOM, K_FIELD3D_FF, K_ONCHIP, K_FWD_ONCHIP, K_COUNT
};

struct KernelStat {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};

struct PendingEvent {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace snac

struct snac_plan {
  int device = 0;
  int sms = 152;             // multiprocessors of the device (grid sizing)
  int precision = SNAC_FP64;
  int nu1 = 2, nu2 = 2, max_outer = 20, max_cycles = 40, max_coarse = 64;
  double inner_reduction = 0.0;  // 0: automatic (resolved at plan creation)
  double shift = 0.0;  // Helmholtz shift (<= 0), included in sigma and in the residual's diagonal
  int fused = -1;
  // FP64 plans without fused levels keep the right-hand side of every smoothed level (all but the
  // coarsest) divided by the diagonal, which saves one FP64 operation per smoothing update
  bool scaled_f = false;
  int bottom = -1;  // first level of the one-launch bottom sub-cycle (kern_bottom.cu), -1: none
  void* d_bottom = nullptr;  // its BottomLevel<inner type> table
  // the whole hierarchy fits in one CTA's shared memory: each wavenumber's solve runs on chip,
  // its convergence decided on the device (kern_bottom.cu, k_onchip)
  bool onchip = false;
  int onchip_opt = 0;         // snac_options.onchip
  int bottom_cells = 0;       // snac_options.bottom_cells
  void* d_onchip = nullptr;   // BottomLevel<inner type> table from level 0
  double* d_pweight = nullptr;
  int* h_cycles = nullptr;    // per wavenumber: V-cycles of the last on-chip solve (mapped pinned)
  int* dh_cycles = nullptr;
  int* d_fused = nullptr;     // the fused transform + on-chip launch's counters: next item, chunks done
  int* h_wait = nullptr;      // set by that launch when a bounded wait gave up (mapped pinned)
  int* dh_wait = nullptr;
  int nblk = 0;
  int nz = 0;    // wavenumbers held in mode space (q0 .. q0 + nz - 1)
  int nzt = 0;   // cells along the homogeneous axis: the transform length, the 3-D field's z planes
  int q0 = 0;    // first wavenumber held (nonzero only in a wavenumber-range plan)
  bool ranged = false;  // a wavenumber-range plan: mode space only, no 3-D field
  double dz = 0.0;
  int kind = 0;
  double theta = 1.0;
  bool singular = false;
  long long n3 = 0;  // cells of the 3-D field
  double vol_total = 0.0;
  double area_total = 0.0;
  std::vector<long long> blk_off3;  // 3-D offset of each block
  std::vector<snac::CallerBlk> cblk;  // caller offset and strides of each block's internal axes
  snac::CallerBlk* d_cblk = nullptr;
  std::vector<snac::HostLevel> lev;
  // z direction
  std::vector<snac::Coef<double>> cz;
  snac::Coef<double>* d_cz = nullptr;
  float4* d_czff = nullptr;  // per plane: {lo, hi} of cz as rounded float pairs (float-float residual)
  // level-0 coefficients of the float-float residual (mixed plans) as rounded float pairs:
  // {lo, hi} of every x column and y row entry, and the full diagonal cx.d + cy.d + cz.d per cell
  float4* d_cxff = nullptr;
  float4* d_cyff = nullptr;
  float2* d_dgff = nullptr;
  // eigenvalue shifts lambda_q / dz^2 and the Parseval weight of every mode
  std::vector<double> sigma, pweight;
  double* d_sigma64 = nullptr;
  float* d_sigma32 = nullptr;
  // coarsest level: S = V^1/2 A V^-1/2 = Q diag(Lam) Q^T
  int nc = 0;
  int null_index = -1;
  double* d_Q = nullptr;      // nc x nc, row-major, column k = eigenvector k
  double* d_QT = nullptr;     // its transpose (row k = eigenvector k)
  double* d_lam = nullptr;    // nc
  double* d_sqa = nullptr;    // sqrt(area) of the coarsest cells
  int* d_singular_mode = nullptr;  // per mode: 1 if the reduced system is singular
  // transforms
  snac::TwiddleOffsets tw{};
  double* d_tw64 = nullptr;  // double2 table
  float* d_tw32 = nullptr;   // float2 table
  int tc64 = 8, tc32 = 16;  // columns per transform CTA (transform_columns)
  std::vector<snac::ChunkDev> chunks64, chunks32;
  snac::ChunkDev* d_chunks64 = nullptr;
  snac::ChunkDev* d_chunks32 = nullptr;
  double* d_area0 = nullptr;  // area of every level-0 cell
  // scratch
  double* d_r3 = nullptr;       // 3-D residual
  double* d_partial = nullptr;  // per-CTA partial sums
  int npartial = 0;
  double* d_sums = nullptr;     // reduced sums (SUM_SLOTS)
  int* d_flag = nullptr;        // nonzero-initial-guess flag of the pre-pass
  double* d_mode_part = nullptr;  // per-mode, per-tile partial sums of squares
  double* d_mode_norm2 = nullptr; // per-mode ||r_q||^2
  int* d_active = nullptr;
  // pinned host buffers of the solve's control data, mapped into the device address space (dh_*):
  // kernels move them, so a solve issues no copy-engine work and never queues behind another
  // stream's bulk host copies
  double* h_sums = nullptr;
  double* h_mode_norm2 = nullptr;
  int* h_active = nullptr;
  double* dh_sums = nullptr;
  double* dh_mode_norm2 = nullptr;
  int* dh_active = nullptr;
  int* d_check = nullptr;         // modes whose residual norm is due after a round (predictive checks)
  int* h_check = nullptr;
  int* dh_check = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  // sharded solves: transform tables of a pencil of pen_tcols columns (one pseudo-block)
  long long pen_tcols = -1;
  snac::BlockDev* d_pen_tblk = nullptr;
  snac::CallerBlk* d_pen_tcb = nullptr;
  std::vector<snac::ChunkDev> pen_ch64, pen_ch32;
  snac::ChunkDev* d_pen_ch64 = nullptr;
  snac::ChunkDev* d_pen_ch32 = nullptr;
  std::vector<void*> pen_tallocs;
  // the pencil of the pencil residual: plane cells pen_c0 .. pen_c0 + pen_ncols - 1 and its halo
  long long pen_c0 = 0, pen_ncols = 0, pen_nhalo = 0;
  int* d_pen_cell = nullptr;      // per pencil cell: block, i, j, then the p_ext columns of W, E, S, N
  double* d_pen_part = nullptr;   // per-CTA partial sums (8 per CTA)
  int pen_nparts = 0;
  std::vector<void*> pen_allocs;
  // results
  snac_solve_info info{};
  std::vector<int32_t> mode_cycles;
  // tracing
  bool profiling = false;
  // One V-cycle round (all levels + the per-mode norms) captured as a CUDA graph per number of active
  // modes, replayed on the solve's stream; `delta` = the launch statistics of one round.
  struct RoundGraph {
    cudaGraphExec_t exec = nullptr;
    snac::KernelStat delta[snac::K_COUNT];
  };
  std::map<int, RoundGraph> round_graphs;
  bool graphs = true;                   // off after a failed capture
  cudaStream_t capture_stream = nullptr;  // private stream the rounds are captured on
  snac::KernelStat kstats[snac::K_COUNT];
  std::vector<snac::PendingEvent> pending;
  std::vector<cudaEvent_t> event_pool;
};

namespace snac {

// ---- launchers (field kernels: 3-D FP64 residual and reductions) ----
// mode 0: r = (f - fshift) - A p; d_sums = {||r||^2, ||f - fshift||^2 if need_f2, sum V p if need_vp}
// mode 1: r = A p
cudaError_t launch_field3d(snac_plan* P, int mode, const double* f, const double* p, double* r, double fshift,
                           bool need_f2, bool need_vp, cudaStream_t s);
// The same residual (mode 0) in float-float arithmetic, written in FP32 (mixed plans' intermediate
// defect-correction steps; kern_ffresid.cu). fscale: the RMS of f (any positive value; it sets the
// power-of-two scaling of the FP32 squares).
cudaError_t launch_field3d_ff(snac_plan* P, const double* f, const double* p, float* r, double fshift, double fscale,
                              bool need_f2, bool need_vp, cudaStream_t s);
// d_sums = {sum V f, sum V |f|, ||f||^2, sum f} (V sums only for singular plans) and
// d_sums[SUM_NONZERO] = 1 if p has a nonzero entry, else 0
cudaError_t launch_prepass(snac_plan* P, const double* f, const double* p, cudaStream_t s);
// reduce d_partial[npart][4] into out[4] (device)
cudaError_t launch_reduce_partials(snac_plan* P, int npart, double* out, cudaStream_t s);
// make the update of the singular mode 0 keep the volume-weighted mean of p at zero
cudaError_t launch_fix_mean(snac_plan* P, void* u0, cudaStream_t s);
// p -= c (c read from device d_c)
cudaError_t launch_shift(snac_plan* P, double* p, const double* d_c, cudaStream_t s);

// ---- transforms ----
// modes = F(in3 - shift0) along z (shift0 != 0 only for the kinds with a zero eigenvalue)
// split: write the modes in colour-split order (the plan's own level-0 f of a scaled FP64 plan).
cudaError_t launch_forward(snac_plan* P, const double* in3, void* modes, double shift0, bool split, cudaStream_t s);
// The same from an FP32 3-D field in the caller layout (the float-float residual's output; mixed plans).
cudaError_t launch_forward_f32(snac_plan* P, const float* in3, void* modes, cudaStream_t s);
// Level-0 mode planes from plain to colour-split order.
cudaError_t launch_to_split(snac_plan* P, const double* src, double* dst, cudaStream_t s);
// p3 += F^-1(modes) / theta; subtract: p3 -= F^-1(modes) / theta (takes a correction back)
cudaError_t launch_backward_update(snac_plan* P, const void* modes, double* p3, cudaStream_t s, bool subtract = false);
// Pencils of a sharded solve ([z][c] fields of ncols columns): forward transform, backward update.
cudaError_t launch_pencil_forward(snac_plan* P, long long ncols, const double* in, void* modes, cudaStream_t s);
cudaError_t launch_pencil_backward(snac_plan* P, long long ncols, const void* modes, double* p, cudaStream_t s);

// ---- multigrid ----
cudaError_t launch_mode_operator(snac_plan* P, const void* u, void* out, cudaStream_t s);
// 1 / diagonal of every mode's reduced operator on every smoothed level (FP64 plans), once per plan
cudaError_t launch_inverse_diagonals(snac_plan* P, cudaStream_t s);
// one V-cycle of the active modes on the plan's level buffers (level 0: d_u / d_f)
// skip_first0: level 0's first colour-0 half-sweep of this cycle was done by launch_check_sweep.
cudaError_t launch_vcycle(snac_plan* P, int nactive, cudaStream_t s, bool skip_first0 = false);
// Scaled FP64 plans: the next cycle's first colour-0 half-sweep at level 0 for the active modes, with
// the residual norms (before it) of the ncheck modes in d_check (ascending) into d_mode_norm2.
cudaError_t launch_check_sweep(snac_plan* P, int nact, int ncheck, cudaStream_t s);
// per-mode ||f - A u||^2 at level 0 for the active modes -> d_mode_norm2[q]; after_cycle: u is the
// result of a V-cycle (post-smoothing ended on black, so only red cells carry a residual); otherwise
// u is zero and the norm is that of f
// zero_u (with !after_cycle): also set the listed modes' level-0 iterate to zero in the same pass.
cudaError_t launch_mode_norms(snac_plan* P, int nactive, bool after_cycle, cudaStream_t s, const int* d_list = nullptr,
                              bool zero_u = false);
// The V-cycle from level P->bottom down to the coarsest and back, one CTA per active mode.
cudaError_t launch_bottom(snac_plan* P, int nact, cudaStream_t s);
// Plans whose hierarchy fits on chip: the complete solve of each active wavenumber from a zero
// iterate, one CTA each, to ||r_q||^2 <= target^2 / (n_z w_q) (or stagnation, or max_cycles);
// per-mode cycles into dh_cycles and final ||r_q||^2 into dh_mode_norm2.
cudaError_t launch_onchip(snac_plan* P, int nact, double target, cudaStream_t s);
// The same for the wavenumbers of several plans (one precision) in one persistent launch; h_items
// (plan index, wavenumber), targets per plan; d_scratch of onchip_batch_scratch(nplans, nitems) bytes.
size_t onchip_batch_scratch(int nplans, int nitems);
// The forward transform of in3 (FP64, or FP32 with in_f32; shift0: mean removed from f at k = 0)
// and the on-chip solves of every wavenumber in one persistent launch (kern_bottom.cu): a solve
// waits for its plan's transform chunks, at most wait_s seconds (then *h_wait = 1 and the solve is
// skipped). extra_need > 0 only for the self-test of the timeout (a count nothing reaches).
bool fused_ready(const snac_plan* P);
cudaError_t launch_fwd_onchip(snac_plan* P, const void* in3, bool in_f32, double shift0, double target, double wait_s,
                              int extra_need, cudaStream_t s);
struct FusedInput {
  const void* in3;
  bool in_f32;
  double shift0;
};
size_t fwd_onchip_batch_scratch(int nplans, int nitems);
cudaError_t launch_fwd_onchip_batch(snac_plan* const* plans, const FusedInput* inputs, const double* targets,
                                    int nplans, double wait_s, void* d_scratch, int sms, cudaStream_t s);
constexpr double WAIT_LIMIT_S = 1.0;  // bound of every device-side wait of a solve
cudaError_t launch_onchip_batch(snac_plan* const* plans, const double* targets, int nplans, const int2* h_items,
                                int nitems, void* d_scratch, int sms, cudaStream_t s);
// Shared-memory layout of that kernel when it starts at level lb, for inner type width w: per level
// the element offsets of u, f (-1: the top level's f stays in global memory, as in FP64 plans, so
// that two CTAs fit on one multiprocessor) and 1/diag (-1 on the coarsest level), the byte offset of
// the level's block table copy; the byte offset of the coarsest solve's vectors and the total.
struct BottomLayout {
  int su[BOTTOM_MAX_LEVELS], sf[BOTTOM_MAX_LEVELS], sinv[BOTTOM_MAX_LEVELS], sblk[BOTTOM_MAX_LEVELS];
  int coarse_off;
  size_t bytes;
};
BottomLayout bottom_layout(const snac_plan* P, int lb, size_t w);
// Small transfers through mapped pinned memory, done by one-CTA kernels (no copy engine).
cudaError_t launch_to_host(const double* d_src, double* dh_dst, int n, cudaStream_t s);
cudaError_t launch_from_host(const int* dh_src, int* d_dst, int n, cudaStream_t s);
cudaError_t launch_fill(double* d, int n, double v, cudaStream_t s);

// fused FP32 levels: smoothing + residual + restriction (down), prolongation + smoothing (+ level-0
// residual norm partials into d_mode_part) (up)
cudaError_t launch_fused_down(snac_plan* P, int l, int nact, bool zero_u, bool zero_coarse, cudaStream_t s);
cudaError_t launch_fused_up(snac_plan* P, int l, int nact, bool norms, cudaStream_t s);

int plan_inner_size(const snac_plan* P);  // bytes of the inner type
// the block-layout checks of plan creation (sizes, widths, face kinds, z pair, connectivity)
int check_layout(int nblocks, const snac_block* blocks, int homog_axis);

// Counts one launch of `kind` with its algorithmic bytes / flops; with profiling on, brackets it
// with a CUDA event pair on stream s (construct just before the launch, destroy just after).
class LaunchScope {
 public:
  LaunchScope(snac_plan* P, int kind, double bytes, double flops, cudaStream_t s);
  ~LaunchScope();

 private:
  snac_plan* P_;
  int kind_;
  cudaStream_t s_;
  cudaEvent_t b_ = nullptr;
};

// Accumulate the durations of completed event pairs (call after a stream synchronisation).
void profile_resolve(snac_plan* P);
void profile_release(snac_plan* P);

}  // namespace snac
