// Fused multigrid tile kernels (the reduced equations of Eq. 9; Algorithm 1, second loop). On
// GB300 the FP32 multigrid is bound by memory latency and instruction issue, so each level of a
// V-cycle runs as two kernels that keep a tile of one mode's plane on chip:
//
//   k_fdown: load u, f on a 52x52 tile plus a halo of FUSED_HALO = 6 cells (a 64x64 window) -> nu1
//            red-black Gauss-Seidel sweeps -> store the tile's u -> residual on its red cells ->
//            area-weighted restriction into the coarse right-hand side;
//   k_fup:   load u, f on the window and the coarse correction around it -> three-point
//            prolongation and correction -> nu2 sweeps -> store the tile's u (on level 0 also the
//            per-mode sums of squared residuals).
//
// A CTA copies its tile's tables once (FusedTab: coefficients, weights and the plane offsets of
// every window row and column, built on the host), derives from them each thread's own cell table
// (plane offsets of its cells and their diagonals without the shift), and then runs the tile for a
// run of consecutive active modes. While it smooths one mode, the next mode's cells (and, going up, its coarse
// correction window) stream into shared memory with per-thread asynchronous copies (cp.async), so
// the global-load latency of a mode is hidden behind the previous mode's sweeps.
//
// Registers. Warp w (of 8, 256 threads per CTA) holds window rows 8w..8w+7, lane k holds columns
// 2k (parity 0) and 2k+1 (parity 1) of those rows: u, f and 1/diag of 16 cells per thread, and the
// y couplings of its rows. The rows of one colour in a half-sweep are independent, so each warp has
// eight updates in flight (two CTAs of 8 warps per multiprocessor at up to 128 registers measured
// faster than 16 warps of four rows at 64 registers). In a row the cells of one colour
// all have the same column parity, so a colour update of a row is one cell per lane: the west/east
// neighbours come from the thread itself or from one warp shuffle, the south/north neighbours from
// the thread's own registers; only the first and last row of each strip pass through shared memory
// (once per half-sweep, only the colour that changed). Coarse cells are exactly (row pair) x
// (column pair): restriction and prolongation stay in registers too.
//
// Exactness. Every window cell is updated in every half-sweep of its colour. The neighbours of an
// edge cell beyond the window are unknown (the update reads zero or the cell's own pair instead), so
// wrong values enter from the edge one cell per half-sweep -- as stale ones would if the edge were
// left alone, and without a per-cell test in the update. After 2 nu <= FUSED_HALO - 2
// half-sweeps the tile and the ring around it (used by the residual) equal the global Gauss-Seidel
// sweep. Window cells outside the tile's block belong to the connected blocks and use that block's
// coefficients, so sweeps across block interfaces are exact too. Cells with no owner (beyond a
// physical face, a re-entrant corner, or past the clipped window of a ragged tile) carry f = 0 and
// a zero inverse diagonal, so they stay 0; their coupling coefficients are 0. The halo must fit in
// the neighbouring blocks: levels whose blocks are all at least FUSED_MIN_BLOCK cells wide.
//
// Each tile reads one iterate buffer and writes the other (neighbouring CTAs store their smoothed
// tiles while this one may still be loading its halo).
#include <algorithm>

#include "fused_tab.h"
#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
namespace {

constexpr int FH = FUSED_HALO;
constexpr int WN = FWN;
constexpr int HW = FHW;
constexpr int CW = FCW;
constexpr int RPW = 8;  // rows per warp
constexpr int FWARPS = WN / RPW;
constexpr int FTHREADS = 32 * FWARPS;
constexpr int FMINB = 2;  // CTAs per multiprocessor
static_assert(FTILE_X == FTILE_Y && HW == 32 && FWARPS * RPW == WN, "the fused kernels assume a 64x64 window");
static_assert(FH % 2 == 0 && 2 * 2 <= FH - 2, "nu <= 2 sweeps must stay exact inside the halo");

template <typename T>
struct alignas(2 * sizeof(T)) Pair {
  T a, b;
};

template <typename T>
struct Shared {
  FusedTab<T> tab;
  Pair<T> stage[RPW][2][FTHREADS];  // next mode's u, f column pairs, each thread's own slots (0: no owner)
  Pair<T> diag[RPW][FTHREADS];      // diagonal of the thread's cells without the shift (+inf: no owner)
  int goff[RPW][FTHREADS];          // plane offset of the thread's column pair in each of its rows (-1: none)
  int coff[CW * CW];                // plane offset of each coarse window cell (-1: no owner; k_fup)
  T halo[FWARPS][2][2][HW];         // [warp][first/last row][parity][lane]
  T e[2][CW][CW];                   // coarse correction around the tile, this mode and the next (k_fup)
  double wsum[FWARPS];
};
static_assert(2 * sizeof(Shared<float>) + 2048 <= 228 * 1024, "two FP32 CTAs per multiprocessor");

// Per-thread asynchronous global -> shared copies (completion is tracked by the issuing thread).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(src), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Per-thread state: rows RPW w .. RPW w + RPW - 1 of window columns 2k, 2k+1.
template <typename T>
struct Cells {
  T u[RPW][2], f[RPW][2], inv[RPW][2];
};

// Copy the tile's tables into shared memory (16-byte words).
template <typename T>
__device__ __forceinline__ void copy_tab(Shared<T>& S, const FusedTab<T>* __restrict__ tab) {
  static_assert(sizeof(FusedTab<T>) % 16 == 0, "FusedTab is copied in 16-byte words");
  const uint4* src = reinterpret_cast<const uint4*>(tab);
  uint4* dst = reinterpret_cast<uint4*>(&S.tab);
  for (int i = threadIdx.x; i < (int)(sizeof(FusedTab<T>) / 16); i += FTHREADS) dst[i] = src[i];
}

// Reciprocal of the diagonal: FP32 levels use the hardware approximation (relative error below
// 2^-22; the FP32 smoother only needs to converge, the FP64 outer iteration fixes the rest), FP64
// levels the exact quotient.
__device__ __forceinline__ float recip(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Each thread's own table, derived once per CTA from the tile's: plane offsets of its column pair
// in its RPW rows, and the shift-free diagonals of its cells. Cells with no owner get offset -1,
// diagonal +inf (so 1/diag = 0) and zero staging slots, which no copy ever overwrites. With
// `coarse`, also the offsets of the coarse window, whose unowned cells are zeroed in both buffers.
template <typename T>
__device__ __forceinline__ void thread_tables(Shared<T>& S, bool coarse) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const FusedTab<T>& tb = S.tab;
  const int col = tb.col[lane], rx = tb.colrx[lane];
  int off[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int wj = RPW * warp + r;
    const int ro = tb.rowoff[rx][wj];
    off[r] = -1;
    if (col != FUSED_NONE && ro != FUSED_NONE) {
      off[r] = ro + col;  // even: block sizes and offsets are even
      const int ry = tb.rowry[wj];
      const T yd = tb.yd[rx][wj];
      S.diag[r][threadIdx.x] = Pair<T>{tb.xd[ry][0][lane] + yd, tb.xd[ry][1][lane] + yd};
    } else {
      S.diag[r][threadIdx.x] = Pair<T>{(T)INFINITY, (T)INFINITY};
      S.stage[r][0][threadIdx.x] = Pair<T>{0, 0};
      S.stage[r][1][threadIdx.x] = Pair<T>{0, 0};
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) S.goff[r][threadIdx.x] = off[r];
  if (coarse) {
    for (int idx = threadIdx.x; idx < CW * CW; idx += FTHREADS) {
      const int cj = idx / CW, ci = idx % CW;
      const int cc = tb.ccol[ci];
      const int ro = tb.crowoff[tb.ccolrx[ci]][cj];
      const bool own = cc != FUSED_NONE && ro != FUSED_NONE;
      S.coff[idx] = own ? ro + cc : -1;
      if (!own) S.e[0][cj][ci] = S.e[1][cj][ci] = (T)0;
    }
  }
}

// Start the copies of the thread's owned cells of one mode (u if asked, and f) into its own
// staging slots.
template <typename T>
__device__ __forceinline__ void prefetch_cells(Shared<T>& S, long long base, const T* __restrict__ u,
                                               const T* __restrict__ f, bool load_u) {
  int off[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) off[r] = S.goff[r][threadIdx.x];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    if (off[r] < 0) continue;
    const long long a = base + off[r];
    if (load_u) cp_async<2 * sizeof(T)>(&S.stage[r][0][threadIdx.x], u + a);
    cp_async<2 * sizeof(T)>(&S.stage[r][1][threadIdx.x], f + a);
  }
}

// The thread's 2 RPW cells of u (zero if asked), f and 1/diag, from its completed staging slots.
template <typename T>
__device__ __forceinline__ void take_cells(Cells<T>& C, const Shared<T>& S, bool zero_u, T sg) {
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const Pair<T> v = zero_u ? Pair<T>{0, 0} : S.stage[r][0][threadIdx.x];
    const Pair<T> g = S.stage[r][1][threadIdx.x];
    const Pair<T> d = S.diag[r][threadIdx.x];
    C.u[r][0] = v.a;
    C.u[r][1] = v.b;
    C.f[r][0] = g.a;
    C.f[r][1] = g.b;
    C.inv[r][0] = recip(d.a + sg);
    C.inv[r][1] = recip(d.b + sg);
  }
}

// Start the copies of one mode's coarse correction window into S.e[buf] (its unowned cells stay 0).
template <typename T>
__device__ __forceinline__ void prefetch_coarse(Shared<T>& S, int buf, long long cbase, const T* __restrict__ uc) {
  T* e = &S.e[buf][0][0];
  for (int idx = threadIdx.x; idx < CW * CW; idx += FTHREADS) {
    const int o = S.coff[idx];
    if (o >= 0) cp_async<sizeof(T)>(e + idx, uc + cbase + o);
  }
}

// The strip's first and last rows, both parities.
template <typename T>
__device__ __forceinline__ void write_halo(Shared<T>& S, const Cells<T>& C) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  S.halo[warp][0][0][lane] = C.u[0][0];
  S.halo[warp][0][1][lane] = C.u[0][1];
  S.halo[warp][1][0][lane] = C.u[RPW - 1][0];
  S.halo[warp][1][1][lane] = C.u[RPW - 1][1];
}

static_assert(RPW % 2 == 0, "a strip's last row has the parity of its second row");

// After a half-sweep whose first row updated parity PA: only the cells of that colour changed, the
// first row's at parity PA and the last row's at parity PA ^ 1. The next half-sweep reads only
// entries of this colour (the neighbours of the other colour), and this half-sweep read only the
// other colour's entries, so one buffer serves both with a barrier between half-sweeps.
template <typename T, int PA>
__device__ __forceinline__ void write_halo_colour(Shared<T>& S, const Cells<T>& C) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  S.halo[warp][0][PA][lane] = C.u[0][PA];
  S.halo[warp][1][PA ^ 1][lane] = C.u[RPW - 1][PA ^ 1];
}

// The strip-edge neighbours a pass over the strip uses when its first row has colour parity PA:
// row 0 reads the south strip's last row at parity PA, row RPW - 1 the north strip's first row at
// parity PA ^ 1 (zero beyond the window).
template <typename T, int PA>
__device__ __forceinline__ void edge_values(const Shared<T>& S, T& south, T& north) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  south = warp > 0 ? S.halo[warp - 1][1][PA][lane] : (T)0;
  north = warp < FWARPS - 1 ? S.halo[warp + 1][0][PA ^ 1][lane] : (T)0;
}

// Gauss-Seidel update of row r of the strip, the colour's cells having column parity P. At the
// window's west and east edges the shuffles return the lane's own pair (see Exactness).
template <typename T, int P>
__device__ __forceinline__ void update_row(Cells<T>& C, FP2<T> cx, FP2<T> cy, int r, T sn, T nn) {
  T w, e;
  if (P == 0) {
    w = __shfl_up_sync(0xffffffffu, C.u[r][1], 1);
    e = C.u[r][1];
  } else {
    w = C.u[r][0];
    e = __shfl_down_sync(0xffffffffu, C.u[r][0], 1);
  }
  T a = cx.a * w;
  a = fma(cx.b, e, a);
  a = fma(cy.a, sn, a);
  a = fma(cy.b, nn, a);
  C.u[r][P] = (C.f[r][P] - a) * C.inv[r][P];
}

// One half-sweep of the strip; P0 = column parity of the colour in the strip's first row. UNI: all
// rows of the strip lie in one region row, so the x coefficients are one pair per parity.
template <typename T, int P0, bool UNI>
__device__ __forceinline__ void half_sweep(Cells<T>& C, Shared<T>& S, const int (&ry)[RPW], const FP2<T> (&cy)[RPW]) {
  const int lane = threadIdx.x & 31;
  constexpr int PA = P0, PB = P0 ^ 1;
  const FusedTab<T>& tb = S.tab;
  T south, north;
  edge_values<T, PA>(S, south, north);
  FP2<T> cxa, cxb;
  if (UNI) {
    cxa = tb.xc[ry[0]][PA][lane];
    cxb = tb.xc[ry[0]][PB][lane];
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    if ((r & 1) == 0) {  // parity PA; never the last row
      const T sn = r > 0 ? C.u[r > 0 ? r - 1 : 0][PA] : south;
      const T nn = C.u[r < RPW - 1 ? r + 1 : 0][PA];
      update_row<T, PA>(C, UNI ? cxa : tb.xc[ry[r]][PA][lane], cy[r], r, sn, nn);
    } else {             // parity PB; never the first row
      const T sn = C.u[r > 0 ? r - 1 : 0][PB];
      const T nn = r < RPW - 1 ? C.u[r < RPW - 1 ? r + 1 : 0][PB] : north;
      update_row<T, PB>(C, UNI ? cxb : tb.xc[ry[r]][PB][lane], cy[r], r, sn, nn);
    }
  }
  write_halo_colour<T, PA>(S, C);
}

// nu red-black sweeps of the whole window. On return the strip-edge rows of the last colour are in
// S.halo (the neighbours of the other colour, for the residuals that follow).
// `after_first_barrier` runs once every thread has passed the barrier that follows the first
// write of the halo rows (all earlier shared-memory reads of the CTA are then complete).
template <typename T, typename Hook>
__device__ void sweeps(Cells<T>& C, Shared<T>& S, int nu, Hook&& after_first_barrier) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int ry[RPW];
  FP2<T> cy[RPW];  // y couplings of the thread's rows, in registers for all half-sweeps
  const int rx = S.tab.colrx[lane];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    ry[r] = S.tab.rowry[RPW * warp + r];
    cy[r] = S.tab.yc[rx][RPW * warp + r];
  }
  const bool uni = ry[0] == ry[RPW - 1];  // region rows are monotonic in the row
  const int pbase = S.tab.pbase;
  write_halo(S, C);
  __syncthreads();
  after_first_barrier();
  for (int s = 0; s < 2 * nu; ++s) {
    const int colour = s & 1;
    const int p0 = (colour - pbase - RPW * warp) & 1;
    if (uni) {
      if (p0 == 0) half_sweep<T, 0, true>(C, S, ry, cy);
      else half_sweep<T, 1, true>(C, S, ry, cy);
    } else {
      if (p0 == 0) half_sweep<T, 0, false>(C, S, ry, cy);
      else half_sweep<T, 1, false>(C, S, ry, cy);
    }
    __syncthreads();
  }
}

// Residual of the cell of parity P in row r with the tile block's own coefficients (tile rows only).
template <typename T, int P>
__device__ __forceinline__ T resid_row(const Cells<T>& C, FP2<T> cx, T xd, FP2<T> cy, T yd, int r, T sn, T nn) {
  T w, e;
  if (P == 0) {
    w = __shfl_up_sync(0xffffffffu, C.u[r][1], 1);
    e = C.u[r][1];
  } else {
    w = C.u[r][0];
    e = __shfl_down_sync(0xffffffffu, C.u[r][0], 1);
  }
  T a = cx.a * w;
  a = fma(cx.b, e, a);
  a = fma(cy.a, sn, a);
  a = fma(cy.b, nn, a);
  a = fma(xd + yd, C.u[r][P], a);
  return C.f[r][P] - a;
}

// rr[r] = residual of the red cell of row r (the black cells carry none after a sweep ending on
// black); P0 = column parity of the red cells in the strip's first row.
template <typename T, int P0>
__device__ __forceinline__ void red_residuals(const Cells<T>& C, const Shared<T>& S, T sg, T (&rr)[RPW]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int PA = P0, PB = P0 ^ 1;
  const FusedTab<T>& tb = S.tab;
  T south, north;
  edge_values<T, PA>(S, south, north);
  const FP2<T> cxa = tb.xc[1][PA][lane], cxb = tb.xc[1][PB][lane];
  const T xda = tb.xd[1][PA][lane] + sg, xdb = tb.xd[1][PB][lane] + sg;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    const int wj = RPW * warp + r;
    const FP2<T> cy = tb.yc[1][wj];
    const T yd = tb.yd[1][wj];
    if ((r & 1) == 0) {
      const T sn = r > 0 ? C.u[r > 0 ? r - 1 : 0][PA] : south;
      const T nn = C.u[r < RPW - 1 ? r + 1 : 0][PA];
      rr[r] = resid_row<T, PA>(C, cxa, xda, cy, yd, r, sn, nn);
    } else {
      const T sn = C.u[r > 0 ? r - 1 : 0][PB];
      const T nn = r < RPW - 1 ? C.u[r < RPW - 1 ? r + 1 : 0][PB] : north;
      rr[r] = resid_row<T, PB>(C, cxb, xdb, cy, yd, r, sn, nn);
    }
  }
}

// Red residuals of the strip; returns the column parity of the red cells in its first row.
template <typename T>
__device__ __forceinline__ int strip_residuals(const Cells<T>& C, const Shared<T>& S, T sg, T (&rr)[RPW]) {
  const int warp = threadIdx.x >> 5;
  const int p0 = (0 - S.tab.pbase - RPW * warp) & 1;
  if (p0 == 0) red_residuals<T, 0>(C, S, sg, rr);
  else red_residuals<T, 1>(C, S, sg, rr);
  return p0;
}

__device__ __forceinline__ bool in_tile(int w, int extent) { return w >= FH && w < FH + extent; }

// Store the tile's u (window rows/columns FH .. FH + extent, all in the tile's own block, where
// the thread's load offsets are the block's own), one column pair per row.
template <typename T>
__device__ __forceinline__ void store_tile(const Cells<T>& C, const Shared<T>& S, long long base, T* __restrict__ u) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (!in_tile(2 * lane, S.tab.tw)) return;
  int off[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) off[r] = S.goff[r][threadIdx.x];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    if (!in_tile(RPW * warp + r, S.tab.th)) continue;
    *reinterpret_cast<Pair<T>*>(u + base + off[r]) = Pair<T>{C.u[r][0], C.u[r][1]};
  }
}

// Modes per CTA: enough CTAs for about three waves of two per multiprocessor, at most 8 modes.
inline int modes_per_cta(int sms, int ntiles, int nact) {
  const long long mpc = (long long)ntiles * nact / (3LL * 2 * sms);
  return (int)std::min<long long>(8, std::max<long long>(1, mpc));
}

// CTA (tile blockIdx.x, modes active[m0 .. m1)), m0 = blockIdx.y * mpc.
template <typename T>
__global__ void __launch_bounds__(FTHREADS, FMINB)
    k_fdown(const FusedTab<T>* __restrict__ tabs, long long fncell, long long cncell, const int* __restrict__ active,
            int nact, int mpc, const T* __restrict__ sigma, const T* __restrict__ u, T* __restrict__ u_out,
            const T* __restrict__ f, T* __restrict__ fc, T* __restrict__ uc, int nu, int zero_u, int zero_coarse) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T>& S = *reinterpret_cast<Shared<T>*>(smem_raw);
  const int m0 = blockIdx.y * mpc, m1 = min(nact, m0 + mpc);
  copy_tab(S, tabs + blockIdx.x);
  __syncthreads();
  thread_tables(S, false);
  const FusedTab<T>& tb = S.tab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int q = active[m0];
  T sg = sigma[q];
  prefetch_cells(S, (long long)q * fncell, u, f, zero_u == 0);
  cp_async_commit();
  for (int mi = m0; mi < m1; ++mi) {
    const int qn = mi + 1 < m1 ? active[mi + 1] : -1;
    const long long base = (long long)q * fncell;
    cp_async_wait_all();
    Cells<T> C;
    take_cells(C, S, zero_u != 0, sg);
    T sgn = 0;
    sweeps(C, S, nu, [&] {
      if (qn >= 0) {
        sgn = sigma[qn];
        prefetch_cells(S, (long long)qn * fncell, u, f, zero_u == 0);
        cp_async_commit();
      }
    });
    store_tile(C, S, base, u_out);
    // restriction: coarse cell = (column pair k, row pair (2h, 2h+1)) of the strip; its red children
    // are one per row, the black ones carry no residual after the sweep
    T rr[RPW];
    const int p0 = strip_residuals(C, S, sg, rr);
    if (in_tile(2 * lane, tb.tw)) {
      const long long cbase = (long long)q * cncell + tb.cout0 + lane;
      const T wa = tb.rx[p0][lane], wb = tb.rx[p0 ^ 1][lane];  // weights of the red cells of rows 2h, 2h + 1
#pragma unroll
      for (int h = 0; h < RPW / 2; ++h) {
        const int wj = RPW * warp + 2 * h;
        if (!in_tile(wj, tb.th)) continue;
        const T acc = fma(wb * tb.ry[wj + 1], rr[2 * h + 1], wa * tb.ry[wj] * rr[2 * h]);
        const long long cc = cbase + (long long)(wj / 2) * tb.cnx;
        fc[cc] = acc;
        if (zero_coarse) uc[cc] = 0;
      }
    }
    __syncthreads();  // the next mode rewrites the halo rows
    q = qn;
    sg = sgn;
  }
}

template <typename T>
__global__ void __launch_bounds__(FTHREADS, FMINB)
    k_fup(const FusedTab<T>* __restrict__ tabs, int nftiles, long long fncell, long long cncell,
          const int* __restrict__ active, int nact, int mpc, const T* __restrict__ sigma, const T* __restrict__ u,
          T* __restrict__ u_out, const T* __restrict__ f, const T* __restrict__ uc, int nu, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T>& S = *reinterpret_cast<Shared<T>*>(smem_raw);
  const int m0 = blockIdx.y * mpc, m1 = min(nact, m0 + mpc);
  copy_tab(S, tabs + blockIdx.x);
  __syncthreads();
  thread_tables(S, true);
  const FusedTab<T>& tb = S.tab;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int q = active[m0];
  T sg = sigma[q];
  prefetch_cells(S, (long long)q * fncell, u, f, true);
  prefetch_coarse(S, 0, (long long)q * cncell, uc);
  cp_async_commit();
  for (int mi = m0; mi < m1; ++mi) {
    const int qn = mi + 1 < m1 ? active[mi + 1] : -1;
    const int eb = (mi - m0) & 1;
    const long long base = (long long)q * fncell;
    cp_async_wait_all();
    __syncthreads();  // every thread's part of the coarse window is in place
    Cells<T> C;
    take_cells(C, S, false, sg);
    // three-point prolongation onto the thread's owned cells: parent column lane + 1 of the coarse
    // window (both columns of the pair), parent row (RPW / 2) warp + r / 2 + 1. Only the colour-1
    // cells: the first post-smoothing half-sweep rewrites every updated colour-0 cell from its
    // neighbours and f alone, and the window edge is wrong either way (Exactness).
    const int rxc = tb.colrx[lane];
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      const int wj = RPW * warp + r;
      const int ry = tb.rowry[wj];
      const int cj = (RPW / 2) * warp + r / 2 + 1;
      const int cjy = (r & 1) ? cj + 1 : cj - 1;
      const int ci = lane + 1;
      const int p1 = (1 - tb.pbase - wj) & 1;  // column parity of this row's colour-1 cell
      const FP2<T> wy = tb.py[rxc][wj];
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        if (p != p1 || C.inv[r][p] == (T)0) continue;  // colour 0, or unowned
        const FP2<T> wx = tb.px[ry][p][lane];
        const T eC = S.e[eb][cj][ci];
        const T eX = S.e[eb][cj][p ? ci + 1 : ci - 1];
        const T eY = S.e[eb][cjy][ci];
        C.u[r][p] += fma(eC, (T)1 + wx.a + wy.a, fma(wx.b, eX, wy.b * eY));
      }
    }
    T sgn = 0;
    // the next mode's window goes to the other coarse buffer, last read by the previous mode
    sweeps(C, S, nu, [&] {
      if (qn >= 0) {
        sgn = sigma[qn];
        prefetch_cells(S, (long long)qn * fncell, u, f, true);
        prefetch_coarse(S, eb ^ 1, (long long)qn * cncell, uc);
        cp_async_commit();
      }
    });
    store_tile(C, S, base, u_out);
    if (part != nullptr) {
      // sum of squared residuals over the tile's cells (only red cells carry one after a sweep)
      T rr[RPW];
      strip_residuals(C, S, sg, rr);
      T r2 = 0;
      if (in_tile(2 * lane, tb.tw)) {
#pragma unroll
        for (int r = 0; r < RPW; ++r)
          if (in_tile(RPW * warp + r, tb.th)) r2 = fma(rr[r], rr[r], r2);
      }
      r2 = warp_sum_t(r2);  // in the kernel's type, widened once per warp
      if (lane == 0) S.wsum[warp] = (double)r2;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < FWARPS; ++w) sum += S.wsum[w];
        part[(long long)q * nftiles + blockIdx.x] = sum;
      }
    }
    __syncthreads();  // the next mode rewrites the halo rows and wsum
    q = qn;
    sg = sgn;
  }
}

template <typename T>
cudaError_t fused_down_t(snac_plan* P, int l, int nact, bool zero_u, bool zero_coarse, const T* sigma, cudaStream_t s) {
  const HostLevel& h = P->lev[l];
  const HostLevel& hc = P->lev[l + 1];
  const int nt = (int)h.ftiles.size();
  const int mpc = modes_per_cta(P->sms, nt, nact);
  dim3 g((unsigned)nt, (unsigned)((nact + mpc - 1) / mpc));
  const double cells = (double)h.ncell * nact, w = sizeof(T);
  const size_t smem = sizeof(Shared<T>);
  cudaFuncSetAttribute(k_fdown<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // read u (unless zero) and f, write u and the coarse right-hand side
  LaunchScope ls(P, K_FDOWN, w * cells * ((zero_u ? 2.0 : 3.0) + 0.25 + (zero_coarse ? 0.25 : 0.0)),
                 cells * (2.0 * P->nu1 * 11.0 + 7.5), s);
  // iterate: read d_u, write d_u2 (the up kernel of this level reads d_u2 and writes d_u back)
  k_fdown<T><<<g, FTHREADS, smem, s>>>((const FusedTab<T>*)h.d_ftab, h.ncell, hc.ncell, P->d_active, nact, mpc, sigma,
                                       (const T*)h.d_u, (T*)h.d_u2, (const T*)h.d_f, (T*)hc.d_f, (T*)hc.d_u, P->nu1,
                                       zero_u ? 1 : 0, zero_coarse ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fused_up_t(snac_plan* P, int l, int nact, bool norms, const T* sigma, cudaStream_t s) {
  const HostLevel& h = P->lev[l];
  const HostLevel& hc = P->lev[l + 1];
  const int nt = (int)h.ftiles.size();
  const int mpc = modes_per_cta(P->sms, nt, nact);
  dim3 g((unsigned)nt, (unsigned)((nact + mpc - 1) / mpc));
  const double cells = (double)h.ncell * nact, w = sizeof(T);
  const size_t smem = sizeof(Shared<T>);
  cudaFuncSetAttribute(k_fup<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // read u, f and the coarse correction, write u
  LaunchScope ls(P, K_FUP, w * cells * 3.25, cells * (8.0 + 2.0 * P->nu2 * 11.0 + (norms ? 7.0 : 0.0)), s);
  k_fup<T><<<g, FTHREADS, smem, s>>>((const FusedTab<T>*)h.d_ftab, nt, h.ncell, hc.ncell, P->d_active, nact, mpc,
                                     sigma, (const T*)h.d_u2, (T*)h.d_u, (const T*)h.d_f, (const T*)hc.d_u, P->nu2,
                                     norms ? P->d_mode_part : nullptr);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fused_down(snac_plan* P, int l, int nact, bool zero_u, bool zero_coarse, cudaStream_t s) {
  if (P->precision == SNAC_FP64) return fused_down_t<double>(P, l, nact, zero_u, zero_coarse, P->d_sigma64, s);
  return fused_down_t<float>(P, l, nact, zero_u, zero_coarse, P->d_sigma32, s);
}

cudaError_t launch_fused_up(snac_plan* P, int l, int nact, bool norms, cudaStream_t s) {
  if (P->precision == SNAC_FP64) return fused_up_t<double>(P, l, nact, norms, P->d_sigma64, s);
  return fused_up_t<float>(P, l, nact, norms, P->d_sigma32, s);
}

}  // namespace snac
