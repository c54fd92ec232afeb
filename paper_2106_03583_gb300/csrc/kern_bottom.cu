// The bottom of every V-cycle in one kernel (the reduced equations of Eq. 9; Algorithm 1, second
// loop): from the first level whose planes fit in shared memory down to the coarsest and back, one
// CTA per active wavenumber. The coarse levels hold few cells per mode, so run level by level they
// are many small launches that fill the GPU badly (a 16x16 block inside a 64x64 fused window, grids
// of four tiles); here each mode's u, f and 1/diag of those levels stay on chip for the whole
// sub-cycle (FP64 plans read the top level's f from L2, so that two CTAs share a multiprocessor),
// the levels' block tables are copied to shared memory, and the only DRAM traffic is the top level's
// right-hand side in and its correction out.
//
// The arithmetic is that of the level-by-level path: red-black Gauss-Seidel (colour = parity of the
// global index-space position), red-only residuals after a sweep ending on black, area-weighted
// restriction, three-point prolongation onto the cells that the following half-sweep keeps, and the
// coarsest plane solved through the eigen-decomposition of its symmetrised operator. From the zero
// iterate of each level, the first colour-0 half-sweep is u = f / diag, which is written directly.
#include <algorithm>
#include <vector>

#include "kern_common.cuh"
#include "snac_impl.h"
#include "transform_dev.cuh"

namespace snac {
namespace {

constexpr int BT = BOTTOM_THREADS;

// Kernel arguments (by value): the mode data and the coarsest factors; the sub-cycle's levels are
// a small device table (BottomLevel, built with the plan), read per level.
template <typename T>
struct BottomArgs {
  int nlev;                                 // levels of the sub-cycle; the last is the coarsest
  int split;                                // the inverse diagonals are in colour-split order
  int nu1, nu2;
  const BottomLevel<T>* lv;
  int coarse_off;                           // byte offset of the coarsest solve's two FP64 vectors
  const int* active;
  const T* sigma;
  const double* sigma64;
  const int* singular_mode;
  const T* f_top;                           // right-hand side of the top level, [q][cell]
  T* u_top;                                 // its correction, [q][cell]
  const double* Q;
  const double* QT;
  const double* lam;
  const double* sqa;
  int nc;
  int null_index;
};

// Shared-memory arrays of one level of the sub-cycle.
template <typename T>
struct LevelSmem {
  T* u;
  T* f;    // shared memory, or the top level's global right-hand side (read only)
  T* inv;  // smoothed levels only
};

// n / d for 0 <= n < 2^16 and 1 <= d < 2^16 (the on-chip levels have at most 8192 cells): a
// single-precision estimate from the approximate reciprocal (relative error below 2^-21, so the
// estimate is within 2^-5 of n / d), corrected by one step either way -- no integer division in
// the per-cell index arithmetic.
__device__ __forceinline__ int small_div(int n, int d) {
  int q = __float2int_rz(__fdividef((float)n, (float)d));
  const int r = n - q * d;
  q += r >= d ? 1 : 0;
  q -= r < 0 ? 1 : 0;
  return q;
}

// Cell (b, i, j) of the idx-th cell of colour c of a level (blocks in order, rows of each block in
// order, the colour's cells of a row in order of i). Returns false past the last cell.
__device__ __forceinline__ bool colour_cell(const BlockDev* __restrict__ blk, int nblk, int idx, int c, int& b,
                                            BlockDev& B, int& i, int& j) {
  for (b = 0; b < nblk; ++b) {
    B = blk[b];
    const int half = (B.nx >> 1) * B.ny;
    if (idx < half) {
      const int hx = B.nx >> 1;
      j = small_div(idx, hx);
      i = 2 * (idx - j * hx) + ((c ^ B.par ^ j) & 1);
      return true;
    }
    idx -= half;
  }
  return false;
}

// Any cell: (b, i, j) of plane index c.
__device__ __forceinline__ void plane_cell(const BlockDev* __restrict__ blk, int nblk, int c, int& b, BlockDev& B, int& i,
                                           int& j) {
  for (b = 0; b < nblk - 1; ++b) {
    if (c < blk[b + 1].off) break;
  }
  B = blk[b];
  const int l = c - (int)B.off;
  j = small_div(l, B.nx);
  i = l - j * B.nx;
}

// Plane indices of the four neighbours of cell c = (i, j) of block B (the same cells nbr_plane
// gives, in int arithmetic for the on-chip levels): inside the block directly; across a face the
// connected block's cell from the block table, or the cell itself on a physical face.
__device__ __forceinline__ void nbr_int(const BlockDev* __restrict__ blk, const BlockDev& B, int i, int j, int c,
                                        int& w, int& e, int& s, int& n) {
  w = c - 1;
  e = c + 1;
  s = c - B.nx;
  n = c + B.nx;
  if (i == 0) {
    const int k = B.nbr[0];
    w = k >= 0 ? (int)blk[k].off + j * blk[k].nx + blk[k].nx - 1 : c;
  }
  if (i == B.nx - 1) {
    const int k = B.nbr[1];
    e = k >= 0 ? (int)blk[k].off + j * blk[k].nx : c;
  }
  if (j == 0) {
    const int k = B.nbr[2];
    s = k >= 0 ? (int)blk[k].off + (blk[k].ny - 1) * blk[k].nx + i : c;
  }
  if (j == B.ny - 1) {
    const int k = B.nbr[3];
    n = k >= 0 ? (int)blk[k].off + i : c;
  }
}

// One Gauss-Seidel half-sweep of colour c on a level.
template <typename T>
__device__ void half_sweep(const LevelView<T>& L, const LevelSmem<T>& S, int c) {
  const int ncol = (int)(L.ncell >> 1);
  for (int idx = threadIdx.x; idx < ncol; idx += BT) {
    int b, i, j;
    BlockDev B;
    if (!colour_cell(L.blk, L.nblk, idx, c, b, B, i, j)) break;
    const int cc = (int)B.off + j * B.nx + i;
    int w, e, s, n;
    nbr_int(L.blk, B, i, j, cc, w, e, s, n);
    const Coef<T> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
    T a = cx.lo * S.u[w];
    a = fma(cx.hi, S.u[e], a);
    a = fma(cy.lo, S.u[s], a);
    a = fma(cy.hi, S.u[n], a);
    S.u[cc] = (S.f[cc] - a) * S.inv[cc];
  }
  __syncthreads();
}

// Residual on the colour-0 cells of the fine level (the colour-1 cells carry none after a sweep
// ending on colour 1), restricted into the coarse right-hand side; the coarse iterate starts with
// its first colour-0 half-sweep done (u = f / diag on colour 0, zero on colour 1).
template <typename T>
__device__ void restrict_to(const LevelView<T>& F, const LevelSmem<T>& SF, const LevelView<T>& C,
                            const LevelSmem<T>& SC, T sg, bool coarse_smoothed) {
  for (int cc = threadIdx.x; cc < (int)C.ncell; cc += BT) {
    int b, I, J;
    BlockDev Bc;
    plane_cell(C.blk, C.nblk, cc, b, Bc, I, J);
    const BlockDev Bf = F.blk[b];
    T acc = 0;
#pragma unroll
    for (int dj = 0; dj < 2; ++dj) {
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj;
        if ((Bf.par + i + j) & 1) continue;
        const int c = (int)Bf.off + j * Bf.nx + i;
        int w, e, s, n;
        nbr_int(F.blk, Bf, i, j, c, w, e, s, n);
        const Coef<T> cx = F.cx[Bf.xo + i], cy = F.cy[Bf.yo + j];
        T a = cx.lo * SF.u[w];
        a = fma(cx.hi, SF.u[e], a);
        a = fma(cy.lo, SF.u[s], a);
        a = fma(cy.hi, SF.u[n], a);
        a = fma(F.dxy[c] + sg, SF.u[c], a);
        acc = fma(F.wr[c], SF.f[c] - a, acc);  // rx * ry
      }
    }
    SC.f[cc] = acc;
    SC.u[cc] = (coarse_smoothed && ((Bc.par + I + J) & 1) == 0) ? acc * SC.inv[cc] : (T)0;
  }
  __syncthreads();
}

// u_f += e_C (1 + sx + sy) + nx e_X + ny e_Y on the colour-1 cells of the fine level (the first
// post-smoothing half-sweep rewrites colour 0), or on every cell when no post-smoothing follows.
template <typename T>
__device__ void prolong_from(const LevelView<T>& F, const LevelSmem<T>& SF, const LevelView<T>& C,
                             const LevelSmem<T>& SC, bool colour1_only) {
  const int nfine = (int)F.ncell;
  for (int idx = threadIdx.x; idx < (colour1_only ? nfine >> 1 : nfine); idx += BT) {
    int b, i, j;
    BlockDev Bf;
    if (colour1_only) {
      if (!colour_cell(F.blk, F.nblk, idx, 1, b, Bf, i, j)) break;
    } else {
      plane_cell(F.blk, F.nblk, idx, b, Bf, i, j);
    }
    const BlockDev Bc = C.blk[b];
    const int I = i >> 1, J = j >> 1;
    const int cI = (int)Bc.off + J * Bc.nx + I;
    int w, e, s, n;
    nbr_int(C.blk, Bc, I, J, cI, w, e, s, n);
    const T eC = SC.u[cI];
    const T eX = SC.u[(i & 1) ? e : w];
    const T eY = SC.u[(j & 1) ? n : s];
    const PW<T> px = F.px[Bf.xo + i], py = F.py[Bf.yo + j];
    const int c = (int)(Bf.off + (long long)j * Bf.nx + i);
    T u = fma(eC, F.wp[c], SF.u[c]);  // 1 + self_x + self_y
    u = fma(px.nbr, eX, u);
    SF.u[c] = fma(py.nbr, eY, u);
  }
  __syncthreads();
}

// Coarsest plane: u = V^-1/2 Q (Lam + sigma)^-1 Q^T V^1/2 f (the null eigenvector dropped for a
// singular mode), in FP64. The wavenumber's factors come once per CTA and wavenumber
// (coarse_factors); each product is one thread per entry reading a row of Q^T or Q, so that a cycle
// issues no FP64 division and no cross-lane reduction (GB300's FP64 pipe is 1/64 of FP32).
__device__ void coarse_factors(const double* __restrict__ lam, const double* __restrict__ sqa, int nc, int null_index,
                               double sg, bool sing, double* dinv, double* isq) {
  for (int k = threadIdx.x; k < nc; k += BT) {
    dinv[k] = (sing && k == null_index) ? 0.0 : 1.0 / (lam[k] + sg);
    isq[k] = 1.0 / sqa[k];
  }
}

template <typename T>
__device__ void coarse_solve(const double* __restrict__ Q, const double* __restrict__ QT,
                             const double* __restrict__ sqa, int nc, const LevelSmem<T>& S, const double* dinv,
                             const double* isq, double* b, double* y) {
  for (int i = threadIdx.x; i < nc; i += BT) b[i] = sqa[i] * (double)S.f[i];
  __syncthreads();
  for (int k = threadIdx.x; k < nc; k += BT) {  // y = (Lam + sigma)^-1 Q^T b
    const double* qk = QT + (long long)k * nc;
    double s = 0.0;
    for (int i = 0; i < nc; ++i) s = fma(qk[i], b[i], s);
    y[k] = s * dinv[k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += BT) {  // u = V^-1/2 Q y
    const double* qi = Q + (long long)i * nc;
    double s = 0.0;
    for (int k = 0; k < nc; ++k) s = fma(qi[k], y[k], s);
    S.u[i] = (T)(s * isq[i]);
  }
  __syncthreads();
}

// The level's arrays of mode q: u and 1/diag in shared memory; f there too, or (sf < 0) the level's
// global right-hand side. The block table is the shared-memory copy.
template <typename T>
__device__ __forceinline__ LevelSmem<T> level_smem(unsigned char* raw, const BottomLevel<T>& bl, const T* f_global) {
  T* base = reinterpret_cast<T*>(raw);
  return LevelSmem<T>{base + bl.su, bl.sf >= 0 ? base + bl.sf : const_cast<T*>(f_global),
                      bl.sinv >= 0 ? base + bl.sinv : nullptr};
}

template <typename T>
__device__ __forceinline__ BottomLevel<T> level_at(const BottomArgs<T>& A, unsigned char* raw, int l) {
  BottomLevel<T> bl = A.lv[l];
  bl.L.blk = reinterpret_cast<const BlockDev*>(raw + bl.sblk);
  return bl;
}

template <typename T>
__global__ void __launch_bounds__(BT) k_bottom(const BottomArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int q = A.active[blockIdx.x];
  const int nl = A.nlev;  // levels 0 .. nl-1 of the sub-cycle; the last is the coarsest
  double* b = reinterpret_cast<double*>(smem_raw + A.coarse_off);
  double* y = b + MAX_COARSE;
  double* dinv = y + MAX_COARSE;  // the coarsest solve's factors of this wavenumber
  double* isq = dinv + MAX_COARSE;
  const T sg = A.sigma[q];
  const double sg64 = A.sigma64[q];
  const bool sing = A.singular_mode[q] != 0;
  const T* f0g = A.f_top + (long long)q * A.lv[0].L.ncell;  // the top level's right-hand side
  // the levels' block tables, the top level's right-hand side (when it is kept on chip), and 1/diag
  // of every smoothed level
  for (int l = 0; l < nl; ++l) {
    const BottomLevel<T> bl = A.lv[l];
    const unsigned* src = reinterpret_cast<const unsigned*>(bl.L.blk);
    unsigned* dst = reinterpret_cast<unsigned*>(smem_raw + bl.sblk);
    const int words = bl.L.nblk * (int)(sizeof(BlockDev) / sizeof(unsigned));
    for (int k = threadIdx.x; k < words; k += BT) dst[k] = src[k];
  }
  {
    const BottomLevel<T> top = A.lv[0];
    if (top.sf >= 0) {
      T* f0 = reinterpret_cast<T*>(smem_raw) + top.sf;
      for (int c = threadIdx.x; c < (int)top.L.ncell; c += BT) f0[c] = f0g[c];
    }
  }
  coarse_factors(A.lam, A.sqa, A.nc, A.null_index, sg64, sing, dinv, isq);
  __syncthreads();
  for (int l = 0; l + 1 < nl; ++l) {
    const BottomLevel<T> bl = level_at(A, smem_raw, l);
    const LevelSmem<T> S = level_smem(smem_raw, bl, f0g);
    const int n = (int)bl.L.ncell;
    for (int c = threadIdx.x; c < n; c += BT) {
      T iv;
      if (bl.invd != nullptr) {  // FP64: the plan's inverse diagonals (colour-split order if split)
        int b0, i, j;
        BlockDev B;
        plane_cell(bl.L.blk, bl.L.nblk, c, b0, B, i, j);
        iv = (T)bl.invd[(long long)q * n + (A.split ? split_cell(B, i, j) : c)];
      } else {
        iv = (T)1 / (bl.L.dxy[c] + sg);
      }
      S.inv[c] = iv;
    }
  }
  __syncthreads();
  // the top level's first colour-0 half-sweep from its zero iterate
  {
    const BottomLevel<T> top = level_at(A, smem_raw, 0);
    const LevelSmem<T> S = level_smem(smem_raw, top, f0g);
    const int n0 = (int)top.L.ncell;
    for (int c = threadIdx.x; c < n0; c += BT) {
      int b0, i, j;
      BlockDev B;
      plane_cell(top.L.blk, top.L.nblk, c, b0, B, i, j);
      S.u[c] = (nl > 1 && ((B.par + i + j) & 1) == 0) ? S.f[c] * S.inv[c] : (T)0;
    }
    __syncthreads();
  }
  // down: nu1 sweeps (the first colour-0 half-sweep already done), residual, restriction
  for (int l = 0; l + 1 < nl; ++l) {
    const BottomLevel<T> F = level_at(A, smem_raw, l), C = level_at(A, smem_raw, l + 1);
    const LevelSmem<T> SF = level_smem(smem_raw, F, f0g), SC = level_smem(smem_raw, C, f0g);
    for (int it = 0; it < A.nu1; ++it) {
      if (it > 0) half_sweep(F.L, SF, 0);
      half_sweep(F.L, SF, 1);
    }
    restrict_to(F.L, SF, C.L, SC, sg, l + 2 < nl);  // plans run it with nu1 >= 1
  }
  {
    const BottomLevel<T> C = level_at(A, smem_raw, nl - 1);
    coarse_solve(A.Q, A.QT, A.sqa, A.nc, level_smem(smem_raw, C, f0g), dinv, isq, b, y);
  }
  // up: prolongation onto the colour-1 cells, nu2 sweeps
  for (int l = nl - 2; l >= 0; --l) {
    const BottomLevel<T> F = level_at(A, smem_raw, l), C = level_at(A, smem_raw, l + 1);
    const LevelSmem<T> SF = level_smem(smem_raw, F, f0g), SC = level_smem(smem_raw, C, f0g);
    prolong_from(F.L, SF, C.L, SC, true);
    for (int it = 0; it < A.nu2; ++it) {
      half_sweep(F.L, SF, 0);
      half_sweep(F.L, SF, 1);
    }
  }
  // the top level's correction, back to the level-by-level part of the cycle
  {
    const BottomLevel<T> top = A.lv[0];
    const LevelSmem<T> S = level_smem(smem_raw, top, f0g);
    const int n0 = (int)top.L.ncell;
    T* u0 = A.u_top + (long long)q * n0;
    for (int c = threadIdx.x; c < n0; c += BT) u0[c] = S.u[c];
  }
}

// ---- whole-mode solves on chip, with their convergence decided on the device ----
//
// When a plan's whole hierarchy, from level 0, fits in one CTA's shared memory, a wavenumber's
// complete multigrid solve runs in one CTA: its right-hand side comes in once, V-cycles run on chip
// until the mode meets its share of the target (w_q ||r_q||^2 <= target^2 / n_z, the rule of the
// level-by-level path) or stops improving (a cycle that reduces ||r_q||^2 by less than 0.36), or
// max_cycles; its correction goes out once. There is no host round trip per cycle: the residual
// norm after every cycle is reduced in the CTA and the loop stops on the device.

// Block-wide sum of one double, returned to every thread in a fixed order (scratch: 32 doubles).
__device__ __forceinline__ double block_sum_all(double v, double* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();  // the scratch's previous readers are done
  if (lane == 0) scratch[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < BT / 32; ++w) t += scratch[w];
  return t;
}

// ||f - A u||^2 over the colour-0 cells of a level (after a sweep ending on colour 1 the colour-1
// cells carry no residual).
template <typename T>
__device__ double colour0_resid2(const LevelView<T>& L, const LevelSmem<T>& S, T sg, double* scratch) {
  double acc = 0.0;
  const int ncol = (int)(L.ncell >> 1);
  for (int idx = threadIdx.x; idx < ncol; idx += BT) {
    int b, i, j;
    BlockDev B;
    if (!colour_cell(L.blk, L.nblk, idx, 0, b, B, i, j)) break;
    const int c = (int)B.off + j * B.nx + i;
    int w, e, s, n;
    nbr_int(L.blk, B, i, j, c, w, e, s, n);
    const Coef<T> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
    T a = cx.lo * S.u[w];
    a = fma(cx.hi, S.u[e], a);
    a = fma(cy.lo, S.u[s], a);
    a = fma(cy.hi, S.u[n], a);
    a = fma(L.dxy[c] + sg, S.u[c], a);
    const double r = (double)(S.f[c] - a);
    acc = fma(r, r, acc);
  }
  return block_sum_all(acc, scratch);
}

template <typename T>
struct OnchipArgs {
  BottomArgs<T> B;          // the hierarchy from level 0 (f_top, u_top: the level-0 mode fields)
  const double* pweight;    // Parseval weight of every wavenumber the plan holds
  double t2nz;              // target^2 / n_z: mode q is done when ||r_q||^2 <= t2nz / pweight[q]
  int max_cycles;
  int* cycles;              // per wavenumber: V-cycles run
  double* norm2;            // per wavenumber: ||r_q||^2 on return
};

// One wavenumber's solve, from a zero iterate, by one CTA.
template <typename T>
__device__ void onchip_mode(const OnchipArgs<T>& O, int q, unsigned char* smem_raw) {
  const BottomArgs<T>& A = O.B;
  const int nl = A.nlev;
  double* b = reinterpret_cast<double*>(smem_raw + A.coarse_off);
  double* y = b + MAX_COARSE;
  double* dinv = y + MAX_COARSE;  // the coarsest solve's factors of this wavenumber
  double* isq = dinv + MAX_COARSE;
  const T sg = A.sigma[q];
  const double sg64 = A.sigma64[q];
  const bool sing = A.singular_mode[q] != 0;
  const T* f0g = A.f_top + (long long)q * A.lv[0].L.ncell;
  for (int l = 0; l < nl; ++l) {
    const BottomLevel<T> bl = A.lv[l];
    const unsigned* src = reinterpret_cast<const unsigned*>(bl.L.blk);
    unsigned* dst = reinterpret_cast<unsigned*>(smem_raw + bl.sblk);
    const int words = bl.L.nblk * (int)(sizeof(BlockDev) / sizeof(unsigned));
    for (int k = threadIdx.x; k < words; k += BT) dst[k] = src[k];
  }
  {
    const BottomLevel<T> top = A.lv[0];
    if (top.sf >= 0) {
      T* f0 = reinterpret_cast<T*>(smem_raw) + top.sf;
      for (int c = threadIdx.x; c < (int)top.L.ncell; c += BT) f0[c] = f0g[c];
    }
  }
  coarse_factors(A.lam, A.sqa, A.nc, A.null_index, sg64, sing, dinv, isq);
  __syncthreads();
  for (int l = 0; l + 1 < nl; ++l) {
    const BottomLevel<T> bl = level_at(A, smem_raw, l);
    const LevelSmem<T> S = level_smem(smem_raw, bl, f0g);
    const int n = (int)bl.L.ncell;
    for (int c = threadIdx.x; c < n; c += BT)
      S.inv[c] = bl.invd != nullptr ? (T)bl.invd[(long long)q * n + c] : (T)1 / (bl.L.dxy[c] + sg);
  }
  const BottomLevel<T> top = level_at(A, smem_raw, 0);
  const LevelSmem<T> S0 = level_smem(smem_raw, top, f0g);
  const int n0 = (int)top.L.ncell;
  double f2 = 0.0;
  for (int c = threadIdx.x; c < n0; c += BT) {
    const double v = (double)S0.f[c];
    f2 = fma(v, v, f2);
    S0.u[c] = (T)0;
  }
  double r2 = block_sum_all(f2, y);  // (its barriers also publish u and 1/diag)
  const double thr2 = O.t2nz / O.pweight[q];
  int cyc = 0;
  if (r2 > thr2) {
    double prev = r2;
    while (cyc < O.max_cycles) {
      // down: nu1 sweeps (on the coarse levels the first colour-0 half-sweep is done by the
      // restriction that fills them), residual, restriction
      for (int l = 0; l + 1 < nl; ++l) {
        const BottomLevel<T> F = level_at(A, smem_raw, l), C = level_at(A, smem_raw, l + 1);
        const LevelSmem<T> SF = level_smem(smem_raw, F, f0g), SC = level_smem(smem_raw, C, f0g);
        for (int it = 0; it < A.nu1; ++it) {
          if (it > 0 || l == 0) half_sweep(F.L, SF, 0);
          half_sweep(F.L, SF, 1);
        }
        restrict_to(F.L, SF, C.L, SC, sg, l + 2 < nl);
      }
      {
        const BottomLevel<T> C = level_at(A, smem_raw, nl - 1);
        coarse_solve(A.Q, A.QT, A.sqa, A.nc, level_smem(smem_raw, C, f0g), dinv, isq, b, y);
      }
      for (int l = nl - 2; l >= 0; --l) {
        const BottomLevel<T> F = level_at(A, smem_raw, l), C = level_at(A, smem_raw, l + 1);
        const LevelSmem<T> SF = level_smem(smem_raw, F, f0g), SC = level_smem(smem_raw, C, f0g);
        prolong_from(F.L, SF, C.L, SC, true);
        for (int it = 0; it < A.nu2; ++it) {
          half_sweep(F.L, SF, 0);
          half_sweep(F.L, SF, 1);
        }
      }
      ++cyc;
      r2 = colour0_resid2(top.L, S0, sg, y);
      if (!(r2 > thr2) || r2 > 0.36 * prev) break;  // done, stagnant, or not finite
      prev = r2;
    }
  }
  T* u0 = A.u_top + (long long)q * n0;
  for (int c = threadIdx.x; c < n0; c += BT) u0[c] = S0.u[c];
  if (threadIdx.x == 0) {
    O.cycles[q] = cyc;
    O.norm2[q] = r2;
  }
  __syncthreads();  // the shared memory is free for the next wavenumber
}

// One plan: CTA k solves wavenumber active[k].
template <typename T>
__global__ void __launch_bounds__(BT, 1) k_onchip(const OnchipArgs<T> O) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  onchip_mode(O, O.B.active[blockIdx.x], smem_raw);
}

// Many plans in one persistent launch: every CTA takes (problem, wavenumber) items from a queue
// (an atomic counter, zero at launch) until none is left; each item uses its own problem's tables.
template <typename T>
__global__ void __launch_bounds__(BT, 1) k_onchip_batch(const OnchipArgs<T>* __restrict__ args, const int2* __restrict__ items,
                                                     int nitems, int* __restrict__ next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int item;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int k = item;
    __syncthreads();
    if (k >= nitems) break;
    const int2 w = items[k];
    const OnchipArgs<T> O = args[w.x];
    onchip_mode(O, w.y, smem_raw);
  }
}

// ---- the forward transform and the on-chip solves in one persistent launch ----
//
// Items: first the forward-transform chunks of every plan (TC columns each), then the wavenumber
// solves. A CTA that finishes a chunk counts it for its plan (release); a solve item waits until all
// of its plan's chunks are counted (acquire). Items are claimed in increasing order and a claimed
// item runs to completion, so every chunk a solve waits for is already held by a running CTA: the
// wait always ends. It is still bounded: past wait_ns (global timer) the item gives up, sets its
// plan's status word and skips its work, so that the host reports SNAC_ERR_TIMEOUT and the context
// stays usable.
template <typename T>
struct FwdArgs {
  const ChunkDev* chunks;
  const BlockDev* blk;
  const CallerBlk* cb;
  Tw<T> tw;
  const void* in3;       // the 3-D field transformed: FP64 (f or the FP64 residual) or FP32
  T* out;                // level-0 right-hand side, [q][cell]
  long long ncell;
  T sub0;                // F(1) x (mean removed from f), on mode 0 (k = 0 from a zero guess)
  int n, kind, in_f32, nchunks;
  int need;              // chunks a solve item waits for (nchunks; more only in the timeout self-test)
  int* done;             // chunks counted so far (zero at launch)
  int* status;           // 1 if a wait of this plan gave up
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int load_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <typename T, int TC>
__device__ void fused_chunk(const FwdArgs<T>& F, int c, unsigned char* smem) {
  const ChunkDev ch = F.chunks[c];
  const int sel = F.kind * 2 + F.in_f32;
#define SNAC_FWD(KD, TI)                                                                                   \
  forward_chunk<T, TC, KD, TI, BT>(ch, F.blk, F.cb, F.n, F.tw, static_cast<const TI*>(F.in3), F.out, F.ncell, F.sub0, 0, smem)
  switch (sel) {
    case 2 * KIND_PP: SNAC_FWD(KIND_PP, double); break;
    case 2 * KIND_PP + 1: SNAC_FWD(KIND_PP, float); break;
    case 2 * KIND_NN: SNAC_FWD(KIND_NN, double); break;
    case 2 * KIND_NN + 1: SNAC_FWD(KIND_NN, float); break;
    case 2 * KIND_DD: SNAC_FWD(KIND_DD, double); break;
    case 2 * KIND_DD + 1: SNAC_FWD(KIND_DD, float); break;
    case 2 * KIND_ND: SNAC_FWD(KIND_ND, double); break;
    case 2 * KIND_ND + 1: SNAC_FWD(KIND_ND, float); break;
    case 2 * KIND_DN: SNAC_FWD(KIND_DN, double); break;
    default: SNAC_FWD(KIND_DN, float); break;
  }
#undef SNAC_FWD
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(F.done, 1);
  }
}

template <typename T>
__device__ void fused_solve(const FwdArgs<T>& F, const OnchipArgs<T>& O, int q, long long wait_ns,
                            unsigned char* smem, int* skip) {
  if (threadIdx.x == 0) {
    const unsigned long long t0 = global_ns();
    int give_up = 0;
    while (load_acquire(F.done) < F.need) {
      if (global_ns() - t0 > (unsigned long long)wait_ns) {
        give_up = 1;
        atomicOr(F.status, 1);
        break;
      }
      __nanosleep(500);
    }
    *skip = give_up;
  }
  __syncthreads();
  const int sk = *skip;
  __syncthreads();
  if (!sk) onchip_mode(O, q, smem);
}

// One plan: items 0 .. nchunks - 1 are its chunks, then its wavenumbers 0 .. nmodes - 1.
template <typename T, int TC>
__global__ void __launch_bounds__(BT, 1) k_fwd_onchip(const FwdArgs<T> F, const OnchipArgs<T> O, int nmodes,
                                                   int* __restrict__ next, long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int item, skip;
  const int nitems = F.nchunks + nmodes;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int k = item;
    __syncthreads();
    if (k >= nitems) break;
    if (k < F.nchunks) fused_chunk<T, TC>(F, k, smem_raw);
    else fused_solve(F, O, k - F.nchunks, wait_ns, smem_raw, &skip);
  }
}

// Several plans: items (type, plan, index) from a table -- every plan's chunks first, then every
// plan's wavenumbers.
template <typename T, int TC>
__global__ void __launch_bounds__(BT, 1) k_fwd_onchip_batch(const FwdArgs<T>* __restrict__ fargs,
                                                         const OnchipArgs<T>* __restrict__ args,
                                                         const int4* __restrict__ items, int nitems,
                                                         int* __restrict__ next, long long wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int item, skip;
  for (;;) {
    if (threadIdx.x == 0) item = atomicAdd(next, 1);
    __syncthreads();
    const int k = item;
    __syncthreads();
    if (k >= nitems) break;
    const int4 it = items[k];
    const FwdArgs<T> F = fargs[it.y];
    if (it.x == 0) {
      fused_chunk<T, TC>(F, it.z, smem_raw);
    } else {
      const OnchipArgs<T> O = args[it.y];
      fused_solve(F, O, it.z, wait_ns, smem_raw, &skip);
    }
  }
}

template <typename T>
OnchipArgs<T> onchip_args(snac_plan* P, double target) {
  OnchipArgs<T> O{};
  BottomArgs<T>& A = O.B;
  const int L = (int)P->lev.size() - 1;
  const BottomLayout lay = bottom_layout(P, 0, sizeof(T));
  A.nlev = L + 1;
  A.split = 0;
  A.nu1 = P->nu1;
  A.nu2 = P->nu2;
  A.lv = (const BottomLevel<T>*)P->d_onchip;
  A.coarse_off = lay.coarse_off;
  A.active = P->d_active;
  if constexpr (sizeof(T) == 8) A.sigma = (const T*)P->d_sigma64;
  else A.sigma = (const T*)P->d_sigma32;
  A.sigma64 = P->d_sigma64;
  A.singular_mode = P->d_singular_mode;
  A.f_top = (const T*)P->lev[0].d_f;
  A.u_top = (T*)P->lev[0].d_u;
  A.Q = P->d_Q;
  A.QT = P->d_QT;
  A.lam = P->d_lam;
  A.sqa = P->d_sqa;
  A.nc = P->nc;
  A.null_index = P->null_index;
  O.pweight = P->d_pweight;
  O.t2nz = target * target / (double)P->nzt;
  O.max_cycles = P->max_cycles;
  O.cycles = P->dh_cycles;
  O.norm2 = P->dh_mode_norm2;
  return O;
}

// algorithmic bytes and flops of one on-chip V-cycle of one wavenumber, and of its load and store
double onchip_cycle_flops(const snac_plan* P) {
  double fl = 0.0;
  const int L = (int)P->lev.size() - 1;
  for (int l = 0; l < L; ++l) fl += (double)P->lev[l].ncell * (12.0 * (P->nu1 + P->nu2) + 15.0 + 8.0);
  return fl + 4.0 * P->nc * P->nc + 7.0 * P->lev[0].ncell;
}

template <typename T>
cudaError_t onchip_t(snac_plan* P, int nact, double target, cudaStream_t s) {
  const OnchipArgs<T> O = onchip_args<T>(P, target);
  const BottomLayout lay = bottom_layout(P, 0, sizeof(T));
  cudaFuncSetAttribute(k_onchip<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, BOTTOM_MAX_SMEM);
  const double w = sizeof(T);
  // per wavenumber: f in, u out; the flops of an assumed 4 cycles (the kernel decides how many run)
  LaunchScope ls(P, K_ONCHIP, 2.0 * w * (double)P->lev[0].ncell * nact, 4.0 * onchip_cycle_flops(P) * nact, s);
  k_onchip<T><<<nact, BT, lay.bytes, s>>>(O);
  return cudaGetLastError();
}

template <typename T>
cudaError_t bottom_t(snac_plan* P, int nact, cudaStream_t s) {
  BottomArgs<T> A{};
  const int lb = P->bottom, L = (int)P->lev.size() - 1;
  const BottomLayout lay = bottom_layout(P, lb, sizeof(T));
  A.nlev = L - lb + 1;
  A.split = P->scaled_f ? 1 : 0;
  A.nu1 = P->nu1;
  A.nu2 = P->nu2;
  A.lv = (const BottomLevel<T>*)P->d_bottom;
  A.coarse_off = lay.coarse_off;
  A.active = P->d_active;
  if constexpr (sizeof(T) == 8) A.sigma = (const T*)P->d_sigma64;
  else A.sigma = (const T*)P->d_sigma32;
  A.sigma64 = P->d_sigma64;
  A.singular_mode = P->d_singular_mode;
  A.f_top = (const T*)P->lev[lb].d_f;
  A.u_top = (T*)P->lev[lb].d_u;
  A.Q = P->d_Q;
  A.QT = P->d_QT;
  A.lam = P->d_lam;
  A.sqa = P->d_sqa;
  A.nc = P->nc;
  A.null_index = P->null_index;
  cudaFuncSetAttribute(k_bottom<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, BOTTOM_MAX_SMEM);
  double flops = 0.0;
  for (int l = lb; l < L; ++l) flops += (double)P->lev[l].ncell * nact * (12.0 * (P->nu1 + P->nu2) + 15.0 + 8.0);
  // DRAM: the top level's right-hand side in and its correction out (tables and factors stay in L2)
  const double w = sizeof(T);
  LaunchScope ls(P, K_BOTTOM, 2.0 * w * (double)P->lev[lb].ncell * nact, flops + 4.0 * P->nc * P->nc * nact, s);
  k_bottom<T><<<nact, BT, lay.bytes, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

BottomLayout bottom_layout(const snac_plan* P, int lb, size_t w) {
  BottomLayout lay{};
  const int L = (int)P->lev.size() - 1;
  size_t el = 0;  // elements of the inner type
  for (int l = lb; l <= L && l - lb < BOTTOM_MAX_LEVELS; ++l) {
    const int k = l - lb;
    const size_t n = (size_t)P->lev[l].ncell;
    lay.su[k] = (int)el;
    el += n;
    if (k == 0 && w == sizeof(double)) {
      lay.sf[k] = -1;
    } else {
      lay.sf[k] = (int)el;
      el += n;
    }
    lay.sinv[k] = -1;
    if (l < L) {
      lay.sinv[k] = (int)el;
      el += n;
    }
  }
  size_t bytes = (el * w + 15) / 16 * 16;
  lay.coarse_off = (int)bytes;
  bytes += 4 * MAX_COARSE * sizeof(double);  // the coarsest solve's b, y and factors
  for (int l = lb; l <= L && l - lb < BOTTOM_MAX_LEVELS; ++l) {
    lay.sblk[l - lb] = (int)bytes;
    bytes += (size_t)P->lev[l].nblk * sizeof(BlockDev);
  }
  lay.bytes = bytes;
  return lay;
}

cudaError_t launch_bottom(snac_plan* P, int nact, cudaStream_t s) {
  if (nact <= 0) return cudaSuccess;
  return P->precision == SNAC_FP64 ? bottom_t<double>(P, nact, s) : bottom_t<float>(P, nact, s);
}

__global__ void k_zero_ints(int* __restrict__ p, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = 0;
}

template <typename T>
FwdArgs<T> fwd_args(snac_plan* P, const void* in3, bool in_f32, double shift0, int* done, int* status, int extra) {
  FwdArgs<T> F{};
  const bool f64 = sizeof(T) == 8;
  F.chunks = f64 ? P->d_chunks64 : P->d_chunks32;
  F.blk = P->lev[0].d_blk;
  F.cb = P->d_cblk;
  const Cx<T>* t = reinterpret_cast<const Cx<T>*>(f64 ? (const void*)P->d_tw64 : (const void*)P->d_tw32);
  F.tw = Tw<T>{t + P->tw.fft, t + P->tw.twn, t + P->tw.tw2n, t + P->tw.tw4a, t + P->tw.tw4b};
  F.in3 = in3;
  F.out = (T*)P->lev[0].d_f;
  F.ncell = P->lev[0].ncell;
  // F(1) in mode 0: n for the real DFT (half-complex), 2n for the DCT-II
  F.sub0 = (T)(shift0 * (P->kind == KIND_PP ? (double)P->nzt : 2.0 * P->nzt));
  F.n = P->nzt;
  F.kind = P->kind;
  F.in_f32 = in_f32 ? 1 : 0;
  F.nchunks = (int)(f64 ? P->chunks64.size() : P->chunks32.size());
  F.need = F.nchunks + extra;
  F.done = done;
  F.status = status;
  return F;
}

template <typename T>
constexpr int fused_tc() {
  return sizeof(T) == 8 ? 8 : 16;
}

template <typename T>
size_t fused_smem(const snac_plan* P) {
  const size_t fft = 2 * (size_t)(P->nzt / 2) * fused_tc<T>() * sizeof(Cx<T>);
  return std::max(fft, bottom_layout(P, 0, sizeof(T)).bytes);
}

template <typename T>
cudaError_t fwd_onchip_t(snac_plan* P, const void* in3, bool in_f32, double shift0, double target, double wait_s,
                         int extra, cudaStream_t s) {
  constexpr int TC = fused_tc<T>();
  *P->h_wait = 0;
  k_zero_ints<<<1, 32, 0, s>>>(P->d_fused, 2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const FwdArgs<T> F = fwd_args<T>(P, in3, in_f32, shift0, P->d_fused + 1, P->dh_wait, extra);
  const OnchipArgs<T> O = onchip_args<T>(P, target);
  const size_t smem = fused_smem<T>(P);
  cudaFuncSetAttribute(k_fwd_onchip<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, BOTTOM_MAX_SMEM);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_onchip<T, TC>, BT, smem);
  const int nitems = F.nchunks + P->nz;
  // one CTA per multiprocessor: two wavenumber solves never share one (their V-cycles are bound by
  // the SM's own pipes), and the transform chunks still spread over every SM
  const int grid = std::max(1, std::min(nitems, std::min(std::max(1, per_sm), 1) * P->sms));
  const double w = sizeof(T), n3 = (double)P->n3;
  LaunchScope ls(P, K_FWD_ONCHIP, (in_f32 ? 4.0 : 8.0) * n3 + w * n3 + 2.0 * w * (double)P->lev[0].ncell * P->nz,
                 (2.5 * std::log2((double)P->nzt) + 8.0) * n3 + 4.0 * onchip_cycle_flops(P) * P->nz, s);
  k_fwd_onchip<T, TC><<<grid, BT, smem, s>>>(F, O, P->nz, P->d_fused, (long long)(wait_s * 1e9));
  return cudaGetLastError();
}

cudaError_t launch_onchip(snac_plan* P, int nact, double target, cudaStream_t s) {
  if (nact <= 0) return cudaSuccess;
  if (!P->d_onchip) return cudaErrorInvalidValue;
  return P->precision == SNAC_FP64 ? onchip_t<double>(P, nact, target, s) : onchip_t<float>(P, nact, target, s);
}

bool fused_ready(const snac_plan* P) {
  return P->onchip && P->d_fused && !P->ranged &&
         (P->precision == SNAC_FP64 ? P->tc64 == fused_tc<double>() : P->tc32 == fused_tc<float>());
}

cudaError_t launch_fwd_onchip(snac_plan* P, const void* in3, bool in_f32, double shift0, double target, double wait_s,
                              int extra_need, cudaStream_t s) {
  if (!fused_ready(P) || (in_f32 && P->precision != SNAC_MIXED)) return cudaErrorInvalidValue;
  if (P->precision == SNAC_FP64) return fwd_onchip_t<double>(P, in3, in_f32, shift0, target, wait_s, extra_need, s);
  return fwd_onchip_t<float>(P, in3, in_f32, shift0, target, wait_s, extra_need, s);
}

size_t fwd_onchip_batch_scratch(int nplans, int nitems) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up((size_t)nplans * sizeof(FwdArgs<double>)) + up((size_t)nplans * sizeof(OnchipArgs<double>)) +
         up((size_t)nitems * sizeof(int4)) + up((size_t)(1 + nplans) * sizeof(int));
}

template <typename T>
cudaError_t fwd_onchip_batch_t(snac_plan* const* plans, const FusedInput* inputs, const double* targets, int nplans,
                               double wait_s, void* d_scratch, int sms, cudaStream_t s) {
  constexpr int TC = fused_tc<T>();
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  char* base = static_cast<char*>(d_scratch);
  FwdArgs<T>* d_fargs = reinterpret_cast<FwdArgs<T>*>(base);
  OnchipArgs<T>* d_args = reinterpret_cast<OnchipArgs<T>*>(base + up((size_t)nplans * sizeof(FwdArgs<double>)));
  int4* d_items = reinterpret_cast<int4*>(reinterpret_cast<char*>(d_args) + up((size_t)nplans * sizeof(OnchipArgs<double>)));
  std::vector<FwdArgs<T>> fargs(nplans);
  std::vector<OnchipArgs<T>> args(nplans);
  std::vector<int4> items;
  size_t smem = 0;
  for (int k = 0; k < nplans; ++k)
    for (int c = 0; c < (int)(sizeof(T) == 8 ? plans[k]->chunks64.size() : plans[k]->chunks32.size()); ++c)
      items.push_back(make_int4(0, k, c, 0));
  for (int k = 0; k < nplans; ++k)
    for (int q = 0; q < plans[k]->nz; ++q) items.push_back(make_int4(1, k, q, 0));
  int* d_ctr = reinterpret_cast<int*>(reinterpret_cast<char*>(d_items) + up(items.size() * sizeof(int4)));
  for (int k = 0; k < nplans; ++k) {
    snac_plan* P = plans[k];
    *P->h_wait = 0;
    fargs[k] = fwd_args<T>(P, inputs[k].in3, inputs[k].in_f32, inputs[k].shift0, d_ctr + 1 + k, P->dh_wait, 0);
    args[k] = onchip_args<T>(P, targets[k]);
    smem = std::max(smem, fused_smem<T>(P));
    KernelStat& ks = P->kstats[K_FWD_ONCHIP];  // each plan counts the shared launch once
    ++ks.launches;
    const double w = sizeof(T), n3 = (double)P->n3;
    ks.bytes += (inputs[k].in_f32 ? 4.0 : 8.0) * n3 + w * n3 + 2.0 * w * (double)P->lev[0].ncell * P->nz;
    ks.flops += (2.5 * std::log2((double)P->nzt) + 8.0) * n3 + 4.0 * onchip_cycle_flops(P) * P->nz;
  }
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_fargs, fargs.data(), nplans * sizeof(FwdArgs<T>), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_args, args.data(), nplans * sizeof(OnchipArgs<T>), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  k_zero_ints<<<1, 256, 0, s>>>(d_ctr, 1 + nplans);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cudaFuncSetAttribute(k_fwd_onchip_batch<T, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, BOTTOM_MAX_SMEM);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_onchip_batch<T, TC>, BT, smem);
  const int nitems = (int)items.size();
  const int grid = std::max(1, std::min(nitems, std::min(std::max(1, per_sm), 1) * sms));  // one CTA per SM
  k_fwd_onchip_batch<T, TC><<<grid, BT, smem, s>>>(d_fargs, d_args, d_items, nitems, d_ctr, (long long)(wait_s * 1e9));
  return cudaGetLastError();
}

cudaError_t launch_fwd_onchip_batch(snac_plan* const* plans, const FusedInput* inputs, const double* targets,
                                    int nplans, double wait_s, void* d_scratch, int sms, cudaStream_t s) {
  if (nplans <= 0) return cudaSuccess;
  for (int k = 0; k < nplans; ++k)
    if (!fused_ready(plans[k]) || plans[k]->precision != plans[0]->precision) return cudaErrorInvalidValue;
  if (plans[0]->precision == SNAC_FP64)
    return fwd_onchip_batch_t<double>(plans, inputs, targets, nplans, wait_s, d_scratch, sms, s);
  return fwd_onchip_batch_t<float>(plans, inputs, targets, nplans, wait_s, d_scratch, sms, s);
}

// Many plans, one launch: the items (plan index, wavenumber) of plans of the same precision, every
// plan's level-0 right-hand side in place; targets per plan. Device scratch (args, items, counter)
// is the caller's, `scratch_bytes` long (onchip_batch_scratch gives the size).
size_t onchip_batch_scratch(int nplans, int nitems) {
  return ((size_t)nplans * sizeof(OnchipArgs<double>) + 255) / 256 * 256 + ((size_t)nitems * sizeof(int2) + 255) / 256 * 256 + 256;
}

template <typename T>
cudaError_t onchip_batch_t(snac_plan* const* plans, const double* targets, int nplans, const int2* h_items, int nitems,
                           void* d_scratch, int sms, cudaStream_t s) {
  std::vector<OnchipArgs<T>> args(nplans);
  size_t smem = 0;
  for (int k = 0; k < nplans; ++k) {
    args[k] = onchip_args<T>(plans[k], targets[k]);
    smem = std::max(smem, bottom_layout(plans[k], 0, sizeof(T)).bytes);
  }
  char* base = static_cast<char*>(d_scratch);
  OnchipArgs<T>* d_args = reinterpret_cast<OnchipArgs<T>*>(base);
  int2* d_items = reinterpret_cast<int2*>(base + ((size_t)nplans * sizeof(OnchipArgs<double>) + 255) / 256 * 256);
  int* d_next = reinterpret_cast<int*>(reinterpret_cast<char*>(d_items) + ((size_t)nitems * sizeof(int2) + 255) / 256 * 256);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_args, args.data(), nplans * sizeof(OnchipArgs<T>), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d_items, h_items, nitems * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_next, 0, sizeof(int), s)) != cudaSuccess)
    return e;
  cudaFuncSetAttribute(k_onchip_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, BOTTOM_MAX_SMEM);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onchip_batch<T>, BT, smem);
  const int grid = std::max(1, std::min(nitems, std::max(1, per_sm) * sms));
  for (int k = 0; k < nplans; ++k) {  // each plan counts the shared launch once, with its own items
    snac_plan* P = plans[k];
    double n = 0.0;
    for (int i = 0; i < nitems; ++i) n += h_items[i].x == k ? 1.0 : 0.0;
    KernelStat& ks = P->kstats[K_ONCHIP];
    ++ks.launches;
    ks.bytes += 2.0 * sizeof(T) * (double)P->lev[0].ncell * n;
    ks.flops += 4.0 * onchip_cycle_flops(P) * n;
  }
  k_onchip_batch<T><<<grid, BT, smem, s>>>(d_args, d_items, nitems, d_next);
  return cudaGetLastError();
}

cudaError_t launch_onchip_batch(snac_plan* const* plans, const double* targets, int nplans, const int2* h_items,
                                int nitems, void* d_scratch, int sms, cudaStream_t s) {
  if (nplans <= 0 || nitems <= 0) return cudaSuccess;
  if (plans[0]->precision == SNAC_FP64)
    return onchip_batch_t<double>(plans, targets, nplans, h_items, nitems, d_scratch, sms, s);
  return onchip_batch_t<float>(plans, targets, nplans, h_items, nitems, d_scratch, sms, s);
}

}  // namespace snac
