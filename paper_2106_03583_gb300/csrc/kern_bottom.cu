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
#include "kern_common.cuh"
#include "snac_impl.h"

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

// Cell (b, i, j) of the idx-th cell of colour c of a level (blocks in order, rows of each block in
// order, the colour's cells of a row in order of i). Returns false past the last cell.
__device__ __forceinline__ bool colour_cell(const BlockDev* __restrict__ blk, int nblk, int idx, int c, int& b,
                                            BlockDev& B, int& i, int& j) {
  for (b = 0; b < nblk; ++b) {
    B = blk[b];
    const int half = (B.nx >> 1) * B.ny;
    if (idx < half) {
      const int hx = B.nx >> 1;
      j = idx / hx;
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
  j = l / B.nx;
  i = l - j * B.nx;
}

// One Gauss-Seidel half-sweep of colour c on a level.
template <typename T>
__device__ void half_sweep(const LevelView<T>& L, const LevelSmem<T>& S, int c) {
  const int ncol = (int)(L.ncell >> 1);
  for (int idx = threadIdx.x; idx < ncol; idx += BT) {
    int b, i, j;
    BlockDev B;
    if (!colour_cell(L.blk, L.nblk, idx, c, b, B, i, j)) break;
    long long w, e, s, n;
    nbr_plane(L.blk, B, b, i, j, w, e, s, n);
    const int cc = (int)(B.off + (long long)j * B.nx + i);
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
        long long w, e, s, n;
        nbr_plane(F.blk, Bf, b, i, j, w, e, s, n);
        const int c = (int)(Bf.off + (long long)j * Bf.nx + i);
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
    long long w, e, s, n;
    nbr_plane(C.blk, Bc, b, I, J, w, e, s, n);
    const T eC = SC.u[Bc.off + (long long)J * Bc.nx + I];
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
// singular mode), in FP64.
template <typename T>
__device__ void coarse_solve(const double* __restrict__ Q, const double* __restrict__ lam,
                             const double* __restrict__ sqa, int nc, int null_index, const LevelSmem<T>& S, double sg,
                             bool sing, double* b, double* y) {
  for (int i = threadIdx.x; i < nc; i += BT) b[i] = sqa[i] * (double)S.f[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < nc; k += BT / 32) {
    double s = 0.0;
    for (int i = lane; i < nc; i += 32) s = fma(Q[(long long)i * nc + k], b[i], s);
    s = warp_sum(s);
    if (lane == 0) y[k] = (sing && k == null_index) ? 0.0 : s / (lam[k] + sg);
  }
  __syncthreads();
  for (int i = warp; i < nc; i += BT / 32) {
    double s = 0.0;
    for (int k = lane; k < nc; k += 32) s = fma(Q[(long long)i * nc + k], y[k], s);
    s = warp_sum(s);
    if (lane == 0) S.u[i] = (T)(s / sqa[i]);
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
    coarse_solve(A.Q, A.lam, A.sqa, A.nc, A.null_index, level_smem(smem_raw, C, f0g), sg64, sing, b, y);
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
  bytes += 2 * MAX_COARSE * sizeof(double);
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

}  // namespace snac
