// Multigrid for the reduced 2-D equations of every wavenumber (Eq. 9, Sec. 2; Algorithm 1 second
// loop), batched over the active wavenumbers in each launch (grid.y = active mode).
//
// Reduced operator of mode q at one level: (A_xy + sigma_q) u, sigma_q = lambda_q / dz^2 (Table 1),
// with A_xy the x-y part of Eq. 8 rediscretised on the level's widths. V(nu1, nu2) cycle with
// red-black Gauss-Seidel (colour = parity of the global index-space position), area-weighted
// restriction of the residual, three-point affine prolongation, and a direct solve of the coarsest
// plane through the eigen-decomposition of its symmetrised operator.
#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
namespace {

template <typename T>
__device__ __forceinline__ T apply_row(const Coef<T>& cx, const Coef<T>& cy, T diag, T uc, T uw, T ue, T us, T un) {
  T a = cx.lo * uw;
  a = fma(cx.hi, ue, a);
  a = fma(cy.lo, us, a);
  a = fma(cy.hi, un, a);
  return fma(diag, uc, a);
}

// One colour of one Gauss-Seidel sweep: u_c = (f_c - sum_nbr a u_nbr) / diag_c on every cell of that
// colour. 128 threads cover a 32x8 tile: each thread owns the one cell of its row pair that has the
// colour, so every lane of every warp works. FP64 plans read the precomputed inverse diagonal (the
// FP64 pipe is the bound there); FP32 plans form it on the fly.
// SCALED: the level holds g = f / diag instead of f (FP64 plans without fused levels), and the
// update is u_c = g_c - (sum_nbr a u_nbr) / diag_c, one FP64 operation fewer per cell; g and 1/diag
// are in colour-split order (split_cell), so the colour's values are contiguous.
constexpr int COLOUR_THREADS = 128;

template <typename T, bool PRE_INV, bool SCALED>
__global__ void __launch_bounds__(COLOUR_THREADS) k_smooth(LevelView<T> L, const int* __restrict__ active,
                                                            const T* __restrict__ sigma, const double* __restrict__ invd,
                                                            T* __restrict__ u, const T* __restrict__ f, int colour) {
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int j = t.y0 + (threadIdx.x >> 4);
  const int i = t.x0 + 2 * (threadIdx.x & 15) + ((colour ^ B.par ^ j) & 1);
  if (i >= B.nx || j >= B.ny) return;
  const int q = active[blockIdx.y];
  const long long base = (long long)q * L.ncell;
  long long w, e, s, n;
  nbr_plane(L.blk, B, t.b, i, j, w, e, s, n);
  const long long c = B.off + (long long)j * B.nx + i;
  const long long cg = SCALED ? split_cell(B, i, j) : c;  // position of the cell's f and 1/diag
  const Coef<T> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
  T id;
  if constexpr (PRE_INV) {
    id = invd[base + cg];
  } else {
    id = recip(cx.d + cy.d + sigma[q]);
  }
  T a = cx.lo * u[base + w];
  a = fma(cx.hi, u[base + e], a);
  a = fma(cy.lo, u[base + s], a);
  a = fma(cy.hi, u[base + n], a);
  if constexpr (SCALED) u[base + c] = fma(-a, id, f[base + cg]);
  else u[base + c] = (f[base + c] - a) * id;
}

// The first colour-0 half-sweep of the next V-cycle at level 0 of a scaled FP64 plan, which also
// yields the residual norm of the state before it: after a cycle that ends on colour 1 only colour-0
// cells carry a residual, and a colour-0 cell's residual d (g - u) - a uses the neighbour sum a that
// its update forms anyway. Every active mode is updated; each CTA walks tiles blockIdx.x, + gridDim.x,
// ... so that the norm's reduction is paid once per CTA, and writes one partial of r^2 for the modes
// of the (ascending) check list.
constexpr int CHECK_CTAS = 64;

__global__ void __launch_bounds__(COLOUR_THREADS) k_smooth_check(LevelView<double> L, const int* __restrict__ active,
                                                                  const double* __restrict__ sigma,
                                                                  const double* __restrict__ invd, double* __restrict__ u,
                                                                  const double* __restrict__ g,
                                                                  const int* __restrict__ check, int ncheck,
                                                                  double* __restrict__ part) {
  __shared__ double sh[COLOUR_THREADS / 32];
  __shared__ int is_checked;
  const int q = active[blockIdx.y];
  if (threadIdx.x == 0) {
    int lo = 0, hi = ncheck;  // binary search of q in the ascending check list
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (check[mid] < q) lo = mid + 1;
      else hi = mid;
    }
    is_checked = lo < ncheck && check[lo] == q;
  }
  const long long base = (long long)q * L.ncell;
  const double sg = sigma[q];
  double r2 = 0.0;
  for (int tile = blockIdx.x; tile < L.ntiles; tile += gridDim.x) {
    const TileDev t = L.tiles[tile];
    const BlockDev B = L.blk[t.b];
    const int j = t.y0 + (threadIdx.x >> 4);
    const int i = t.x0 + 2 * (threadIdx.x & 15) + ((B.par ^ j) & 1);
    if (i >= B.nx || j >= B.ny) continue;
    long long w, e, s, n;
    nbr_plane(L.blk, B, t.b, i, j, w, e, s, n);
    const long long c = B.off + (long long)j * B.nx + i;
    const long long cg = split_cell(B, i, j);
    const Coef<double> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
    double a = cx.lo * u[base + w];
    a = fma(cx.hi, u[base + e], a);
    a = fma(cy.lo, u[base + s], a);
    a = fma(cy.hi, u[base + n], a);
    const double gv = g[base + cg], u0 = u[base + c];
    u[base + c] = fma(-a, invd[base + cg], gv);
    const double r = fma(L.dxy[c] + sg, gv - u0, -a);
    r2 = fma(r, r, r2);
  }
  __syncthreads();
  if (!is_checked) return;
  r2 = warp_sum(r2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < COLOUR_THREADS / 32; ++k) v += sh[k];
    part[(long long)q * gridDim.x + blockIdx.x] = v;
  }
}

// Residual of cell c with the off-diagonal sum a and the diagonal: f - (a + diag u) from f, or
// diag (g - u) - a from the scaled right-hand side g = f / diag (the same number of operations).
template <typename T, bool SCALED>
__device__ __forceinline__ T cell_residual(const Coef<T>& cx, const Coef<T>& cy, T diag, T fc, T uc, T uw, T ue, T us,
                                           T un) {
  if constexpr (SCALED) {
    T a = cx.lo * uw;
    a = fma(cx.hi, ue, a);
    a = fma(cy.lo, us, a);
    a = fma(cy.hi, un, a);
    return fma(diag, fc - uc, -a);
  } else {
    return fc - apply_row(cx, cy, diag, uc, uw, ue, us, un);
  }
}

__global__ void __launch_bounds__(TILE_THREADS) k_invd(LevelView<double> L, const double* __restrict__ sigma,
                                                        double* __restrict__ invd, int split) {
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  if (i >= B.nx || j >= B.ny) return;
  const int q = blockIdx.y;
  const long long c = split ? split_cell(B, i, j) : B.off + (long long)j * B.nx + i;
  invd[(long long)q * L.ncell + c] = 1.0 / (L.cx[B.xo + i].d + L.cy[B.yo + j].d + sigma[q]);
}

// Plain -> colour-split order of every mode plane of a level (the scaled FP64 levels' f).
__global__ void __launch_bounds__(TILE_THREADS) k_to_split(LevelView<double> L, const double* __restrict__ src,
                                                            double* __restrict__ dst) {
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  if (i >= B.nx || j >= B.ny) return;
  const long long base = (long long)blockIdx.y * L.ncell;
  dst[base + split_cell(B, i, j)] = src[base + B.off + (long long)j * B.nx + i];
}

// Coarse right-hand side = area-weighted average of the fine residual over the four children;
// the coarse iterate starts at zero.
// After a red-black sweep ending on black, every black cell has zero residual (its update solved its
// own row), so with RED_ONLY only the two red children of each coarse cell are evaluated.
// SCALED: the fine level holds f / diag (colour-split order). With invd_c the coarse level does too
// (its right-hand side is written times its inverse diagonal, both in colour-split order), and with
// first_red the coarse level's first colour-0 half-sweep is done here: from a zero iterate it sets
// each colour-0 cell to f / diag, which is the value written, and the coarse smoothing starts with
// colour 1.
template <typename T, bool RED_ONLY, bool SCALED>
__global__ void __launch_bounds__(TILE_THREADS) k_restrict(LevelView<T> F, LevelView<T> C, const int* __restrict__ active,
                                                            const T* __restrict__ sigma, const T* __restrict__ uf,
                                                            const T* __restrict__ ff, T* __restrict__ fc,
                                                            T* __restrict__ uc, const double* __restrict__ invd_c,
                                                            int first_red) {
  const TileDev t = C.tiles[blockIdx.x];
  const BlockDev Bc = C.blk[t.b];
  const int I = t.x0 + (threadIdx.x % TILE_X), J = t.y0 + (threadIdx.x / TILE_X);
  if (I >= Bc.nx || J >= Bc.ny) return;
  const int q = active[blockIdx.y];
  const BlockDev Bf = F.blk[t.b];
  const long long bf = (long long)q * F.ncell;
  const T sg = sigma[q];
  T acc = 0;
#pragma unroll
  for (int dj = 0; dj < 2; ++dj) {
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      const int i = 2 * I + di, j = 2 * J + dj;
      if (RED_ONLY && ((Bf.par + i + j) & 1)) continue;
      long long w, e, s, n;
      nbr_plane(F.blk, Bf, t.b, i, j, w, e, s, n);
      const long long c = Bf.off + (long long)j * Bf.nx + i;
      const Coef<T> cx = F.cx[Bf.xo + i], cy = F.cy[Bf.yo + j];
      const T diag = F.dxy[c] + sg;
      const long long cf = SCALED ? split_cell(Bf, i, j) : c;
      const T r = cell_residual<T, SCALED>(cx, cy, diag, ff[bf + cf], uf[bf + c], uf[bf + w], uf[bf + e], uf[bf + s],
                                           uf[bf + n]);
      acc = fma(F.wr[c], r, acc);  // rx * ry
    }
  }
  const long long cb = (long long)q * C.ncell;
  const long long cc = cb + Bc.off + (long long)J * Bc.nx + I;
  if (invd_c != nullptr) {
    const long long cs = cb + split_cell(Bc, I, J);
    acc *= (T)invd_c[cs];
    fc[cs] = acc;
  } else {
    fc[cc] = acc;
  }
  uc[cc] = (first_red && ((Bc.par + I + J) & 1) == 0) ? acc : (T)0;
}

// u_f += e_C (1 + sx + sy) + nx e_X + ny e_Y: parent C, coarse neighbours X / Y on the fine cell's side.
// With ONE_COLOUR only the cells of `colour` are corrected (COLOUR_THREADS threads per tile, as in
// k_smooth): when a post-smoothing half-sweep of the other colour follows, it overwrites the other
// colour's cells from their neighbours and f alone, so correcting them would be wasted work.
template <typename T, bool ONE_COLOUR>
__global__ void __launch_bounds__(TILE_THREADS) k_prolong(LevelView<T> F, LevelView<T> C, const int* __restrict__ active,
                                                           T* __restrict__ uf, const T* __restrict__ uc, int colour) {
  const TileDev t = F.tiles[blockIdx.x];
  const BlockDev Bf = F.blk[t.b];
  int i, j;
  if (ONE_COLOUR) {
    j = t.y0 + (threadIdx.x >> 4);
    i = t.x0 + 2 * (threadIdx.x & 15) + ((colour ^ Bf.par ^ j) & 1);
  } else {
    i = t.x0 + (threadIdx.x % TILE_X);
    j = t.y0 + (threadIdx.x / TILE_X);
  }
  if (i >= Bf.nx || j >= Bf.ny) return;
  const int q = active[blockIdx.y];
  const BlockDev Bc = C.blk[t.b];
  const int I = i >> 1, J = j >> 1;
  long long w, e, s, n;
  nbr_plane(C.blk, Bc, t.b, I, J, w, e, s, n);
  const long long bc = (long long)q * C.ncell;
  const T eC = uc[bc + Bc.off + (long long)J * Bc.nx + I];
  const T eX = uc[bc + ((i & 1) ? e : w)];
  const T eY = uc[bc + ((j & 1) ? n : s)];
  const PW<T> px = F.px[Bf.xo + i], py = F.py[Bf.yo + j];
  const long long cl = Bf.off + (long long)j * Bf.nx + i;
  const long long c = (long long)q * F.ncell + cl;
  // accumulated into u directly: three FMAs (the FP64 pipe bounds this kernel in FP64 plans); the
  // parent's weight 1 + self_x + self_y comes from the level's table
  T u = fma(eC, F.wp[cl], uf[c]);
  u = fma(px.nbr, eX, u);
  uf[c] = fma(py.nbr, eY, u);
}

// Direct solve of the coarsest plane: with V the cell areas, S = V^1/2 A V^-1/2 = Q Lam Q^T, so
// (A + sigma)^-1 b = V^-1/2 Q (Lam + sigma)^-1 Q^T V^1/2 b. For a singular mode the null eigenvector
// (constant in the V-weighted sense) is dropped: the zero-mean solution. One CTA per mode, in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_coarse(const double* __restrict__ Q, const double* __restrict__ QT,
                                                const double* __restrict__ lam, const double* __restrict__ sqa, int nc,
                                                const int* __restrict__ active, const double* __restrict__ sigma,
                                                const int* __restrict__ singular_mode, int null_index,
                                                const T* __restrict__ fcoarse, T* __restrict__ ucoarse,
                                                long long ncell) {
  __shared__ double b[MAX_COARSE], y[MAX_COARSE];
  const int q = active[blockIdx.x];
  const long long base = (long long)q * ncell;
  for (int i = threadIdx.x; i < nc; i += blockDim.x) b[i] = sqa[i] * (double)fcoarse[base + i];
  __syncthreads();
  const double sg = sigma[q];
  const bool sing = singular_mode[q] != 0;
  // one thread per entry, reading a row of Q^T (then of Q): no cross-lane reductions, and the FP64
  // divisions of the lanes of a warp run together
  for (int k = threadIdx.x; k < nc; k += blockDim.x) {
    const double* qk = QT + (long long)k * nc;
    double s = 0.0;
    for (int i = 0; i < nc; ++i) s = fma(qk[i], b[i], s);
    y[k] = (sing && k == null_index) ? 0.0 : s / (lam[k] + sg);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    const double* qi = Q + (long long)i * nc;
    double s = 0.0;
    for (int k = 0; k < nc; ++k) s = fma(qi[k], y[k], s);
    ucoarse[base + i] = (T)(s / sqa[i]);
  }
}

// out = (A_xy + sigma_q) u for every listed mode.
template <typename T>
__global__ void __launch_bounds__(TILE_THREADS) k_mode_apply(LevelView<T> L, const int* __restrict__ active,
                                                              const T* __restrict__ sigma, const T* __restrict__ u,
                                                              T* __restrict__ out) {
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  if (i >= B.nx || j >= B.ny) return;
  const int q = active[blockIdx.y];
  const long long base = (long long)q * L.ncell;
  long long w, e, s, n;
  nbr_plane(L.blk, B, t.b, i, j, w, e, s, n);
  const long long c = B.off + (long long)j * B.nx + i;
  const Coef<T> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
  const T diag = cx.d + cy.d + sigma[q];
  out[base + c] = apply_row(cx, cy, diag, u[base + c], u[base + w], u[base + e], u[base + s], u[base + n]);
}

// Per-tile partial sums of (f - (A + sigma) u)^2 for every listed mode (FP64 accumulation). With
// RED_ONLY (after a sweep ending on black) only the red cells carry a residual.
template <typename T, bool RED_ONLY, bool SCALED>
__global__ void __launch_bounds__(TILE_THREADS) k_mode_resid2(LevelView<T> L, const int* __restrict__ active,
                                                               const T* __restrict__ sigma, const T* __restrict__ u,
                                                               const T* __restrict__ f, double* __restrict__ part) {
  __shared__ double sh[32];
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  int i, j;
  if (RED_ONLY) {
    j = t.y0 + (threadIdx.x >> 4);
    i = t.x0 + 2 * (threadIdx.x & 15) + ((B.par ^ j) & 1);
  } else {
    i = t.x0 + (threadIdx.x % TILE_X);
    j = t.y0 + (threadIdx.x / TILE_X);
  }
  const int q = active[blockIdx.y];
  T r2 = 0;
  if (i < B.nx && j < B.ny) {
    const long long base = (long long)q * L.ncell;
    long long w, e, s, n;
    nbr_plane(L.blk, B, t.b, i, j, w, e, s, n);
    const long long c = B.off + (long long)j * B.nx + i;
    const Coef<T> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
    const T diag = L.dxy[c] + sigma[q];
    const T r = cell_residual<T, SCALED>(cx, cy, diag, f[base + (SCALED ? split_cell(B, i, j) : c)], u[base + c],
                                         u[base + w], u[base + e], u[base + s], u[base + n]);
    r2 = r * r;
  }
  r2 = warp_sum_t(r2);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = (double)r2;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) part[(long long)q * L.ntiles + blockIdx.x] = v;
  }
}

// Per-tile partial sums of f^2 (the residual of a zero iterate) for every listed mode: a plain
// streaming pass over the plane, one partial per CTA-row of MODE_SQ_CTAS CTAs. With u, the listed
// modes' iterate is set to zero in the same pass.
constexpr int MODE_SQ_CTAS = 64;

template <typename T>
__global__ void __launch_bounds__(256) k_mode_sumsq(const T* __restrict__ f, long long ncell, const int* __restrict__ active,
                                                    double* __restrict__ part, T* __restrict__ u) {
  __shared__ double sh[32];
  const int q = active[blockIdx.y];
  const T* fq = f + (long long)q * ncell;
  T* uq = u ? u + (long long)q * ncell : nullptr;
  T s = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const T v = fq[c];
    s = fma(v, v, s);
    if (uq) uq[c] = 0;
  }
  s = warp_sum_t(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = (double)s;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) part[(long long)q * MODE_SQ_CTAS + blockIdx.x] = v;
  }
}

// The same sums for the right-hand side as the transform left it, which is then scaled in place by
// the level's inverse diagonal (the form the SCALED kernels read).
__global__ void __launch_bounds__(256) k_mode_sumsq_scale(double* __restrict__ f, const double* __restrict__ invd,
                                                          long long ncell, const int* __restrict__ active,
                                                          double* __restrict__ part, double* __restrict__ u) {
  __shared__ double sh[32];
  const int q = active[blockIdx.y];
  double* fq = f + (long long)q * ncell;
  const double* iq = invd + (long long)q * ncell;
  double* uq = u ? u + (long long)q * ncell : nullptr;
  double s = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x) {
    const double v = fq[c];
    s = fma(v, v, s);
    fq[c] = v * iq[c];
    if (uq) uq[c] = 0.0;
  }
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) part[(long long)q * MODE_SQ_CTAS + blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(256) k_mode_reduce(const double* __restrict__ part, int ntiles,
                                                     const int* __restrict__ active, double* __restrict__ norm2) {
  __shared__ double sh[32];
  const int q = active[blockIdx.x];
  double s = 0.0;
  for (int k = threadIdx.x; k < ntiles; k += blockDim.x) s += part[(long long)q * ntiles + k];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) norm2[q] = v;
  }
}

template <typename T>
const T* sigma_ptr(const snac_plan* P);
template <>
const double* sigma_ptr<double>(const snac_plan* P) { return P->d_sigma64; }
template <>
const float* sigma_ptr<float>(const snac_plan* P) { return P->d_sigma32; }

template <typename T>
cudaError_t vcycle_t(snac_plan* P, int nact, cudaStream_t st, bool skip_first0) {
  const int L = (int)P->lev.size() - 1;
  const T* sg = sigma_ptr<T>(P);
  const int* act = P->d_active;
  const double w = sizeof(T);
  constexpr bool pre_inv = sizeof(T) == 8;
  // FP64 plans without fused levels: the smoothed levels hold f / diag (see k_smooth)
  const bool scaled = sizeof(T) == 8 && P->scaled_f;
  auto smooth = [&](int l, int nu, bool skip_first) {
    const HostLevel& h = P->lev[l];
    const LevelView<T> V = level_view<T>(h);
    dim3 g((unsigned)h.tiles.size(), (unsigned)nact);
    const double cells = (double)h.ncell * nact;
    for (int it = 0; it < nu; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        if (skip_first && it == 0 && colour == 0) continue;  // done by the restriction
        // Gauss-Seidel half-sweep: read the other colour and f of this colour, write this colour
        LaunchScope ls(P, K_SMOOTH, 1.5 * w * cells, (pre_inv ? 9.0 : 12.0) * 0.5 * cells, st);
        auto go = [&](auto kern) {
          kern<<<g, COLOUR_THREADS, 0, st>>>(V, act, sg, h.d_invd, (T*)h.d_u, (const T*)h.d_f, colour);
        };
        if constexpr (sizeof(T) == 8) {
          if (scaled) go(k_smooth<T, pre_inv, true>);
          else go(k_smooth<T, pre_inv, false>);
        } else {
          go(k_smooth<T, pre_inv, false>);
        }
      }
  };
  // levels from P->bottom on run as one sub-cycle launch (kern_bottom.cu); above it level by level
  const int top = P->bottom > 0 ? P->bottom : L;
  for (int l = 0; l < top; ++l) {
    const HostLevel& h = P->lev[l];
    const HostLevel& hc = P->lev[l + 1];
    if (h.fused) {
      // the coarse iterate of a fused level below starts at zero without being read; a per-colour
      // level below reads it, so it is written as zero
      const bool zero_coarse = l + 1 < L && !hc.fused;
      cudaError_t e = launch_fused_down(P, l, nact, l > 0, zero_coarse, st);
      if (e != cudaSuccess) return e;
      continue;
    }
    // a level below 0 starts from zero: with scaled right-hand sides its first colour-0 half-sweep
    // is folded into the restriction that fills it; at level 0 the norm check may have done it
    smooth(l, P->nu1, (scaled && l > 0 && P->nu1 > 0) || (l == 0 && skip_first0));
    dim3 g((unsigned)hc.tiles.size(), (unsigned)nact);
    const double cells = (double)h.ncell * nact;
    const bool coarse_smoothed = l + 1 < top;  // the sub-cycle's top level takes a plain f
    const double* invd_c = scaled && coarse_smoothed ? hc.d_invd : nullptr;
    const int first_red = scaled && coarse_smoothed && P->nu1 > 0 ? 1 : 0;
    LaunchScope ls(P, K_RESTRICT, (2.5 + (invd_c ? 0.25 : 0.0)) * w * cells, (P->nu1 > 0 ? 7.5 : 15.0) * cells, st);
    auto restrict_k = [&](auto kern) {
      kern<<<g, TILE_THREADS, 0, st>>>(level_view<T>(h), level_view<T>(hc), act, sg, (const T*)h.d_u,
                                       (const T*)h.d_f, (T*)hc.d_f, (T*)hc.d_u, invd_c, first_red);
    };
    if constexpr (sizeof(T) == 8) {
      if (scaled && P->nu1 > 0) restrict_k(k_restrict<T, true, true>);
      else if (scaled) restrict_k(k_restrict<T, false, true>);
      else if (P->nu1 > 0) restrict_k(k_restrict<T, true, false>);
      else restrict_k(k_restrict<T, false, false>);
    } else {
      if (P->nu1 > 0) restrict_k(k_restrict<T, true, false>);
      else restrict_k(k_restrict<T, false, false>);
    }
  }
  if (top < L) {
    cudaError_t e = launch_bottom(P, nact, st);
    if (e != cudaSuccess) return e;
  } else {
    const HostLevel& h = P->lev[L];
    LaunchScope ls(P, K_COARSE, 2.0 * w * P->nc * nact + 8.0 * P->nc * P->nc, 4.0 * P->nc * P->nc * nact, st);
    k_coarse<T><<<nact, 256, 0, st>>>(P->d_Q, P->d_QT, P->d_lam, P->d_sqa, P->nc, act, P->d_sigma64, P->d_singular_mode,
                                      P->null_index, (const T*)h.d_f, (T*)h.d_u, h.ncell);
  }
  for (int l = top - 1; l >= 0; --l) {
    const HostLevel& h = P->lev[l];
    const HostLevel& hc = P->lev[l + 1];
    if (h.fused) {
      cudaError_t e = launch_fused_up(P, l, nact, l == 0, st);
      if (e != cudaSuccess) return e;
      continue;
    }
    dim3 g((unsigned)h.tiles.size(), (unsigned)nact);
    {
      const double cells = (double)h.ncell * nact;
      if (P->nu2 > 0) {
        // post-smoothing starts with colour 0: correct the colour-1 cells only (read and write u
        // there, read the coarse correction)
        LaunchScope ls(P, K_PROLONG, 1.25 * w * cells, 3.5 * cells, st);
        k_prolong<T, true><<<g, COLOUR_THREADS, 0, st>>>(level_view<T>(h), level_view<T>(hc), act, (T*)h.d_u,
                                                          (const T*)hc.d_u, 1);
      } else {
        LaunchScope ls(P, K_PROLONG, 2.25 * w * cells, 7.0 * cells, st);
        k_prolong<T, false><<<g, TILE_THREADS, 0, st>>>(level_view<T>(h), level_view<T>(hc), act, (T*)h.d_u,
                                                         (const T*)hc.d_u, 0);
      }
    }
    smooth(l, P->nu2, false);
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t mode_norms_t(snac_plan* P, int nact, bool after_cycle, cudaStream_t st, const int* list, bool zero_u) {
  const HostLevel& h = P->lev[0];
  const bool scaled = sizeof(T) == 8 && P->scaled_f;
  if (!after_cycle) {  // zero iterate: the residual is the right-hand side itself
    if (scaled) {  // ... which is then scaled into the form the smoothed levels hold
      LaunchScope ls(P, K_MODE_RESID, (zero_u ? 4.0 : 3.0) * sizeof(T) * h.ncell * nact, 3.0 * h.ncell * nact, st);
      k_mode_sumsq_scale<<<dim3(MODE_SQ_CTAS, nact), 256, 0, st>>>((double*)h.d_f, h.d_invd, h.ncell, list,
                                                                   P->d_mode_part, zero_u ? (double*)h.d_u : nullptr);
    } else {
      LaunchScope ls(P, K_MODE_RESID, (zero_u ? 2.0 : 1.0) * sizeof(T) * h.ncell * nact, 2.0 * h.ncell * nact, st);
      k_mode_sumsq<T><<<dim3(MODE_SQ_CTAS, nact), 256, 0, st>>>((const T*)h.d_f, h.ncell, list, P->d_mode_part,
                                                                zero_u ? (T*)h.d_u : nullptr);
    }
    LaunchScope ls(P, K_MODE_REDUCE, 8.0 * MODE_SQ_CTAS * nact, (double)MODE_SQ_CTAS * nact, st);
    k_mode_reduce<<<nact, 256, 0, st>>>(P->d_mode_part, MODE_SQ_CTAS, list, P->d_mode_norm2);
    return cudaGetLastError();
  }
  if (after_cycle && h.fused) {  // the level-0 up kernel left one partial per fused tile
    LaunchScope ls(P, K_MODE_REDUCE, 8.0 * h.ftiles.size() * nact, (double)h.ftiles.size() * nact, st);
    k_mode_reduce<<<nact, 256, 0, st>>>(P->d_mode_part, (int)h.ftiles.size(), list, P->d_mode_norm2);
    return cudaGetLastError();
  }
  dim3 g((unsigned)h.tiles.size(), (unsigned)nact);
  const double cells = (double)h.ncell * nact;
  {
    // after post-smoothing only the red cells carry a residual (read u everywhere, f on red cells)
    const bool red = after_cycle && P->nu2 > 0 && P->lev.size() > 1;
    LaunchScope ls(P, K_MODE_RESID, (red ? 1.5 : 2.0) * sizeof(T) * cells, (red ? 7.0 : 14.0) * cells, st);
    auto resid = [&](auto kern, int threads) {
      kern<<<g, threads, 0, st>>>(level_view<T>(h), list, sigma_ptr<T>(P), (const T*)h.d_u, (const T*)h.d_f,
                                  P->d_mode_part);
    };
    // a single-level plan never scales (its one level is the coarsest, solved directly)
    if constexpr (sizeof(T) == 8) {
      if (scaled && red) resid(k_mode_resid2<T, true, true>, COLOUR_THREADS);
      else if (scaled) resid(k_mode_resid2<T, false, true>, TILE_THREADS);
      else if (red) resid(k_mode_resid2<T, true, false>, COLOUR_THREADS);
      else resid(k_mode_resid2<T, false, false>, TILE_THREADS);
    } else {
      if (red) resid(k_mode_resid2<T, true, false>, COLOUR_THREADS);
      else resid(k_mode_resid2<T, false, false>, TILE_THREADS);
    }
  }
  LaunchScope ls(P, K_MODE_REDUCE, 8.0 * h.tiles.size() * nact, (double)h.tiles.size() * nact, st);
  k_mode_reduce<<<nact, 256, 0, st>>>(P->d_mode_part, (int)h.tiles.size(), list, P->d_mode_norm2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t mode_operator_t(snac_plan* P, const void* u, void* out, cudaStream_t st) {
  const HostLevel& h = P->lev[0];
  dim3 g((unsigned)h.tiles.size(), (unsigned)P->nz);
  const double cells = (double)h.ncell * P->nz;
  LaunchScope ls(P, K_MODE_APPLY, 2.0 * sizeof(T) * cells, 12.0 * cells, st);
  k_mode_apply<T><<<g, TILE_THREADS, 0, st>>>(level_view<T>(h), P->d_active, sigma_ptr<T>(P), (const T*)u, (T*)out);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_inverse_diagonals(snac_plan* P, cudaStream_t s) {
  for (size_t l = 0; l + 1 < P->lev.size(); ++l) {
    const HostLevel& h = P->lev[l];
    dim3 g((unsigned)h.tiles.size(), (unsigned)P->nz);
    k_invd<<<g, TILE_THREADS, 0, s>>>(level_view<double>(h), P->d_sigma64, h.d_invd, P->scaled_f ? 1 : 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_to_split(snac_plan* P, const double* src, double* dst, cudaStream_t s) {
  const HostLevel& h = P->lev[0];
  dim3 g((unsigned)h.tiles.size(), (unsigned)P->nz);
  k_to_split<<<g, TILE_THREADS, 0, s>>>(level_view<double>(h), src, dst);
  return cudaGetLastError();
}

cudaError_t launch_vcycle(snac_plan* P, int nact, cudaStream_t s, bool skip_first0) {
  if (nact <= 0) return cudaSuccess;
  return P->precision == SNAC_FP64 ? vcycle_t<double>(P, nact, s, skip_first0)
                                   : vcycle_t<float>(P, nact, s, skip_first0);
}

cudaError_t launch_check_sweep(snac_plan* P, int nact, int ncheck, cudaStream_t s) {
  if (nact <= 0) return cudaSuccess;
  const HostLevel& h = P->lev[0];
  const int ctas = std::min<int>(CHECK_CTAS, (int)h.tiles.size());
  dim3 g((unsigned)ctas, (unsigned)nact);
  const double cells = (double)h.ncell * nact;
  {
    // the half-sweep's traffic (other colour, g and 1/diag of this colour, write this colour) plus u of
    // this colour; the update's 9 flops and the residual's 5 per colour-0 cell
    LaunchScope ls(P, K_SMOOTH, 2.0 * 8.0 * cells, 7.0 * cells, s);
    k_smooth_check<<<g, COLOUR_THREADS, 0, s>>>(level_view<double>(h), P->d_active, P->d_sigma64, h.d_invd,
                                                 (double*)h.d_u, (const double*)h.d_f, P->d_check, ncheck,
                                                 P->d_mode_part);
  }
  LaunchScope ls(P, K_MODE_REDUCE, 8.0 * ctas * ncheck, (double)ctas * ncheck, s);
  k_mode_reduce<<<ncheck, 256, 0, s>>>(P->d_mode_part, ctas, P->d_check, P->d_mode_norm2);
  return cudaGetLastError();
}

cudaError_t launch_mode_norms(snac_plan* P, int nact, bool after_cycle, cudaStream_t s, const int* d_list,
                              bool zero_u) {
  if (nact <= 0) return cudaSuccess;
  const int* list = d_list ? d_list : P->d_active;
  return P->precision == SNAC_FP64 ? mode_norms_t<double>(P, nact, after_cycle, s, list, zero_u && !after_cycle)
                                   : mode_norms_t<float>(P, nact, after_cycle, s, list, zero_u && !after_cycle);
}

// Requires d_active = 0..n_z-1.
cudaError_t launch_mode_operator(snac_plan* P, const void* u, void* out, cudaStream_t s) {
  return P->precision == SNAC_FP64 ? mode_operator_t<double>(P, u, out, s) : mode_operator_t<float>(P, u, out, s);
}

}  // namespace snac
