// Fused multigrid tile kernels for FP32 plans (the reduced equations of Eq. 9; Algorithm 1, second
// loop). On GB300 the FP32 multigrid is bound by HBM traffic, so each level of a V-cycle runs as two
// kernels that keep a tile of the plane in shared memory:
//
//   k_fdown: load u, f on the tile plus a halo of FH cells -> nu1 red-black sweeps in shared memory
//            -> write the tile's u -> residual on its red cells -> area-weighted restriction into the
//            coarse right-hand side;
//   k_fup:   load u, f on the tile plus halo and the coarse correction around it -> three-point
//            prolongation and correction -> nu2 sweeps -> write the tile's u (on level 0 also the
//            per-mode sums of squared residuals).
//
// Each red-black half-sweep makes one more ring of the window stale, so after 2 nu half-sweeps the
// tile plus one ring is exact when FH >= 2 nu + 1 (FH = 5 allows nu <= 2): the result equals the
// global Gauss-Seidel sweep. Window cells outside the tile's block belong to the connected blocks
// (a 3x3 table of regions built from the block connectivity, corners through either neighbour);
// each window cell uses the coefficients of the block that owns it, so sweeps across block
// interfaces are exact too. Cells with no owner (beyond a physical face, a re-entrant corner) stay 0
// and are never coupled (their coupling coefficient is 0). The halo must fit inside the neighbouring
// blocks: levels whose blocks are all at least 16 cells wide use these kernels.
#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
namespace {

constexpr int FH = 5;
constexpr int WX = FTILE_X + 2 * FH, WY = FTILE_Y + 2 * FH;  // window
constexpr int CWX = FTILE_X / 2 + 8, CWY = FTILE_Y / 2 + 8;  // coarse window (parents +- 1 ring)
constexpr int FTHREADS = 256;

struct Regions {
  int blk[3][3];  // [ry][rx], ry/rx = 0 (south/west), 1 (the tile's block), 2 (north/east); -1: none
};

__device__ __forceinline__ int nbr_of(const BlockDev* blk, int b, int f) { return b < 0 ? -1 : blk[b].nbr[f]; }

__device__ void build_regions(const BlockDev* __restrict__ blk, int b, Regions& R) {
  const BlockDev& B = blk[b];
  const int W = B.nbr[0], E = B.nbr[1], S = B.nbr[2], N = B.nbr[3];
  R.blk[1][1] = b;
  R.blk[1][0] = W;
  R.blk[1][2] = E;
  R.blk[0][1] = S;
  R.blk[2][1] = N;
  int sw = nbr_of(blk, W, 2);
  if (sw < 0) sw = nbr_of(blk, S, 0);
  int se = nbr_of(blk, E, 2);
  if (se < 0) se = nbr_of(blk, S, 1);
  int nw = nbr_of(blk, W, 3);
  if (nw < 0) nw = nbr_of(blk, N, 0);
  int ne = nbr_of(blk, E, 3);
  if (ne < 0) ne = nbr_of(blk, N, 1);
  R.blk[0][0] = sw;
  R.blk[0][2] = se;
  R.blk[2][0] = nw;
  R.blk[2][2] = ne;
}

// Region index of a block-local coordinate along one axis, and the coordinate inside that region's
// block (n = the tile block's extent, nr = the region block's extent).
__device__ __forceinline__ int region_of(int i, int n) { return i < 0 ? 0 : (i >= n ? 2 : 1); }
__device__ __forceinline__ int local_in(int i, int r, int n, int nr) { return r == 0 ? i + nr : (r == 2 ? i - n : i); }

template <typename T>
struct Shared {
  T u[WY][WX];
  T f[WY][WX];
  Coef<T> xc[3][WX];  // x-pieces of window column wi in region row ry
  Coef<T> yc[3][WY];  // y-pieces of window row wj in region column rx
  PW<T> px[3][WX];
  PW<T> py[3][WY];
  T e[CWY][CWX];
  Regions R;
  double wsum[FTHREADS / 32];
};

// Per-CTA set-up: regions, coefficient (and prolongation weight) tables, window of u and f.
template <typename T, bool PROLONG>
__device__ void load_window(Shared<T>& S, const LevelView<T>& F, const TileDev& t, int tw, int th, long long base,
                            const T* __restrict__ u, const T* __restrict__ f, bool zero_u) {
  // u is never the buffer the same launch writes: neighbouring CTAs store their smoothed tiles while
  // this one may still be loading its halo (the caller alternates two iterate buffers)
  if (threadIdx.x == 0) build_regions(F.blk, t.b, S.R);
  __syncthreads();
  const BlockDev& B = F.blk[t.b];
  const int x0 = t.x0 - FH, y0 = t.y0 - FH;
  for (int idx = threadIdx.x; idx < 3 * WX; idx += blockDim.x) {
    const int ry = idx / WX, wi = idx % WX;
    const int i = x0 + wi, rx = region_of(i, B.nx);
    const int rb = S.R.blk[ry][rx];
    Coef<T> c{0, 0, -1, 1};
    PW<T> w{0, 0};
    if (rb >= 0 && wi < tw + 2 * FH) {
      const BlockDev& RB = F.blk[rb];
      const int ii = local_in(i, rx, B.nx, RB.nx);
      if (ii >= 0 && ii < RB.nx) {
        c = F.cx[RB.xo + ii];
        if (PROLONG) w = F.px[RB.xo + ii];
      }
    }
    S.xc[ry][wi] = c;
    if (PROLONG) S.px[ry][wi] = w;
  }
  for (int idx = threadIdx.x; idx < 3 * WY; idx += blockDim.x) {
    const int rx = idx / WY, wj = idx % WY;
    const int j = y0 + wj, ry = region_of(j, B.ny);
    const int rb = S.R.blk[ry][rx];
    Coef<T> c{0, 0, -1, 1};
    PW<T> w{0, 0};
    if (rb >= 0 && wj < th + 2 * FH) {
      const BlockDev& RB = F.blk[rb];
      const int jj = local_in(j, ry, B.ny, RB.ny);
      if (jj >= 0 && jj < RB.ny) {
        c = F.cy[RB.yo + jj];
        if (PROLONG) w = F.py[RB.yo + jj];
      }
    }
    S.yc[rx][wj] = c;
    if (PROLONG) S.py[rx][wj] = w;
  }
  for (int idx = threadIdx.x; idx < WX * WY; idx += blockDim.x) {
    const int wj = idx / WX, wi = idx % WX;
    T uv = 0, fv = 0;
    if (wi < tw + 2 * FH && wj < th + 2 * FH) {
      const int i = x0 + wi, j = y0 + wj;
      const int rx = region_of(i, B.nx), ry = region_of(j, B.ny);
      const int rb = S.R.blk[ry][rx];
      if (rb >= 0) {
        const BlockDev& RB = F.blk[rb];
        const int ii = local_in(i, rx, B.nx, RB.nx), jj = local_in(j, ry, B.ny, RB.ny);
        if (ii >= 0 && ii < RB.nx && jj >= 0 && jj < RB.ny) {
          const long long a = base + RB.off + (long long)jj * RB.nx + ii;
          if (!zero_u) uv = u[a];
          fv = f[a];
        }
      }
    }
    S.u[wj][wi] = uv;
    S.f[wj][wi] = fv;
  }
}

// Is window cell (wi, wj) owned by a block (inside the clipped window)?
template <typename T>
__device__ __forceinline__ bool owned(const Shared<T>& S, const BlockDev& B, int x0w, int y0w, int wi, int wj, int tw,
                                      int th) {
  if (wi >= tw + 2 * FH || wj >= th + 2 * FH) return false;
  const int rx = region_of(x0w + wi, B.nx), ry = region_of(y0w + wj, B.ny);
  return S.R.blk[ry][rx] >= 0;
}

// nu red-black Gauss-Seidel sweeps on the window; half-sweep s updates the ring-s-shrunk window.
template <typename T>
__device__ void sweeps(Shared<T>& S, const BlockDev& B, int tx0, int ty0, int tw, int th, T sg, int nu) {
  const int x0w = tx0 - FH, y0w = ty0 - FH;
  for (int s = 1; s <= 2 * nu; ++s) {
    const int colour = (s - 1) & 1;
    const int wx1 = tw + 2 * FH - s, wy1 = th + 2 * FH - s;  // exclusive upper bounds
    const int rows = wy1 - s, half = (wx1 - s + 1) / 2;
    for (int idx = threadIdx.x; idx < rows * half; idx += blockDim.x) {
      const int wj = s + idx / half;
      const int k = idx - (idx / half) * half;
      const int base = B.par + x0w + y0w + wj;
      const int wi = s + 2 * k + ((colour - base - s) & 1);
      if (wi >= wx1) continue;
      const int rx = region_of(x0w + wi, B.nx), ry = region_of(y0w + wj, B.ny);
      if (S.R.blk[ry][rx] < 0) continue;
      const Coef<T> cx = S.xc[ry][wi], cy = S.yc[rx][wj];
      T a = cx.lo * S.u[wj][wi - 1];
      a = fma(cx.hi, S.u[wj][wi + 1], a);
      a = fma(cy.lo, S.u[wj - 1][wi], a);
      a = fma(cy.hi, S.u[wj + 1][wi], a);
      S.u[wj][wi] = (S.f[wj][wi] - a) / (cx.d + cy.d + sg);
    }
    __syncthreads();
  }
}

// Residual of window cell (wi, wj) of the tile's own block.
template <typename T>
__device__ __forceinline__ T resid_at(const Shared<T>& S, int wi, int wj, T sg) {
  const Coef<T> cx = S.xc[1][wi], cy = S.yc[1][wj];
  T a = cx.lo * S.u[wj][wi - 1];
  a = fma(cx.hi, S.u[wj][wi + 1], a);
  a = fma(cy.lo, S.u[wj - 1][wi], a);
  a = fma(cy.hi, S.u[wj + 1][wi], a);
  a = fma(cx.d + cy.d + sg, S.u[wj][wi], a);
  return S.f[wj][wi] - a;
}

template <typename T>
__device__ void store_tile(const Shared<T>& S, const BlockDev& B, const TileDev& t, int tw, int th, long long base,
                           T* __restrict__ u) {
  for (int idx = threadIdx.x; idx < FTILE_X * FTILE_Y; idx += blockDim.x) {
    const int ti = idx % FTILE_X, tj = idx / FTILE_X;
    if (ti < tw && tj < th) u[base + B.off + (long long)(t.y0 + tj) * B.nx + t.x0 + ti] = S.u[tj + FH][ti + FH];
  }
}

template <typename T>
__global__ void __launch_bounds__(FTHREADS) k_fdown(LevelView<T> F, LevelView<T> C, const TileDev* __restrict__ ftiles,
                                                     const int* __restrict__ active, const T* __restrict__ sigma,
                                                     const T* __restrict__ u, T* __restrict__ u_out,
                                                     const T* __restrict__ f, T* __restrict__ fc,
                                                     T* __restrict__ uc, int nu, int zero_u, int zero_coarse) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T>& S = *reinterpret_cast<Shared<T>*>(smem_raw);
  const TileDev t = ftiles[blockIdx.x];
  const int q = active[blockIdx.y];
  const BlockDev B = F.blk[t.b];
  const int tw = min(FTILE_X, B.nx - t.x0), th = min(FTILE_Y, B.ny - t.y0);
  const long long base = (long long)q * F.ncell;
  const T sg = sigma[q];
  load_window<T, false>(S, F, t, tw, th, base, u, f, zero_u != 0);
  __syncthreads();
  sweeps(S, B, t.x0, t.y0, tw, th, sg, nu);
  store_tile(S, B, t, tw, th, base, u_out);
  // restriction of the residual: after a sweep ending on black only red children carry one
  const BlockDev Bc = C.blk[t.b];
  const long long cbase = (long long)q * C.ncell;
  const int cw = (tw + 1) / 2, ch = (th + 1) / 2;
  for (int idx = threadIdx.x; idx < cw * ch; idx += blockDim.x) {
    const int ci = idx % cw, cj = idx / cw;
    const int I = t.x0 / 2 + ci, J = t.y0 / 2 + cj;
    if (I >= Bc.nx || J >= Bc.ny) continue;
    T acc = 0;
#pragma unroll
    for (int dj = 0; dj < 2; ++dj)
#pragma unroll
      for (int di = 0; di < 2; ++di) {
        const int i = 2 * I + di, j = 2 * J + dj;
        if (nu > 0 && ((B.par + i + j) & 1)) continue;
        const T r = resid_at(S, i - t.x0 + FH, j - t.y0 + FH, sg);
        acc = fma(F.rx[B.xo + i] * F.ry[B.yo + j], r, acc);
      }
    const long long cc = cbase + Bc.off + (long long)J * Bc.nx + I;
    fc[cc] = acc;
    if (zero_coarse) uc[cc] = 0;
  }
}

template <typename T>
__global__ void __launch_bounds__(FTHREADS) k_fup(LevelView<T> F, LevelView<T> C, const TileDev* __restrict__ ftiles,
                                                   int nftiles, const int* __restrict__ active,
                                                   const T* __restrict__ sigma, const T* __restrict__ u,
                                                   T* __restrict__ u_out, const T* __restrict__ f,
                                                   const T* __restrict__ uc, int nu, double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Shared<T>& S = *reinterpret_cast<Shared<T>*>(smem_raw);
  const TileDev t = ftiles[blockIdx.x];
  const int q = active[blockIdx.y];
  const BlockDev B = F.blk[t.b];
  const int tw = min(FTILE_X, B.nx - t.x0), th = min(FTILE_Y, B.ny - t.y0);
  const long long base = (long long)q * F.ncell;
  const T sg = sigma[q];
  load_window<T, true>(S, F, t, tw, th, base, u, f, false);
  // coarse window: parents of the window cells and one more ring, in the coarse block's coordinates
  const BlockDev Bc = C.blk[t.b];
  const int cx0 = t.x0 / 2 - 4, cy0 = t.y0 / 2 - 4;
  const long long cbase = (long long)q * C.ncell;
  for (int idx = threadIdx.x; idx < CWX * CWY; idx += blockDim.x) {
    const int cj = idx / CWX, ci = idx % CWX;
    const int I = cx0 + ci, J = cy0 + cj;
    const int rx = region_of(I, Bc.nx), ry = region_of(J, Bc.ny);
    const int rb = S.R.blk[ry][rx];
    T v = 0;
    if (rb >= 0) {
      const BlockDev& RB = C.blk[rb];
      const int ii = local_in(I, rx, Bc.nx, RB.nx), jj = local_in(J, ry, Bc.ny, RB.ny);
      if (ii >= 0 && ii < RB.nx && jj >= 0 && jj < RB.ny) v = uc[cbase + RB.off + (long long)jj * RB.nx + ii];
    }
    S.e[cj][ci] = v;
  }
  __syncthreads();
  // three-point prolongation of the coarse correction onto every owned window cell
  const int x0w = t.x0 - FH, y0w = t.y0 - FH;
  for (int idx = threadIdx.x; idx < WX * WY; idx += blockDim.x) {
    const int wj = idx / WX, wi = idx % WX;
    if (!owned(S, B, x0w, y0w, wi, wj, tw, th)) continue;
    const int i = x0w + wi, j = y0w + wj;
    const int rx = region_of(i, B.nx), ry = region_of(j, B.ny);
    const int ci = (i >> 1) - cx0, cj = (j >> 1) - cy0;
    const PW<T> px = S.px[ry][wi], py = S.py[rx][wj];
    const T eC = S.e[cj][ci];
    const T eX = S.e[cj][(i & 1) ? ci + 1 : ci - 1];
    const T eY = S.e[(j & 1) ? cj + 1 : cj - 1][ci];
    S.u[wj][wi] += fma(eC, (T)1 + px.self + py.self, fma(px.nbr, eX, py.nbr * eY));
  }
  __syncthreads();
  sweeps(S, B, t.x0, t.y0, tw, th, sg, nu);
  store_tile(S, B, t, tw, th, base, u_out);
  if (part == nullptr) return;
  // sum of squared residuals of the tile (only red cells carry one after a sweep ending on black)
  double r2 = 0.0;
  for (int idx = threadIdx.x; idx < FTILE_X * FTILE_Y; idx += blockDim.x) {
    const int ti = idx % FTILE_X, tj = idx / FTILE_X;
    if (ti >= tw || tj >= th) continue;
    if (nu > 0 && ((B.par + t.x0 + ti + t.y0 + tj) & 1)) continue;
    const T r = resid_at(S, ti + FH, tj + FH, sg);
    r2 += (double)r * (double)r;
  }
  r2 = warp_sum(r2);
  if ((threadIdx.x & 31) == 0) S.wsum[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < FTHREADS / 32; ++w) s += S.wsum[w];
    part[(long long)q * nftiles + blockIdx.x] = s;
  }
}

template <typename T>
cudaError_t fused_down_t(snac_plan* P, int l, int nact, bool zero_u, bool zero_coarse, const T* sigma, cudaStream_t s) {
  const HostLevel& h = P->lev[l];
  const HostLevel& hc = P->lev[l + 1];
  dim3 g((unsigned)h.ftiles.size(), (unsigned)nact);
  const double cells = (double)h.ncell * nact, w = sizeof(T);
  const size_t smem = sizeof(Shared<T>);
  cudaFuncSetAttribute(k_fdown<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // read u (unless zero) and f, write u and the coarse right-hand side
  LaunchScope ls(P, K_FDOWN, w * cells * ((zero_u ? 2.0 : 3.0) + 0.25 + (zero_coarse ? 0.25 : 0.0)),
                 cells * (2.0 * P->nu1 * 11.0 + 7.5), s);
  // iterate: read d_u, write d_u2 (the up kernel of this level reads d_u2 and writes d_u back)
  k_fdown<T><<<g, FTHREADS, smem, s>>>(level_view<T>(h), level_view<T>(hc), h.d_ftiles, P->d_active, sigma,
                                       (const T*)h.d_u, (T*)h.d_u2, (const T*)h.d_f, (T*)hc.d_f, (T*)hc.d_u, P->nu1,
                                       zero_u ? 1 : 0, zero_coarse ? 1 : 0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t fused_up_t(snac_plan* P, int l, int nact, bool norms, const T* sigma, cudaStream_t s) {
  const HostLevel& h = P->lev[l];
  const HostLevel& hc = P->lev[l + 1];
  dim3 g((unsigned)h.ftiles.size(), (unsigned)nact);
  const double cells = (double)h.ncell * nact, w = sizeof(T);
  const size_t smem = sizeof(Shared<T>);
  cudaFuncSetAttribute(k_fup<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  // read u, f and the coarse correction, write u
  LaunchScope ls(P, K_FUP, w * cells * 3.25, cells * (8.0 + 2.0 * P->nu2 * 11.0 + (norms ? 7.0 : 0.0)), s);
  k_fup<T><<<g, FTHREADS, smem, s>>>(level_view<T>(h), level_view<T>(hc), h.d_ftiles, (int)h.ftiles.size(),
                                     P->d_active, sigma, (const T*)h.d_u2, (T*)h.d_u, (const T*)h.d_f,
                                     (const T*)hc.d_u, P->nu2, norms ? P->d_mode_part : nullptr);
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
