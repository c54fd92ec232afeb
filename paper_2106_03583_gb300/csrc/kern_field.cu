// FP64 kernels on 3-D fields: the outer residual r = f - A p of the defect-correction loop (Eq. 8),
// the operator itself, right-hand-side statistics, deterministic reductions, and the mean fix of
// singular problems.
#include "snac_impl.h"
#include "kern_common.cuh"

namespace snac {
namespace {

constexpr int ZSPLIT = 16;

// Block-wide sum of NV doubles; the result is valid in thread 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh /* [NV][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nwarp ? sh[k * 32 + lane] : 0.0;
      v[k] = warp_sum(x);
    }
  }
}

// One thread per x-y cell of a tile, looping over the z planes k = blockIdx.y, + gridDim.y, ...
// The z ends carry their boundary condition as a mirrored ghost (coefficient +-1/dz^2 on the cell
// itself, cz[k].lo / hi), so the diagonal dxy + zd is the same on every plane and is formed once
// per column. Only the sums a caller needs are formed: the kernel is bound by the FP64 pipe.
// MODE 0: r = (f - fshift) - A p; partial {||r||^2, ||f - fshift||^2 (NEED_F2), sum V p (NEED_VP)}
// MODE 1: r = A p
// Caller-array offset (at k = 0) of plane cell l of block b, and that block's homogeneous stride.
__device__ __forceinline__ long long caller_cell(const CallerBlk* __restrict__ cb, const BlockDev* __restrict__ blk,
                                                int b, long long l, long long& sk) {
  const CallerBlk c = cb[b];
  const int nx = blk[b].nx;
  sk = c.s[2];
  return c.off3 + (l % nx) * c.s[0] + (l / nx) * c.s[1];
}

template <int MODE, bool SHIFT, bool NEED_F2, bool NEED_VP>
__global__ void __launch_bounds__(TILE_THREADS) k_field3d(LevelView<double> L, const CallerBlk* __restrict__ cb,
                                                           const Coef<double>* __restrict__ cz, int nz, int periodic_z,
                                                           double zd, double dz, const double* __restrict__ f,
                                                           const double* __restrict__ p, double* __restrict__ r,
                                                           double fshift, double* __restrict__ partial) {
  __shared__ double sh[4 * 32];
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  double acc[3] = {0.0, 0.0, 0.0};
  if (i < B.nx && j < B.ny) {
    const Coef<double> cx = L.cx[B.xo + i], cy = L.cy[B.yo + j];
    // caller offsets at k = 0 of the cell and its four plane neighbours (self on a physical face,
    // where the weight is 0), and the stride along the homogeneous axis of each one's block
    long long sc, sw, se, ss, sn;
    const long long base = caller_cell(cb, L.blk, t.b, (long long)j * B.nx + i, sc);
    int bw, be, bs, bn;
    long long lw, le, ls, ln;
    nbr_cells(L.blk, B, t.b, i, j, bw, lw, be, le, bs, ls, bn, ln);
    const long long pw = caller_cell(cb, L.blk, bw, lw, sw), pe = caller_cell(cb, L.blk, be, le, se);
    const long long ps = caller_cell(cb, L.blk, bs, ls, ss), pn = caller_cell(cb, L.blk, bn, ln, sn);
    const double dg = cx.d + cy.d + zd;
    const double va = cx.w * cy.w * dz;
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
      const long long c = base + k * sc;
      const Coef<double> z = cz[k];
      const int kd = k > 0 ? k - 1 : (periodic_z ? nz - 1 : k);
      const int ku = k < nz - 1 ? k + 1 : (periodic_z ? 0 : k);
      const double pc = p[c];
      // with the shift and no ||f - fshift||^2 wanted, fshift enters the chain: r = f - (fshift + A p)
      constexpr bool FOLD = MODE == 0 && SHIFT && !NEED_F2;
      double ap = FOLD ? fma(cx.lo, p[pw + k * sw], fshift) : cx.lo * p[pw + k * sw];
      ap = fma(cx.hi, p[pe + k * se], ap);
      ap = fma(cy.lo, p[ps + k * ss], ap);
      ap = fma(cy.hi, p[pn + k * sn], ap);
      ap = fma(z.lo, p[base + kd * sc], ap);
      ap = fma(z.hi, p[base + ku * sc], ap);
      ap = fma(dg, pc, ap);
      if (MODE == 1) {
        r[c] = ap;
      } else {
        const double fv = SHIFT && !FOLD ? f[c] - fshift : f[c];
        const double rv = fv - ap;
        r[c] = rv;
        acc[0] = fma(rv, rv, acc[0]);
        if (NEED_F2) acc[1] = fma(fv, fv, acc[1]);
        if (NEED_VP) acc[2] = fma(va, pc, acc[2]);
      }
    }
  }
  if (MODE == 1) return;
  block_sum<3>(acc, sh);
  if (threadIdx.x == 0) {
    double* o = partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
    o[3] = 0.0;
  }
}

// Before the first residual: statistics of the right-hand side and whether the initial guess is
// zero. partial {sum V f, sum V |f|, ||f||^2, sum f} (the first two and the last only for singular
// problems); *nonzero = 1 if any p has a bit set other than its sign.
template <bool SING>
__global__ void __launch_bounds__(TILE_THREADS) k_prepass(LevelView<double> L, const CallerBlk* __restrict__ cb, int nz,
                                                           double dz, const double* __restrict__ f,
                                                           const double* __restrict__ p, double* __restrict__ partial,
                                                           int* __restrict__ nonzero) {
  __shared__ double sh[4 * 32];
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  unsigned long long bits = 0;
  if (i < B.nx && j < B.ny) {
    const double va = L.cx[B.xo + i].w * L.cy[B.yo + j].w * dz;
    long long sk;
    const long long base = caller_cell(cb, L.blk, t.b, (long long)j * B.nx + i, sk);
    for (int k = blockIdx.y; k < nz; k += gridDim.y) {
      const long long c = base + k * sk;
      const double fv = f[c];
      bits |= (unsigned long long)__double_as_longlong(p[c]);
      if (SING) {
        acc[0] = fma(va, fv, acc[0]);
        acc[1] = fma(va, fabs(fv), acc[1]);
        acc[3] += fv;
      }
      acc[2] = fma(fv, fv, acc[2]);
    }
  }
  block_sum<4>(acc, sh);
  const int any = __syncthreads_or((bits << 1) != 0ull);  // the shift drops the sign bit (-0.0 is zero)
  if (threadIdx.x == 0) {
    double* o = partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
    o[3] = acc[3];
    if (any) atomicOr(nonzero, 1);
  }
}

// Deterministic sum of npart x 4 partials into out[4] (one CTA, fixed order).
// With `flag`, also out_flag = (double)*flag (read after the kernels that set it), and *flag = 0.
__global__ void __launch_bounds__(1024) k_reduce4(const double* __restrict__ part, int npart, double* __restrict__ out,
                                                  int* __restrict__ flag, double* __restrict__ out_flag) {
  __shared__ double sh[4 * 32];
  double acc[4] = {0, 0, 0, 0};
  for (int i = threadIdx.x; i < npart; i += blockDim.x) {
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[k] += part[4 * (long long)i + k];
  }
  block_sum<4>(acc, sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) out[k] = acc[k];
    if (flag) {
      *out_flag = (double)*flag;
      *flag = 0;  // ready for the next pre-pass
    }
  }
}

// Control data between device memory and mapped pinned host memory (one CTA; n is small).
__global__ void __launch_bounds__(256) k_copy_d(const double* __restrict__ src, double* __restrict__ dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__global__ void __launch_bounds__(256) k_copy_i(const int* __restrict__ src, int* __restrict__ dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
__global__ void __launch_bounds__(256) k_fill_d(double* __restrict__ dst, int n, double v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = v;
}

// The singular mode-0 correction is shifted by a constant so that the updated p has zero
// volume-weighted mean: sum V (p_old + e) = 0, with sum V e = alpha * sum_xy area * e0
// (alpha = dz n / theta) and sum V p_old = sums[2] from the residual pass. Two passes over the
// mode-0 plane: per-CTA partial sums of area * e0, then (after their reduction into sums[4]) the shift.
template <typename T>
__global__ void __launch_bounds__(256) k_area_dot(const T* __restrict__ u0, const double* __restrict__ area,
                                                  long long ncell, double* __restrict__ partial) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
    acc[0] = fma(area[c], (double)u0[c], acc[0]);
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) {
    double* o = partial + 4 * (long long)blockIdx.x;
    o[0] = acc[0];
    o[1] = o[2] = o[3] = 0.0;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_fix_apply(T* __restrict__ u0, long long ncell, const double* __restrict__ sums,
                                                   double alpha, double area_total) {
  const double kappa = -(sums[2] + alpha * sums[4]) / (alpha * area_total);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell; c += (long long)gridDim.x * blockDim.x)
    u0[c] = (T)((double)u0[c] + kappa);
}

__global__ void k_shift(double* __restrict__ p, long long n, const double* __restrict__ c) {
  const double s = *c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] -= s;
}

// c = sums[2] / vol_total (the volume-weighted mean of p) written to sums[3]
__global__ void k_mean_of_p(double* sums, double vol_total) { sums[3] = sums[2] / vol_total; }

template <int MODE, bool SH, bool F2, bool VP>
void field3d_t(const LevelView<double>& L, dim3 grid, snac_plan* P, const double* f, const double* p, double* r,
               double fshift, cudaStream_t s) {
  k_field3d<MODE, SH, F2, VP><<<grid, TILE_THREADS, 0, s>>>(L, P->d_cblk, P->d_cz, P->nzt, P->kind == KIND_PP, P->cz[0].d,
                                                             P->dz, f, p, r, fshift, P->d_partial);
}

template <bool SH>
void residual_t(const LevelView<double>& L, dim3 grid, snac_plan* P, const double* f, const double* p, double* r,
                double fshift, bool need_f2, bool need_vp, cudaStream_t s) {
  if (need_f2 && need_vp) field3d_t<0, SH, true, true>(L, grid, P, f, p, r, fshift, s);
  else if (need_f2) field3d_t<0, SH, true, false>(L, grid, P, f, p, r, fshift, s);
  else if (need_vp) field3d_t<0, SH, false, true>(L, grid, P, f, p, r, fshift, s);
  else field3d_t<0, SH, false, false>(L, grid, P, f, p, r, fshift, s);
}

dim3 field_grid(const snac_plan* P) {
  return dim3((unsigned)P->lev[0].tiles.size(), (unsigned)std::min(P->nzt, ZSPLIT));
}

}  // namespace

cudaError_t launch_field3d(snac_plan* P, int mode, const double* f, const double* p, double* r, double fshift,
                           bool need_f2, bool need_vp, cudaStream_t s) {
  LevelView<double> L = level_view<double>(P->lev[0]);
  const dim3 grid = field_grid(P);
  const double n3 = (double)P->n3;
  {
    // algorithmic bytes: read f and p, write r (mode 0); read p, write A p (mode 1)
    const double fl = mode == 0 ? 17.0 + (fshift != 0.0 ? 1.0 : 0.0) + (need_f2 ? 2.0 : 0.0) + (need_vp ? 2.0 : 0.0)
                                : 13.0;
    LaunchScope ls(P, K_FIELD3D, (mode == 0 ? 24.0 : 16.0) * n3, fl * n3, s);
    if (mode == 1) field3d_t<1, false, false, false>(L, grid, P, f, p, r, fshift, s);
    else if (fshift != 0.0) residual_t<true>(L, grid, P, f, p, r, fshift, need_f2, need_vp, s);
    else residual_t<false>(L, grid, P, f, p, r, fshift, need_f2, need_vp, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || mode == 1) return e;
  return launch_reduce_partials(P, (int)(grid.x * grid.y), P->d_sums, s);
}

cudaError_t launch_prepass(snac_plan* P, const double* f, const double* p, cudaStream_t s) {
  LevelView<double> L = level_view<double>(P->lev[0]);
  const dim3 grid = field_grid(P);
  const double n3 = (double)P->n3;
  cudaError_t e;
  {
    // read f and p (the flag is zero: set at plan creation, reset by the reduction that reads it)
    LaunchScope ls(P, K_FIELD3D, 16.0 * n3, (P->singular ? 7.0 : 2.0) * n3, s);
    if (P->singular)
      k_prepass<true><<<grid, TILE_THREADS, 0, s>>>(L, P->d_cblk, P->nzt, P->dz, f, p, P->d_partial, P->d_flag);
    else
      k_prepass<false><<<grid, TILE_THREADS, 0, s>>>(L, P->d_cblk, P->nzt, P->dz, f, p, P->d_partial, P->d_flag);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int npart = (int)(grid.x * grid.y);
  LaunchScope ls(P, K_REDUCE, 32.0 * npart, 4.0 * npart, s);
  k_reduce4<<<1, 1024, 0, s>>>(P->d_partial, npart, P->d_sums, P->d_flag, P->d_sums + SUM_NONZERO);
  return cudaGetLastError();
}

cudaError_t launch_reduce_partials(snac_plan* P, int npart, double* out, cudaStream_t s) {
  LaunchScope ls(P, K_REDUCE, 32.0 * npart, 4.0 * npart, s);
  k_reduce4<<<1, 1024, 0, s>>>(P->d_partial, npart, out, nullptr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_to_host(const double* d_src, double* dh_dst, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_copy_d<<<1, 256, 0, s>>>(d_src, dh_dst, n);
  return cudaGetLastError();
}

cudaError_t launch_from_host(const int* dh_src, int* d_dst, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_copy_i<<<1, 256, 0, s>>>(dh_src, d_dst, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* d, int n, double v, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_fill_d<<<1, 256, 0, s>>>(d, n, v);
  return cudaGetLastError();
}

cudaError_t launch_fix_mean(snac_plan* P, void* u0, cudaStream_t s) {
  const double alpha = P->dz * P->nzt / P->theta;
  const long long n = P->lev[0].ncell;
  const int w = plan_inner_size(P);
  const int ctas = std::min(MEAN_CTAS, P->npartial);  // one partial per CTA, d_partial holds npartial
  {
    LaunchScope ls(P, K_FIX_MEAN, (double)n * (8.0 + w), 2.0 * n, s);
    if (w == 8) k_area_dot<double><<<ctas, 256, 0, s>>>((const double*)u0, P->d_area0, n, P->d_partial);
    else k_area_dot<float><<<ctas, 256, 0, s>>>((const float*)u0, P->d_area0, n, P->d_partial);
  }
  cudaError_t e = launch_reduce_partials(P, ctas, P->d_sums + 4, s);
  if (e != cudaSuccess) return e;
  LaunchScope ls(P, K_FIX_MEAN, 2.0 * n * w, (double)n, s);
  if (w == 8) k_fix_apply<double><<<MEAN_CTAS, 256, 0, s>>>((double*)u0, n, P->d_sums, alpha, P->area_total);
  else k_fix_apply<float><<<MEAN_CTAS, 256, 0, s>>>((float*)u0, n, P->d_sums, alpha, P->area_total);
  return cudaGetLastError();
}

cudaError_t launch_shift(snac_plan* P, double* p, const double* d_c, cudaStream_t s) {
  {
    LaunchScope ls(P, K_SHIFT, 16.0, 1.0, s);
    k_mean_of_p<<<1, 1, 0, s>>>(P->d_sums, P->vol_total);
  }
  LaunchScope ls(P, K_SHIFT, 16.0 * P->n3, (double)P->n3, s);
  k_shift<<<2 * P->sms, 512, 0, s>>>(p, P->n3, d_c);
  return cudaGetLastError();
}

}  // namespace snac
