// The outer residual r = f - A p of mixed-precision plans in float-float arithmetic (Eq. 8).
//
// On GB300 the FP64 pipe issues 2 FMA lanes per clock per multiprocessor against 128 for FP32, so
// the FP64 residual pass of the defect-correction loop is bound by the FP64 pipe (seven FMAs per
// cell), not by HBM. A mixed plan rounds r to FP32 anyway before its FP32 transform, so r is needed
// in FP32 only -- but computed from f and p without cancellation error: A p nearly cancels f, and
// the terms |c p| are thousands of times larger than r. Here every FP64 operand is split into two
// floats (hi + lo, 47 significant bits) by integer operations on its bit pattern, the coefficients
// into rounded float pairs, and the products and the sum are carried in float-float
// (hi, lo) arithmetic: an exact product of the leading parts (FMA), the cross terms, and an exact
// two-sum of the leading parts. The error of r is below a few units of 2^-47 times
// |f| + sum |c p| per cell; the result is rounded to FP32. No FP64 instruction runs per cell.
//
// The solve uses this pass for the defect-correction steps whose residual is far above the
// tolerance, and the FP64 pass of kern_field.cu for the check that decides convergence.
#include <cmath>

#include "kern_common.cuh"
#include "snac_impl.h"

namespace snac {
namespace {

struct FF {
  float hi, lo;
};

// x = hi + lo + d with |d| < 2^-46 |x|: hi is x truncated to 24 significant bits, lo the next 23
// bits (truncated), both formed from the bit pattern with integer operations. lo is built as the
// difference of two floats that share the exponent of its leading bit position (the second with an
// empty mantissa), which is exact. Values below 2^-103 in magnitude, and zero, give hi = lo = 0;
// values beyond the FP32 range, Inf and NaN give a non-finite hi.
__device__ __forceinline__ FF split64(double x) {
  const unsigned hw = (unsigned)__double2hiint(x);
  unsigned lw = (unsigned)__double2loint(x);
  int t = (int)(hw & 0x7fffffffu) - (920 << 20);  // FP32 exponent - 24 at bits 27..20, mantissa below
  const bool tiny = t < 0;
  t = min(t, 231 << 20) + (24 << 20);             // FP32 exponent at bits 27..20 (255: overflow)
  const unsigned hb = tiny ? 0u : (unsigned)t;
  lw = tiny ? 0u : lw;
  const unsigned hib = __funnelshift_l(lw, hb, 3) | (hw & 0x80000000u);
  const unsigned f0 = (hib & 0xff800000u) - (23u << 23);
  const unsigned f1 = f0 | ((lw >> 6) & 0x007fffffu);
  return {__uint_as_float(hib), __fsub_rn(__uint_as_float(f1), __uint_as_float(f0))};
}

// (sh, sl) -= c x. The leading product c.hi x.hi is split exactly by an FMA; the cross terms go into
// the low part; the leading parts are subtracted by an exact two-sum whose error joins the low part.
// Every operation is an explicitly rounded intrinsic, so the compiler cannot contract or reorder it.
__device__ __forceinline__ void sub_prod(float& sh, float& sl, FF c, FF x) {
  const float h = __fmul_rn(c.hi, x.hi);
  const float e = __fmaf_rn(c.hi, x.hi, -h);
  const float l = __fmaf_rn(c.hi, x.lo, __fmaf_rn(c.lo, x.hi, e));
  const float s = __fsub_rn(sh, h);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(-h, bb));
  sh = s;
  sl = __fsub_rn(__fadd_rn(sl, err), l);
}

// (sh, sl) += (x.hi, x.lo)
__device__ __forceinline__ void add_ff(float& sh, float& sl, FF x) {
  const float s = __fadd_rn(sh, x.hi);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(x.hi, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, x.lo));
}

template <int NV>
__device__ __forceinline__ void block_sum_d(double (&v)[NV], double* sh /* [NV][32] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = warp_sum(v[k]);
    if (lane == 0) sh[k * 32 + warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = warp_sum(lane < nwarp ? sh[k * 32 + lane] : 0.0);
  }
}

// Caller-array offset (at k = 0) of plane cell l of block b, and that block's homogeneous stride.
__device__ __forceinline__ long long caller_cell_ff(const CallerBlk* __restrict__ cb, const BlockDev* __restrict__ blk,
                                                   int b, long long l, long long& sk) {
  const CallerBlk c = cb[b];
  const int nx = blk[b].nx;
  sk = c.s[2];
  return c.off3 + (l % nx) * c.s[0] + (l / nx) * c.s[1];
}

// One thread per x-y cell of a 32 x 8 tile, marching through kchunk consecutive z planes, so that
// the split of p at a cell serves as the centre and as both z neighbours (loads one plane ahead). The coefficients come as
// rounded float pairs from tables built with the plan (no FP64 instruction per cell or per thread,
// apart from the thread's final sums). Interior z planes couple both z neighbours with the same
// coefficient, so their sum is formed first (one product instead of two). r (FP32) is written at the
// caller-layout position of the cell. Partials per CTA: {||r||^2, ||f - fshift||^2 (NEED_F2),
// sum V p (NEED_VP), 0}; the squares are taken of values scaled by nscale (a power of two chosen from
// ||f||, so that FP32 neither underflows nor overflows) and unscaled in FP64 per thread.
template <bool SHIFT, bool NEED_F2, bool NEED_VP>
__global__ void __launch_bounds__(TILE_THREADS, 3)
    k_field3d_ff(LevelView<double> L, const CallerBlk* __restrict__ cb, const float4* __restrict__ cxff,
                 const float4* __restrict__ cyff, const float2* __restrict__ dgff, const float4* __restrict__ czff,
                 int nz, int periodic_z, int kchunk, double dz, const double* __restrict__ f,
                 const double* __restrict__ p, float* __restrict__ r, float2 fsh, float nscale, double inv_nscale2,
                 double* __restrict__ partial) {
  __shared__ double sh[4 * 32];
  const TileDev t = L.tiles[blockIdx.x];
  const BlockDev B = L.blk[t.b];
  const int i = t.x0 + (threadIdx.x % TILE_X), j = t.y0 + (threadIdx.x / TILE_X);
  double acc[3] = {0.0, 0.0, 0.0};
  const int k0 = blockIdx.y * kchunk, k1 = min(nz, k0 + kchunk);
  if (i < B.nx && j < B.ny && k0 < k1) {
    long long sc_, sw_, se_, ss_, sn_;
    const long long base = caller_cell_ff(cb, L.blk, t.b, (long long)j * B.nx + i, sc_);
    int bw, be, bs, bn;
    long long lw, le, ls, ln;
    nbr_cells(L.blk, B, t.b, i, j, bw, lw, be, le, bs, ls, bn, ln);
    const double* __restrict__ qw = p + caller_cell_ff(cb, L.blk, bw, lw, sw_);
    const double* __restrict__ qe = p + caller_cell_ff(cb, L.blk, be, le, se_);
    const double* __restrict__ qs = p + caller_cell_ff(cb, L.blk, bs, ls, ss_);
    const double* __restrict__ qn = p + caller_cell_ff(cb, L.blk, bn, ln, sn_);
    // z strides of the blocks (a block's plane has fewer than 2^31 cells: checked at plan creation)
    const int sc = (int)sc_, sw = (int)sw_, se = (int)se_, ss = (int)ss_, sn = (int)sn_;
    const float4 cx = cxff[B.xo + i], cy = cyff[B.yo + j];
    const float2 d2 = dgff[B.off + (long long)j * B.nx + i];
    const FF cxl{cx.x, cx.y}, cxh{cx.z, cx.w}, cyl{cy.x, cy.y}, cyh{cy.z, cy.w}, dg{d2.x, d2.y};
    float sr = 0.0f, sf = 0.0f, vh = 0.0f, vl = 0.0f;
    const double* __restrict__ qc = p + base;
    const double* __restrict__ qf = f + base;
    float* __restrict__ qr = r + base;
    FF pc = split64(qc[(long long)k0 * sc]);
    const int kd0 = k0 > 0 ? k0 - 1 : (periodic_z ? nz - 1 : k0);
    FF pd = kd0 == k0 ? pc : split64(qc[(long long)kd0 * sc]);
    // The raw loads of a plane (f, the four x-y neighbours, and p one plane up -- the centre itself
    // at a non-periodic top end) are issued one plane ahead, so that their DRAM latency overlaps the
    // previous plane's arithmetic.
    double xu, xf, xw, xe, xs, xn;
    auto load = [&](int k) {
      const int ku = k < nz - 1 ? k + 1 : (periodic_z ? 0 : k);
      xu = qc[(long long)ku * sc];
      xf = qf[(long long)k * sc];
      xw = qw[(long long)k * sw];
      xe = qe[(long long)k * se];
      xs = qs[(long long)k * ss];
      xn = qn[(long long)k * sn];
    };
    load(k0);
    for (int k = k0; k < k1; ++k) {
      const double cu = xu, cf = xf, cw = xw, ce = xe, cs = xs, cn = xn;
      if (k + 1 < k1) load(k + 1);
      const FF pu = split64(cu);
      const FF fv = split64(cf);
      float s_h = fv.hi, s_l = fv.lo;
      if (SHIFT) sub_prod(s_h, s_l, FF{1.0f, 0.0f}, FF{fsh.x, fsh.y});
      if (NEED_F2) {
        const float fr = __fmul_rn(__fadd_rn(s_h, s_l), nscale);
        sf = __fmaf_rn(fr, fr, sf);
      }
      const float4 z = czff[k];
      sub_prod(s_h, s_l, cxl, split64(cw));
      sub_prod(s_h, s_l, cxh, split64(ce));
      sub_prod(s_h, s_l, cyl, split64(cs));
      sub_prod(s_h, s_l, cyh, split64(cn));
      if (z.x == z.z && z.y == z.w) {  // equal couplings (every plane but the ends of a non-periodic axis)
        float zh = pd.hi, zl = pd.lo;
        add_ff(zh, zl, pu);
        sub_prod(s_h, s_l, FF{z.x, z.y}, FF{zh, zl});
      } else {
        sub_prod(s_h, s_l, FF{z.x, z.y}, pd);
        sub_prod(s_h, s_l, FF{z.z, z.w}, pu);
      }
      sub_prod(s_h, s_l, dg, pc);
      const float rv = __fadd_rn(s_h, s_l);
      qr[(long long)k * sc] = rv;
      const float rs = __fmul_rn(rv, nscale);
      sr = __fmaf_rn(rs, rs, sr);
      if (NEED_VP) add_ff(vh, vl, pc);
      pd = pc;
      pc = pu;
    }
    acc[0] = (double)sr * inv_nscale2;
    acc[1] = (double)sf * inv_nscale2;
    // sum over the thread's planes of V p = (cell volume) x (sum of p over the planes)
    if (NEED_VP) acc[2] = L.cx[B.xo + i].w * L.cy[B.yo + j].w * dz * ((double)vh + (double)vl);
  }
  block_sum_d<3>(acc, sh);
  if (threadIdx.x == 0) {
    double* o = partial + 4 * ((long long)blockIdx.y * gridDim.x + blockIdx.x);
    o[0] = acc[0];
    o[1] = acc[1];
    o[2] = acc[2];
    o[3] = 0.0;
  }
}

template <bool SH, bool F2, bool VP>
void ff_t(const LevelView<double>& L, dim3 grid, int kchunk, snac_plan* P, const double* f, const double* p, float* r,
          float2 fsh, float nscale, double inv_nscale2, cudaStream_t s) {
  k_field3d_ff<SH, F2, VP><<<grid, TILE_THREADS, 0, s>>>(L, P->d_cblk, P->d_cxff, P->d_cyff, P->d_dgff, P->d_czff,
                                                          P->nzt, P->kind == KIND_PP, kchunk, P->dz, f, p, r, fsh,
                                                          nscale, inv_nscale2, P->d_partial);
}

template <bool SH>
void ff_sel(const LevelView<double>& L, dim3 grid, int kchunk, snac_plan* P, const double* f, const double* p, float* r,
            float2 fsh, bool need_f2, bool need_vp, float nscale, double inv_nscale2, cudaStream_t s) {
  if (need_f2 && need_vp) ff_t<SH, true, true>(L, grid, kchunk, P, f, p, r, fsh, nscale, inv_nscale2, s);
  else if (need_f2) ff_t<SH, true, false>(L, grid, kchunk, P, f, p, r, fsh, nscale, inv_nscale2, s);
  else if (need_vp) ff_t<SH, false, true>(L, grid, kchunk, P, f, p, r, fsh, nscale, inv_nscale2, s);
  else ff_t<SH, false, false>(L, grid, kchunk, P, f, p, r, fsh, nscale, inv_nscale2, s);
}

}  // namespace

cudaError_t launch_field3d_ff(snac_plan* P, const double* f, const double* p, float* r, double fshift, double fscale,
                              bool need_f2, bool need_vp, cudaStream_t s) {
  if (!P->d_czff || !P->d_cxff) return cudaErrorInvalidValue;
  LevelView<double> L = level_view<double>(P->lev[0]);
  const int zsplit = std::min(P->nzt, 16);
  const int kchunk = (P->nzt + zsplit - 1) / zsplit;
  const dim3 grid((unsigned)P->lev[0].tiles.size(), (unsigned)((P->nzt + kchunk - 1) / kchunk));
  // squares of r / fscale: fscale is ||f|| / sqrt(n) rounded to a power of two
  int ex = 0;
  std::frexp(fscale > 0.0 && std::isfinite(fscale) ? fscale : 1.0, &ex);
  const float nscale = std::ldexp(1.0f, -ex);
  const double inv2 = std::ldexp(1.0, 2 * ex);
  const double n3 = (double)P->n3;
  {
    // algorithmic bytes: read f and p (FP64), write r (FP32); the method's 17 flops per cell
    LaunchScope ls(P, K_FIELD3D_FF, 20.0 * n3, 17.0 * n3, s);
    const float fh = (float)fshift;
    const float2 fsh = make_float2(fh, (float)(fshift - (double)fh));
    if (fshift != 0.0) ff_sel<true>(L, grid, kchunk, P, f, p, r, fsh, need_f2, need_vp, nscale, inv2, s);
    else ff_sel<false>(L, grid, kchunk, P, f, p, r, fsh, need_f2, need_vp, nscale, inv2, s);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(P, (int)(grid.x * grid.y), P->d_sums, s);
}

}  // namespace snac
