// Device helpers shared by the kernels of the library.
#pragma once

#include "snac_impl.h"

namespace snac {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sum in the kernel's own type: FP32 kernels keep their partial norms in FP32 up to the warp
// (GB300 issues FP64 at 1/64 of the FP32 rate) and widen one value per warp.
template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The four x-y neighbours of cell (i, j) of block b: (block, index within that block's plane).
// Inside the block the neighbour is the adjacent cell; across a connected (or periodic) face the
// facing cell of the connected block (faces coincide, Sec. 3.1); on a physical face the cell itself
// (its coupling coefficient is zero there).
__device__ __forceinline__ void nbr_cells(const BlockDev* __restrict__ blk, const BlockDev& B, int b, int i, int j,
                                          int& bw, long long& lw, int& be, long long& le, int& bs, long long& ls,
                                          int& bn, long long& ln) {
  const long long self = (long long)j * B.nx + i;
  bw = be = bs = bn = b;
  lw = le = ls = ln = self;
  if (i > 0) {
    lw = self - 1;
  } else if (B.nbr[0] >= 0) {
    bw = B.nbr[0];
    const BlockDev& N = blk[bw];
    lw = (long long)j * N.nx + (N.nx - 1);
  }
  if (i < B.nx - 1) {
    le = self + 1;
  } else if (B.nbr[1] >= 0) {
    be = B.nbr[1];
    const BlockDev& N = blk[be];
    le = (long long)j * N.nx;
  }
  if (j > 0) {
    ls = self - B.nx;
  } else if (B.nbr[2] >= 0) {
    bs = B.nbr[2];
    const BlockDev& N = blk[bs];
    ls = (long long)(N.ny - 1) * N.nx + i;
  }
  if (j < B.ny - 1) {
    ln = self + B.nx;
  } else if (B.nbr[3] >= 0) {
    bn = B.nbr[3];
    ln = i;
  }
}

// Colour-split position of cell (i, j) of block B in a plane: within each row the cells of colour 0
// ((i + j + par) even) come first in order of i, then those of colour 1 (block widths are even).
// FP64 plans with scaled right-hand sides keep f / diag and 1/diag of their smoothed levels in this
// order, so that a colour kernel reads whole 32-byte sectors of both; the iterate keeps the plain
// order.
__device__ __forceinline__ long long split_cell(const BlockDev& B, int i, int j) {
  return B.off + (long long)j * B.nx + (((i + j + B.par) & 1) ? (B.nx >> 1) : 0) + (i >> 1);
}

// Plane index (within one mode plane of a level) of the four neighbours of (i, j) in block b.
__device__ __forceinline__ void nbr_plane(const BlockDev* __restrict__ blk, const BlockDev& B, int b, int i, int j,
                                          long long& w, long long& e, long long& s, long long& n) {
  int bw, be, bs, bn;
  long long lw, le, ls, ln;
  nbr_cells(blk, B, b, i, j, bw, lw, be, le, bs, ls, bn, ln);
  w = blk[bw].off + lw;
  e = blk[be].off + le;
  s = blk[bs].off + ls;
  n = blk[bn].off + ln;
}

template <typename T>
inline LevelView<T> level_view(const HostLevel& l);

template <>
inline LevelView<double> level_view<double>(const HostLevel& l) {
  return LevelView<double>{l.d_blk, l.d_tiles, l.d_cx64, l.d_cy64, l.d_px64, l.d_py64, l.d_rx64, l.d_ry64,
                           l.ncell, (int)l.tiles.size(), l.nblk, l.d_dxy64, l.d_wr64, l.d_wp64};
}

template <>
inline LevelView<float> level_view<float>(const HostLevel& l) {
  return LevelView<float>{l.d_blk, l.d_tiles, l.d_cx32, l.d_cy32, l.d_px32, l.d_py32, l.d_rx32, l.d_ry32,
                          l.ncell, (int)l.tiles.size(), l.nblk, l.d_dxy32, l.d_wr32, l.d_wp32};
}

// 1/x: the single-precision reciprocal, refined by one Newton step in double.
__device__ __forceinline__ double recip(double x) {
  double r = (double)(1.0f / (float)x);
  return r * fma(-x, r, 2.0);
}
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }

}  // namespace snac
