// Per-tile tables of the fused multigrid kernels: everything that depends on the tile but not on the
// wavenumber, built once per plan on the host and copied whole into shared memory by each CTA.
//
// A fused tile is FTILE_X x FTILE_Y cells of one block; its window adds FUSED_HALO cells on every side
// (FWN x FWN cells). Window cell (wj, wi) is block-local (y0 - FUSED_HALO + wj, x0 - FUSED_HALO + wi)
// of the tile's block; outside that block it belongs to the connected block on that side (region
// row ry / column rx: 0 below, 1 inside, 2 past the block; corners through either neighbour), or to
// no block. Columns are handled in pairs (2k, 2k + 1): the window origin is even and block faces sit
// at even positions, so a pair never straddles a face.
//
// Addressing: the cell of window row wj and column 2k sits at plane offset rowoff[colrx[k]][wj] +
// col[k], where col[k] is the column in the tile's block coordinates and rowoff folds in the shift
// into the region block's own coordinates. The coarse window (parents of the window cells plus one
// ring) is addressed the same way through crowoff / ccol / ccolrx.
#pragma once

#include <climits>

#include "snac_impl.h"

namespace snac {

constexpr int FUSED_HALO = 6;
constexpr int FWN = FTILE_X + 2 * FUSED_HALO;  // window side (64)
constexpr int FHW = FWN / 2;                   // column pairs (32)
constexpr int FCW = FWN / 2 + 2;               // coarse window side (34)
constexpr int FUSED_NONE = INT_MIN;            // row or column with no owner
// the window reaches FUSED_HALO cells into each neighbouring block, and its coarse window (parents
// plus one ring) FUSED_HALO / 2 + 1 coarse cells into the neighbour's coarse block
static_assert(FUSED_MIN_BLOCK >= FUSED_HALO && FUSED_MIN_BLOCK / 2 >= FUSED_HALO / 2 + 1,
              "fused levels need blocks wide enough to hold the halo");

template <typename T>
struct FP2 {
  T a, b;
};

template <typename T>
struct alignas(16) FusedTab {
  FP2<T> xc[3][2][FHW];  // {lo, hi} x-coupling of window column 2k + p in region row ry (0: no owner)
  T xd[3][2][FHW];       // x part of the diagonal
  FP2<T> yc[3][FWN];     // {lo, hi} y-coupling of window row wj in region column rx
  T yd[3][FWN];
  FP2<T> px[3][2][FHW];  // prolongation weights {self, nbr} of window column 2k + p
  FP2<T> py[3][FWN];
  T rx[2][FHW];          // restriction weights (fine width / parent width) of the tile's columns
  T ry[FWN];             // ... and of the rows of the tile's block
  int rowoff[3][FWN];    // plane offset of window row wj in region column rx, FUSED_NONE: no owner
  int crowoff[3][FCW];   // coarse plane offset of coarse window row cj, FUSED_NONE: no owner
  int col[FHW];          // column of window column 2k (tile's block coordinates), FUSED_NONE: clipped
  int colrx[FHW];        // region column of pair k
  int ccol[FCW];         // coarse window column (coarse block coordinates), FUSED_NONE: none
  int ccolrx[FCW];
  int rowry[FWN];        // region row of window row wj
  int cout0;             // coarse plane offset of the parent of window cell (0, 0)
  int cnx;               // width of the tile's coarse block
  int tw, th;            // extent of the tile inside its block
  int pbase;             // colour of window cell (0, 0)
};

}  // namespace snac
