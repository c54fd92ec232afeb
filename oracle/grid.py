"""Multi-block staggered grid and the second-order finite-volume Poisson operator (Eq. 8, Sec. 2-3.1).

Test infrastructure only (see the package docstring).

Readings of the paper used here (the paper prints only the uniform form of Eq. 8 "for simplicity"
and says the implementation is the general non-uniform one, footnote of Sec. 3.3):

* Pressure lives at cell centres. Along a non-homogeneous axis the operator of one row is the
  staggered divergence of the staggered gradient, per unit volume:
      (A p)_i = [ (p_{i+1} - p_i) / h_{i+1/2} - (p_i - p_{i-1}) / h_{i-1/2} ] / w_i
  with w_i the cell width and h the distance between the two cell centres across a face,
  h = (w_i + w_nbr) / 2.
* A physical face mirrors the cell across the face (ghost at distance w_i): homogeneous Dirichlet
  ghost = -p_i, homogeneous Neumann ghost = +p_i (Sec. 3.1 "Dirichlet, Neumann"; the Neumann
  pressure condition is what a prescribed velocity needs).
* A block-block face ("B") or periodic face ("P") takes the neighbouring cell of the connected
  block (Sec. 3.1-3.2: connectivity, periodic = cyclic connectivity). Faces must coincide.
* The homogeneous axis z is uniform with spacing dz and one boundary pair shared by all blocks.

Cells of one z-plane are numbered block by block, [block][y][x] with x fastest; a 3-D field is held
as an (n_z, n_xy) array ("plane-major"), and converted from/to the caller's
[block][z][y][x] layout by ``to_planes``/``from_planes``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import transforms


class LayoutError(ValueError):
    pass


def _n(blk, a):
    return int(blk["hi"][a] - blk["lo"][a] + 1)


def validate(blocks):
    """Check the block graph: sizes, widths, face connectivity and congruence (Sec. 3.1)."""
    if len(blocks) == 0:
        raise LayoutError("no blocks")
    nz = _n(blocks[0], 2)
    wz0 = np.asarray(blocks[0]["dx"][2], dtype=np.float64)
    zbc0 = tuple(blocks[0]["bc"][2])
    for b, blk in enumerate(blocks):
        for a in range(3):
            if _n(blk, a) < 1 or len(blk["dx"][a]) != _n(blk, a):
                raise LayoutError(f"block {b}: widths along axis {a} do not match lo/hi")
            if np.any(np.asarray(blk["dx"][a]) <= 0):
                raise LayoutError(f"block {b}: non-positive cell width")
        if _n(blk, 2) != nz or tuple(blk["bc"][2]) != zbc0:
            raise LayoutError("all blocks must share n_z and the z boundary pair")
        if not np.allclose(blk["dx"][2], wz0, rtol=0, atol=0):
            raise LayoutError("all blocks must share the z grid")
        for a in range(2):
            o = 1 - a
            for s in range(2):
                kind = blk["bc"][a][s]
                if kind not in ("D", "N", "P", "B"):
                    raise LayoutError(f"block {b}: unknown bc {kind!r}")
                if kind == "P" and blk["bc"][a][1 - s] != "P":
                    raise LayoutError(f"block {b}: periodic needs both faces of the axis")
                if kind == "B":
                    c = int(blk["nbr"][a][s])
                    if not (0 <= c < len(blocks)):
                        raise LayoutError(f"block {b}: bad neighbour id")
                    nb = blocks[c]
                    if nb["bc"][a][1 - s] != "B" or int(nb["nbr"][a][1 - s]) != b:
                        raise LayoutError(f"block {b}: connectivity with block {c} is not symmetric")
                    if nb["lo"][o] != blk["lo"][o] or nb["hi"][o] != blk["hi"][o]:
                        raise LayoutError(f"block {b}: face shared with block {c} does not coincide")
                    if not np.array_equal(np.asarray(nb["dx"][o]), np.asarray(blk["dx"][o])):
                        raise LayoutError(f"block {b}: grid not congruent with block {c}")
    zk = zbc0
    if ("P" in zk) and zk != ("P", "P"):
        raise LayoutError("periodic z needs both faces periodic")
    if any(k == "B" for k in zk):
        raise LayoutError("the homogeneous axis cannot be split into blocks")
    if not np.allclose(wz0, wz0[0], rtol=1e-12, atol=0):
        raise LayoutError("the homogeneous axis must be uniform (Sec. 2)")


class Plane:
    """One level of the multi-block x-y grid: cell widths, neighbours and the 2-D operator."""

    def __init__(self, blocks):
        self.blocks = blocks
        self.nb = len(blocks)
        self.nx = [_n(b, 0) for b in blocks]
        self.ny = [_n(b, 1) for b in blocks]
        self.off = np.cumsum([0] + [nx * ny for nx, ny in zip(self.nx, self.ny)])
        self.n = int(self.off[-1])
        lox = min(b["lo"][0] for b in blocks)
        loy = min(b["lo"][1] for b in blocks)
        self.wx = np.concatenate([np.tile(np.asarray(b["dx"][0], float), ny) for b, ny in zip(blocks, self.ny)])
        self.wy = np.concatenate([np.repeat(np.asarray(b["dx"][1], float), nx) for b, nx in zip(blocks, self.nx)])
        self.area = self.wx * self.wy
        # global index-space position of every cell, for the red-black colouring
        gx, gy = [], []
        for b, blk in enumerate(blocks):
            yy, xx = np.meshgrid(np.arange(self.ny[b]), np.arange(self.nx[b]), indexing="ij")
            gx.append((blk["lo"][0] - lox + xx).ravel())
            gy.append((blk["lo"][1] - loy + yy).ravel())
        self.gx, self.gy = np.concatenate(gx), np.concatenate(gy)
        self.red = ((self.gx + self.gy) % 2) == 0
        self.has_dirichlet = any(k == "D" for blk in blocks for a in range(2) for k in blk["bc"][a])
        self._build_neighbours()
        self._build_operator()

    def index_array(self, b):
        """Cell numbers of block b as an (n_y, n_x) array."""
        return self.off[b] + np.arange(self.ny[b])[:, None] * self.nx[b] + np.arange(self.nx[b])[None, :]

    def _build_neighbours(self):
        """nbr[axis][side][cell] = the neighbouring cell across that face, or -1 (Dirichlet face)
        / -2 (Neumann face). Inside a block the neighbour is the adjacent cell; on a "P" face it is
        the block's own cell on the opposite face; on a "B" face the first cell row/column of the
        connected block on its facing side."""
        self.nbr = np.zeros((2, 2, self.n), dtype=np.int64)
        for b in range(self.nb):
            idx = self.index_array(b)
            blk = self.blocks[b]
            for axis in range(2):
                for side in range(2):
                    out = np.empty_like(idx)
                    kind = blk["bc"][axis][side]
                    tgt = b if kind == "P" else int(blk["nbr"][axis][side])
                    if axis == 0:
                        if side == 1:
                            out[:, :-1] = idx[:, 1:]
                            edge = (slice(None), -1)
                        else:
                            out[:, 1:] = idx[:, :-1]
                            edge = (slice(None), 0)
                    else:
                        if side == 1:
                            out[:-1, :] = idx[1:, :]
                            edge = (-1, slice(None))
                        else:
                            out[1:, :] = idx[:-1, :]
                            edge = (0, slice(None))
                    if kind == "D":
                        out[edge] = -1
                    elif kind == "N":
                        out[edge] = -2
                    else:
                        t_idx = self.index_array(tgt)
                        far = 0 if side == 1 else -1     # the connected block's facing row/column
                        out[edge] = t_idx[:, far] if axis == 0 else t_idx[far, :]
                    self.nbr[axis, side, idx.ravel()] = out.ravel()

    def _build_operator(self):
        rows, cols, vals = [], [], []
        diag = np.zeros(self.n)
        w = (self.wx, self.wy)
        for axis in range(2):
            for side in range(2):
                nb = self.nbr[axis, side]
                g = np.arange(self.n)
                inner = nb >= 0
                wc = w[axis][g[inner]]
                wn = w[axis][nb[inner]]
                a = 1.0 / (0.5 * (wc + wn) * wc)          # 1 / (h w)
                rows.append(g[inner]); cols.append(nb[inner]); vals.append(a)
                np.subtract.at(diag, g[inner], a)
                dirich = nb == -1
                wd = w[axis][g[dirich]]
                np.subtract.at(diag, g[dirich], 2.0 / (wd * wd))   # ghost -p at distance w
        self.offdiag = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                     shape=(self.n, self.n))
        self.diag = diag
        self.A = (self.offdiag + sp.diags(diag)).tocsr()

    def coarsen(self):
        """The next-coarser plane: every block halved along x and y, widths summed pairwise."""
        cb = []
        lox = min(b["lo"][0] for b in self.blocks)
        loy = min(b["lo"][1] for b in self.blocks)
        for blk in self.blocks:
            rx, ry = blk["lo"][0] - lox, blk["lo"][1] - loy
            wx, wy = np.asarray(blk["dx"][0]), np.asarray(blk["dx"][1])
            cb.append({"lo": (rx // 2, ry // 2, 0),
                       "hi": (rx // 2 + len(wx) // 2 - 1, ry // 2 + len(wy) // 2 - 1, blk["hi"][2]),
                       "dx": (wx[0::2] + wx[1::2], wy[0::2] + wy[1::2], blk["dx"][2]),
                       "bc": blk["bc"], "nbr": blk["nbr"]})
        return Plane(cb)

    def can_coarsen(self):
        lox = min(b["lo"][0] for b in self.blocks)
        loy = min(b["lo"][1] for b in self.blocks)
        for b, blk in enumerate(self.blocks):
            if self.nx[b] % 2 or self.ny[b] % 2 or self.nx[b] < 4 or self.ny[b] < 4:
                return False
            if (blk["lo"][0] - lox) % 2 or (blk["lo"][1] - loy) % 2:
                return False
        return True


def dzz_matrix(kind: str, n: int, dz: float) -> np.ndarray:
    """The 1-D operator along the uniform homogeneous axis, (p_{k-1} - 2 p_k + p_{k+1}) / dz^2
    (Eq. 8), with periodic wrap (PP) or the staggered ghosts of the end faces (N: +p, D: -p)."""
    D = np.zeros((n, n))
    for k in range(n):
        D[k, k] = -2.0
        if k > 0:
            D[k, k - 1] = 1.0
        if k < n - 1:
            D[k, k + 1] = 1.0
    if kind == "PP":
        D[0, n - 1] += 1.0
        D[n - 1, 0] += 1.0
    else:
        D[0, 0] += 1.0 if kind[0] == "N" else -1.0
        D[n - 1, n - 1] += 1.0 if kind[1] == "N" else -1.0
    return D / (dz * dz)


class Grid:
    """The whole 3-D multi-block problem: x-y plane, z pair, uniform dz.

    ``shift`` (<= 0) gives the Helmholtz form (A + shift I) p = f that the method solves unchanged
    (Sec. 3.3, footnote: the solver applies to the more general Helmholtz equation): every reduced
    equation (Eq. 9) takes the same extra diagonal term, and a nonzero shift removes the null space."""

    def __init__(self, blocks, shift: float = 0.0):
        if not shift <= 0.0:
            raise ValueError("the Helmholtz shift must be <= 0 (A + shift I stays negative definite)")
        self.shift = float(shift)
        validate(blocks)
        self.blocks = blocks
        self.plane = Plane(blocks)
        self.nz = _n(blocks[0], 2)
        self.dz = float(np.asarray(blocks[0]["dx"][2])[0])
        zb = blocks[0]["bc"][2]
        self.kind = transforms.kind_from_bc(zb[0], zb[1])
        if self.kind == "PP" and self.nz % 2:
            raise LayoutError("periodic homogeneous axis needs an even n_z (Table 1)")
        self.Dzz = dzz_matrix(self.kind, self.nz, self.dz)
        # the singular problem: a zero eigenvalue along z and no Dirichlet face in x-y
        self.singular = (self.kind in ("PP", "NN")) and not self.plane.has_dirichlet and self.shift == 0.0
        self.vol = np.outer(np.full(self.nz, self.dz), self.plane.area)     # (n_z, n_xy)

    # ---- layout conversion: caller [block][z][y][x] <-> planes (n_z, n_xy)
    def to_planes(self, v):
        v = np.asarray(v, dtype=np.float64)
        P = np.empty((self.nz, self.plane.n))
        o3 = 0
        pl = self.plane
        for b in range(pl.nb):
            m = pl.nx[b] * pl.ny[b]
            P[:, pl.off[b]:pl.off[b] + m] = v[o3:o3 + self.nz * m].reshape(self.nz, m)
            o3 += self.nz * m
        return P

    def from_planes(self, P):
        pl = self.plane
        out = []
        for b in range(pl.nb):
            m = pl.nx[b] * pl.ny[b]
            out.append(P[:, pl.off[b]:pl.off[b] + m].ravel())
        return np.concatenate(out)

    # ---- the 3-D operator of Eq. 8
    def apply(self, P):
        """A p on planes: the x-y operator on every plane plus the z operator on every column (plus
        shift p)."""
        out = (self.plane.A @ P.T).T + self.Dzz @ P
        if self.shift != 0.0:
            out = out + self.shift * P
        return out

    def matrix(self):
        """The assembled sparse 3-D matrix, plane-major ordering (k * n_xy + cell)."""
        n = self.nz * self.plane.n
        return (sp.kron(sp.identity(self.nz), self.plane.A) + sp.kron(sp.csr_matrix(self.Dzz),
                                                                        sp.identity(self.plane.n))
                + self.shift * sp.identity(n)).tocsr()

    def residual(self, f, p):
        """r = f - A p in the caller's layout."""
        return self.from_planes(self.to_planes(f) - self.apply(self.to_planes(p)))
