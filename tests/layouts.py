"""Small block layouts used by the tests (built with the shared input generator)."""
import numpy as np

from paper_2106_03583_gb300 import inputs

Z_PAIRS = {"PP": ("P", "P"), "NN": ("N", "N"), "DD": ("D", "D"), "ND": ("N", "D"), "DN": ("D", "N")}


def rects(layout, n):
    """Block rectangles (x0, x1, y0, y1) of an n x n-cell block unit."""
    if layout == "1":
        return [(0, 2 * n, 0, 2 * n)]
    if layout == "1x2":
        return [(0, n, 0, 2 * n), (n, 2 * n, 0, 2 * n)]
    if layout == "2x1":
        return [(0, 2 * n, 0, n), (0, 2 * n, n, 2 * n)]
    if layout == "L":
        return [(0, n, 0, n), (n, 2 * n, 0, n), (0, n, n, 2 * n)]
    if layout == "2x2":
        return [(0, n, 0, n), (n, 2 * n, 0, n), (0, n, n, 2 * n), (n, 2 * n, n, 2 * n)]
    raise ValueError(layout)


def make(layout="1", n=4, nz=4, zpair="PP", walls=("D", "D", "N", "N"), stretched=False,
         periodic=(False, False), lz=1.0, lx=1.0, ly=1.0, aniso=1.0):
    """Blocks of a layout whose bounding box is 2n x 2n cells by nz."""
    xf = inputs.tanh_faces(2 * n, 0, 1.3 if stretched else 0.0, 0.0, lx)
    yf = inputs.tanh_faces(2 * n, -1 if stretched else 0, 1.1 if stretched else 0.0, 0.0, ly * aniso)
    zf = np.linspace(0.0, lz, nz + 1)
    wb = {"x-": walls[0], "x+": walls[1], "y-": walls[2], "y+": walls[3]}
    return inputs.make_blocks(xf, yf, zf, rects(layout, n), wb, Z_PAIRS[zpair], periodic=periodic,
                              inner_wall="N")


def homogeneous_along(blocks, f, homog):
    """The same problem with its homogeneous direction (z) relabelled as caller axis `homog` (0 = x,
    1 = y): the two plane axes keep their order on the remaining caller axes. Returns the new blocks,
    the right-hand side in the new [z][y][x] layout, and a function mapping a field in the new layout
    back to the original one."""
    if homog == 2:
        return blocks, f, lambda v: v
    # new caller axis c takes original axis src[c]
    src = (2, 0, 1) if homog == 0 else (0, 2, 1)
    out, pieces, shapes = [], [], []
    o = 0
    for b in blocks:
        n = [int(b["hi"][a] - b["lo"][a] + 1) for a in range(3)]
        out.append({"lo": tuple(b["lo"][src[c]] for c in range(3)), "hi": tuple(b["hi"][src[c]] for c in range(3)),
                    "dx": tuple(b["dx"][src[c]] for c in range(3)), "bc": tuple(b["bc"][src[c]] for c in range(3)),
                    "nbr": tuple(b["nbr"][src[c]] for c in range(3))})
        a3 = np.asarray(f[o:o + n[0] * n[1] * n[2]]).reshape(n[2], n[1], n[0])   # original [z][y][x]
        o += n[0] * n[1] * n[2]
        # new layout [Z][Y][X] = original axes (src[2], src[1], src[0]); array axes are (z, y, x) = (2, 1, 0)
        perm = tuple(2 - src[c] for c in (2, 1, 0))
        pieces.append(np.transpose(a3, perm).ravel())
        shapes.append((perm, tuple(a3.shape[p] for p in perm)))

    def back(v):
        res, o2 = [], 0
        for perm, shp in shapes:
            m = int(np.prod(shp))
            a = np.asarray(v[o2:o2 + m]).reshape(shp)
            o2 += m
            res.append(np.transpose(a, np.argsort(perm)).ravel())
        return np.concatenate(res)

    return out, np.concatenate(pieces), back
