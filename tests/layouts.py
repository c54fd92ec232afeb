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
