"""Pins of the oracle's 3-D operator (Eq. 8 on stretched multi-block grids)."""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import solve as osv
from paper_2106_03583_gb300 import inputs

from layouts import make

LAYOUTS = ["1", "1x2", "2x1", "L", "2x2"]


def staggered_div_grad(blocks, p):
    """D(G p) built from face gradients, the way the projection step (Eqs. 4-5) uses the operators.

    G p on a face between two cells = (p_upper - p_lower) / (centre distance); on a Neumann face 0;
    on a Dirichlet face p = 0 on the face, half a cell from the centre. D = (G_upper - G_lower) / w."""
    g = ogrid.Grid(blocks)
    pl = g.plane
    P = g.to_planes(p)
    out = np.zeros_like(P)
    w = (pl.wx, pl.wy)
    for axis in range(2):
        for side in range(2):
            nb = pl.nbr[axis, side]
            for c in range(pl.n):
                wc = w[axis][c]
                if nb[c] >= 0:
                    h = 0.5 * (wc + w[axis][nb[c]])
                    grad = (P[:, nb[c]] - P[:, c]) / h if side == 1 else (P[:, c] - P[:, nb[c]]) / h
                elif nb[c] == -1:
                    grad = (0.0 - P[:, c]) / (0.5 * wc) if side == 1 else (P[:, c] - 0.0) / (0.5 * wc)
                else:
                    grad = 0.0
                out[:, c] += (grad if side == 1 else -grad) / wc
    dz, nz, kind = g.dz, g.nz, g.kind
    for k in range(nz):
        for side in range(2):
            kk = k + 1 if side == 1 else k - 1
            if 0 <= kk < nz or kind == "PP":
                kk %= nz
                grad = (P[kk] - P[k]) / dz if side == 1 else (P[k] - P[kk]) / dz
            elif kind[side] == "D":
                grad = (0.0 - P[k]) / (0.5 * dz) if side == 1 else (P[k] - 0.0) / (0.5 * dz)
            else:
                grad = 0.0
            out[k] += (grad if side == 1 else -grad) / dz
    return g.from_planes(out)


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("zpair", ["PP", "NN", "DD", "ND", "DN"])
@pytest.mark.parametrize("walls", [("D", "D", "N", "N"), ("N", "N", "N", "N"), ("D", "N", "N", "D")])
def test_operator_is_divergence_of_gradient(layout, zpair, walls):
    blocks = make(layout, n=3, nz=4, zpair=zpair, walls=walls, stretched=True)
    p = np.random.default_rng(3).standard_normal(inputs.total_cells(blocks))
    a = osv.apply_operator(blocks, p)
    b = staggered_div_grad(blocks, p)
    assert np.allclose(a, b, rtol=1e-12, atol=1e-12 * np.abs(a).max())


@pytest.mark.parametrize("layout", LAYOUTS)
def test_volume_weighted_symmetry_and_null_space(layout):
    blocks = make(layout, n=3, nz=4, zpair="NN", walls=("N", "N", "N", "N"), stretched=True)
    g = ogrid.Grid(blocks)
    A = g.matrix().toarray()
    VA = g.vol.ravel()[:, None] * A
    assert np.allclose(VA, VA.T, atol=1e-9 * np.abs(VA).max())
    assert np.allclose(A @ np.ones(A.shape[0]), 0.0, atol=1e-9 * np.abs(A).max())
    assert g.singular
    blocks = make(layout, n=3, nz=4, zpair="NN", walls=("D", "N", "N", "N"), stretched=True)
    g = ogrid.Grid(blocks)
    assert not g.singular
    assert np.abs(g.matrix().toarray() @ np.ones(g.vol.size)).max() > 1.0


def test_periodic_xy_connectivity_symmetry():
    blocks = make("2x2", n=3, nz=4, zpair="PP", periodic=(True, True), stretched=True)
    g = ogrid.Grid(blocks)
    assert g.singular
    A = g.matrix().toarray()
    VA = g.vol.ravel()[:, None] * A
    assert np.allclose(VA, VA.T, atol=1e-9 * np.abs(VA).max())


def test_uniform_grid_is_printed_seven_point_formula():
    """On a uniform periodic box the operator is Eq. 8 exactly."""
    nx, ny, nz = 6, 4, 8
    dx, dy, dz = 0.3, 0.7, 0.2
    xf, yf, zf = np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, np.arange(nz + 1) * dz
    blocks = inputs.make_blocks(xf, yf, zf, [(0, nx, 0, ny)], {}, ("P", "P"), periodic=(True, True))
    phi = np.random.default_rng(0).standard_normal((nz, ny, nx))
    lap = ((np.roll(phi, 1, 2) - 2 * phi + np.roll(phi, -1, 2)) / dx ** 2
           + (np.roll(phi, 1, 1) - 2 * phi + np.roll(phi, -1, 1)) / dy ** 2
           + (np.roll(phi, 1, 0) - 2 * phi + np.roll(phi, -1, 0)) / dz ** 2)
    assert np.allclose(osv.apply_operator(blocks, phi.ravel()), lap.ravel(), rtol=1e-12, atol=1e-10)


def test_second_order_solution_on_stretched_grid():
    """The discrete solution of A p = f for f = -3 pi^2 sin(pi x) cos(pi y) cos(pi z) approaches the
    continuous one at second order on a stretched grid (x Dirichlet, y and z Neumann walls). The
    pointwise truncation error is only first order there; the solution error is second order."""
    errs = []
    for n in (8, 16, 32):
        xf = inputs.tanh_faces(n, 0, 1.5, 0.0, 1.0)
        yf = inputs.tanh_faces(n, 1, 1.2, 0.0, 1.0)
        zf = np.linspace(0.0, 1.0, n + 1)
        blocks = inputs.make_blocks(xf, yf, zf, [(0, n, 0, n)], {"x-": "D", "x+": "D", "y-": "N", "y+": "N"},
                                    ("N", "N"))
        xc, yc, zc = 0.5 * (xf[1:] + xf[:-1]), 0.5 * (yf[1:] + yf[:-1]), 0.5 * (zf[1:] + zf[:-1])
        ph = np.cos(np.pi * zc)[:, None, None] * np.cos(np.pi * yc)[None, :, None] * np.sin(np.pi * xc)[None, None, :]
        p, _ = osv.solve(blocks, (-3 * np.pi ** 2 * ph).ravel())
        errs.append(np.abs(p - ph.ravel()).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)


def test_table2_layout_golden():
    """The four-block layout of Table 2: index-space corners give the connectivity of Fig. 1
    (1-2 and 2-3 along x, 2-4 along y); a congruent global grid on that layout is accepted and its
    oracle solve matches dense LU."""
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_blocks.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                c = [s.split() for s in line.split("|")]
                rows.append((int(c[0][0]), tuple(map(int, c[1])), tuple(map(int, c[2]))))
    assert [r[0] for r in rows] == [1, 2, 3, 4]
    x0 = min(r[1][0] for r in rows)
    y0 = min(r[1][1] for r in rows)
    rects = [(lo[0] - x0, hi[0] - x0 + 1, lo[1] - y0, hi[1] - y0 + 1) for _, lo, hi in rows]
    NX = max(r[1] for r in rects)
    NY = max(r[3] for r in rects)
    nz = rows[0][2][2] - rows[0][1][2] + 1
    assert (NX, NY, nz) == (40, 20, 2)
    xf = inputs.tanh_faces(NX, 0, 1.0, 0.0, 4.0)
    yf = inputs.tanh_faces(NY, 0, 1.0, 0.0, 2.0)
    zf = np.linspace(0.0, 0.1, 4 + 1)           # 4 cells along z so that every pair is exercised
    blocks = inputs.make_blocks(xf, yf, zf, rects, {"x-": "D", "x+": "N", "y-": "N", "y+": "N"}, ("N", "N"))
    assert blocks[0]["nbr"][0][1] == 1 and blocks[1]["nbr"][0][1] == 2 and blocks[1]["nbr"][1][1] == 3
    assert blocks[3]["bc"][1][0] == "B" and blocks[0]["bc"][1][1] == "N"
    f = inputs.uniform_rhs(blocks, 5)
    p, info = osv.solve(blocks, f)
    pd = osv.solve_dense(blocks, f)
    assert np.linalg.norm(p - pd) <= 1e-11 * np.linalg.norm(pd)
