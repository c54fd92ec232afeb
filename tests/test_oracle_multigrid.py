"""Pins of the oracle's multigrid pieces (free choices, since the paper leaves the multigrid to hypre,
Sec. 3.3: cell-centred 2x2 coarsening, red-black Gauss-Seidel, area-weighted restriction, three-point
affine prolongation, rediscretised coarse operators) against facts of the geometry and of multigrid
theory.

The per-cycle GPU parity tests compare the kernels with these pieces one cycle at a time, where the
converged-solution pins (dense LU, eigenfunctions) cannot see them: a wrong weight only slows a
convergent cycle down. Each test also plants a plausible mistake and checks that it fails.
"""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import mg as omg
from paper_2106_03583_gb300 import inputs
from layouts import rects

N = 8   # block unit: the bounding box is 2N x 2N cells


def faces(seed, n):
    """Strongly non-uniform face coordinates (widths U[0.4, 1.6]) starting at 0."""
    w = np.random.default_rng(seed).uniform(0.4, 1.6, n)
    return np.concatenate([[0.0], np.cumsum(w)])


def problem(layout, walls=("N", "N", "N", "N"), periodic=(False, False), seed=0):
    xf, yf = faces(seed, 2 * N), faces(seed + 100, 2 * N)
    blocks = inputs.make_blocks(xf, yf, np.linspace(0.0, 1.0, 3), rects(layout, N),
                                {"x-": walls[0], "x+": walls[1], "y-": walls[2], "y+": walls[3]},
                                ("N", "N"), periodic=periodic, inner_wall="N")
    return blocks, xf, yf


def centres(plane, xf, yf, level):
    """Cell-centre coordinates of every cell of a level, from the global faces (level l keeps every
    2^l-th face)."""
    xl, yl = xf[::2 ** level], yf[::2 ** level]
    cx, cy = [], []
    for b, blk in enumerate(plane.blocks):
        rx, ry, nx, ny = blk["lo"][0], blk["lo"][1], plane.nx[b], plane.ny[b]
        assert np.allclose(np.diff(xl)[rx:rx + nx], blk["dx"][0], rtol=1e-13)
        assert np.allclose(np.diff(yl)[ry:ry + ny], blk["dx"][1], rtol=1e-13)
        xc = 0.5 * (xl[rx:rx + nx] + xl[rx + 1:rx + nx + 1])
        yc = 0.5 * (yl[ry:ry + ny] + yl[ry + 1:ry + ny + 1])
        cx.append(np.tile(xc, ny))
        cy.append(np.repeat(yc, nx))
    return np.concatenate(cx), np.concatenate(cy)


def near_face(plane, axis, kinds):
    """Cells with a face of one of the given neighbour codes (-1 Dirichlet, -2 Neumann) on `axis`."""
    m = np.zeros(plane.n, bool)
    for side in range(2):
        for k in kinds:
            m |= plane.nbr[axis, side] == k
    return m


@pytest.mark.parametrize("layout", ["1", "1x2", "L", "2x2"])
def test_restriction_is_the_area_average(layout):
    """Restriction is the area-weighted mean over the four children: it keeps constants and, because
    the area-weighted mean of the children's centres is the parent's centre, maps the fine x and y
    centre coordinates to the coarse ones; it conserves the area integral."""
    blocks, xf, yf = problem(layout)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    assert len(mg.levels) >= 3
    for l in range(len(mg.levels) - 1):
        F, C, R = mg.levels[l], mg.levels[l + 1], mg.R[l]
        fx, fy = centres(F, xf, yf, l)
        cx, cy = centres(C, xf, yf, l + 1)
        assert np.all(np.diff(R.indptr) == 4)
        assert np.allclose(R @ np.ones(F.n), 1.0, rtol=0, atol=1e-14)
        assert np.allclose(R @ fx, cx, rtol=1e-13)
        assert np.allclose(R @ fy, cy, rtol=1e-13)
        r = np.random.default_rng(l).standard_normal(F.n)
        assert np.isclose(C.area @ (R @ r), F.area @ r, rtol=1e-12)
        # planted: the plain (unweighted) mean misplaces the centre on a stretched grid
        bad = R.copy()
        bad.data[:] = 0.25
        assert not np.allclose(bad @ fx, cx, rtol=1e-6)


@pytest.mark.parametrize("layout", ["1", "1x2", "L", "2x2"])
def test_prolongation_is_exact_for_affine_fields(layout):
    """The three-point affine interpolation reproduces a + b x + c y at every fine cell whose coarse
    parent has no physical face (interpolation along x and y between adjacent coarse centres, across
    block faces too, since connected faces coincide)."""
    blocks, xf, yf = problem(layout)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    for l in range(len(mg.levels) - 1):
        F, C, P = mg.levels[l], mg.levels[l + 1], mg.P[l]
        fx, fy = centres(F, xf, yf, l)
        cx, cy = centres(C, xf, yf, l + 1)
        affine = lambda x, y: 0.7 - 1.3 * x + 2.1 * y
        parent_free = ~(near_face(C, 0, (-1, -2)) | near_face(C, 1, (-1, -2)))
        # the parent of each fine cell is the coarse cell that contains its centre
        par = parent_of(F, C, fx, fy, cx, cy, xf, yf, l)
        mask = parent_free[par]
        if not mask.any():
            assert l > 0 and C.n <= 16        # 2x2-cell coarse blocks have no interior cell
            continue
        e = P @ affine(cx, cy)
        assert np.allclose(e[mask], affine(fx, fy)[mask], rtol=0, atol=1e-12)
        # planted: piecewise-constant prolongation (parent value only) is not exact
        pc = np.zeros(F.n)
        pc[:] = affine(cx, cy)[par]
        assert not np.allclose(pc[mask], affine(fx, fy)[mask], atol=1e-6)


def parent_of(F, C, fx, fy, cx, cy, xf, yf, l):
    """The coarse cell containing each fine centre (same block, geometric containment)."""
    xl, yl = xf[::2 ** (l + 1)], yf[::2 ** (l + 1)]
    par = np.empty(F.n, np.int64)
    for b in range(F.nb):
        fi = F.index_array(b).ravel()
        ci = C.index_array(b)
        rx, ry = C.blocks[b]["lo"][0], C.blocks[b]["lo"][1]
        I = np.searchsorted(xl, fx[fi], side="right") - 1 - rx
        J = np.searchsorted(yl, fy[fi], side="right") - 1 - ry
        assert I.min() >= 0 and I.max() < C.nx[b] and J.min() >= 0 and J.max() < C.ny[b]
        par[fi] = ci[J, I]
    return par


@pytest.mark.parametrize("axis", [0, 1])
def test_prolongation_ghosts_at_physical_faces(axis):
    """At a Dirichlet face the mirrored ghost (-e) makes the interpolation exact for a field that is
    linear along the axis and zero on the face; at a Neumann face the ghost (+e) keeps constants.
    A dropped ghost, a flipped sign or a wrong factor fails one of the two."""
    walls = ["N", "N", "N", "N"]
    walls[2 * axis] = "D"                               # the lower face of `axis`
    blocks, xf, yf = problem("2x2", walls=tuple(walls), seed=3)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    for l in range(len(mg.levels) - 1):
        F, C, P = mg.levels[l], mg.levels[l + 1], mg.P[l]
        fx, fy = centres(F, xf, yf, l)
        cx, cy = centres(C, xf, yf, l + 1)
        par = parent_of(F, C, fx, fy, cx, cy, xf, yf, l)
        # odd about the Dirichlet face, constant along the other axis (whose faces are Neumann)
        g = (lambda x, y: x - xf[0]) if axis == 0 else (lambda x, y: y - yf[0])
        ok = ~near_face(C, axis, (-2,))[par]             # not next to this axis' Neumann face
        assert near_face(C, axis, (-1,))[par][ok].any()
        e = P @ g(cx, cy)
        assert np.allclose(e[ok], g(fx, fy)[ok], rtol=0, atol=1e-12)
    # Neumann everywhere: constants are kept on every cell
    blocks, xf, yf = problem("L", seed=4)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    for l in range(len(mg.levels) - 1):
        assert np.allclose(mg.P[l] @ np.ones(mg.levels[l + 1].n), 1.0, rtol=0, atol=1e-14)


@pytest.mark.parametrize("layout,periodic", [("1", (False, False)), ("L", (False, False)),
                                             ("2x2", (True, False)), ("1x2", (True, True))])
def test_red_black_half_sweep(layout, periodic):
    """Cells of one colour (global index-space parity) are not coupled to each other, across block
    faces and periodic wraps too, so one half-sweep solves every equation of its colour exactly and
    leaves the other colour untouched."""
    blocks, _, _ = problem(layout, walls=("D", "N", "N", "D"), periodic=periodic, seed=5)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    rng = np.random.default_rng(7)
    for l, pl in enumerate(mg.levels[:-1]):
        red = pl.red
        assert red.sum() == pl.n // 2
        Arr = pl.A[red][:, red].tocoo()
        off = Arr.row != Arr.col
        assert np.all(Arr.data[off] == 0.0)
        u, f = rng.standard_normal(pl.n), rng.standard_normal(pl.n)
        for sigma in (0.0, -37.0):
            for colour in (True, False):
                mask = red if colour else ~red
                v = mg.half_sweep(l, sigma, u, f, colour)
                r = f - (pl.A @ v + sigma * v)
                scale = np.abs(f).max() + np.abs(pl.diag).max() * np.abs(v).max()
                assert np.abs(r[mask]).max() <= 1e-13 * scale
                assert np.array_equal(v[~mask], u[~mask])


@pytest.mark.parametrize("layout", ["1", "L", "2x2"])
def test_coarse_operator_is_rediscretised(layout):
    """A coarse level is the same finite-volume operator built on every other face (the 2x2
    coarsening keeps each block's faces and connections): identical to the plane assembled from the
    coarse face arrays directly."""
    walls = ("D", "N", "N", "D")
    blocks, xf, yf = problem(layout, walls=walls, seed=6)
    mg = omg.Multigrid(ogrid.Plane(blocks), max_coarse=4)
    for l in range(1, len(mg.levels)):
        s = 2 ** l
        direct = inputs.make_blocks(xf[::s], yf[::s], np.linspace(0.0, 1.0, 3),
                                    [(a // s, b // s, c // s, d // s) for (a, b, c, d) in rects(layout, N)],
                                    {"x-": walls[0], "x+": walls[1], "y-": walls[2], "y+": walls[3]},
                                    ("N", "N"), inner_wall="N")
        ref = ogrid.Plane(direct)
        lv = mg.levels[l]
        assert ref.n == lv.n
        assert np.array_equal(ref.red, lv.red)
        d = (ref.A - lv.A).tocoo()
        assert np.abs(d.data).max(initial=0.0) <= 1e-12 * np.abs(ref.A.data).max()


def test_vcycle_contraction_is_grid_independent():
    """Textbook multigrid: a V(2,2) cycle with red-black Gauss-Seidel contracts the error of the 2-D
    Poisson problem by a factor well below 1 that does not grow with the mesh (at most 0.2 per cycle
    here, 64x64 and 128x128 cells, Dirichlet walls). A restriction that sums instead of averaging, a
    prolongation at half strength, or a coarse operator built on the fine widths (4x too strong)
    breaks the bound."""
    def factor(n, plant=None):
        xf = np.linspace(0.0, 1.0, n + 1)
        blocks = inputs.make_blocks(xf, xf, np.linspace(0.0, 1.0, 3), [(0, n, 0, n)],
                                    {"x-": "D", "x+": "D", "y-": "D", "y+": "D"}, ("N", "N"))
        mg = omg.Multigrid(ogrid.Plane(blocks), 2, 2, max_coarse=16)
        if plant == "sum":
            mg.R = [4.0 * R for R in mg.R]
        elif plant == "half":
            mg.P = [0.5 * P for P in mg.P]
        elif plant == "coarse":
            for lv in mg.levels[1:]:
                lv.A, lv.diag = 4.0 * lv.A, 4.0 * lv.diag
        u = np.random.default_rng(n).standard_normal(mg.levels[0].n)
        f = np.zeros_like(u)
        rho = []
        for _ in range(7):
            v = mg.vcycle(0, 0.0, u, f, False)
            rho.append(np.linalg.norm(v) / np.linalg.norm(u))
            u = v
        return max(rho[3:])
    for n in (64, 128):
        assert factor(n) <= 0.2
    for plant in ("sum", "half", "coarse"):
        assert factor(64, plant) > 0.5
