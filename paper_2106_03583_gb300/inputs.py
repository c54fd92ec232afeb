"""Seeded synthetic inputs shaped like the paper's workloads: block layouts, grids and right-hand sides.

This module holds no step of the Poisson solve. It only describes problems:

* the block description format that both the CUDA library's binding and the CPU oracle read
  (Sec. 3.1, Table 2: per block ``lo``/``hi`` index-space corners, a grid mapping, and the
  boundary condition of every face, with block-block connectivity);
* hyperbolic-tangent grid clustering (Sec. 3.1, ``gr.type``/``gr.factor`` of Table 2);
* seeded right-hand sides: uniform noise, or the divergence of a random-phase velocity field
  (the right-hand side of Eq. 4 with gamma*dt = 1).

Block description (plain data, one dict per block)::

    {"lo": (x, y, z), "hi": (x, y, z),          # inclusive index-space corners, n = hi - lo + 1
     "dx": (wx, wy, wz),                          # float64 cell widths, lengths n_x, n_y, n_z
     "bc": (("D"|"N"|"P"|"B", ...), ... ),        # per axis (lower face, upper face)
     "nbr": ((i, i), (i, i), (i, i))}             # neighbour block id across "B" faces, else -1

``"D"`` is a homogeneous Dirichlet face, ``"N"`` a homogeneous Neumann face, ``"B"`` a face shared
with block ``nbr``, and ``"P"`` a periodic face (the block connected to itself across the opposite
face, i.e. a cyclic connectivity as in Sec. 3.1). Arrays are laid out per block as ``[z][y][x]``
(x fastest), blocks concatenated in id order.
"""
from __future__ import annotations

import numpy as np
import scipy.fft

__all__ = [
    "tanh_faces",
    "make_blocks",
    "block_sizes",
    "total_cells",
    "uniform_rhs",
    "divergence_rhs",
    "config",
    "CONFIGS",
    "random_problem",
]


def tanh_faces(n: int, gr_type: int, factor: float, lmin: float, lmax: float) -> np.ndarray:
    """Face coordinates x_0..x_n of a tanh-clustered grid on [lmin, lmax] (Sec. 3.1, Table 2).

    The paper takes the mapping from Orlandi's book without printing it. With xi = i/n and
    a = factor (0 = uniform):
      two-sided (type 0):  x = (1 + tanh(a (xi - 1/2)) / tanh(a/2)) / 2
      lower end (type -1): x = 1 + tanh(a (xi - 1)) / tanh(a)
      upper end (type +1): x = tanh(a xi) / tanh(a)
    """
    xi = np.arange(n + 1, dtype=np.float64) / n
    a = float(factor)
    if a == 0.0:
        s = xi
    elif gr_type == 0:
        s = 0.5 * (1.0 + np.tanh(a * (xi - 0.5)) / np.tanh(0.5 * a))
    elif gr_type == -1:
        s = 1.0 + np.tanh(a * (xi - 1.0)) / np.tanh(a)
    elif gr_type == 1:
        s = np.tanh(a * xi) / np.tanh(a)
    else:
        raise ValueError(f"unknown gr_type {gr_type}")
    s[0], s[-1] = 0.0, 1.0
    return lmin + (lmax - lmin) * s


def make_blocks(xfaces, yfaces, zfaces, rects, wall_bc, z_bc, periodic=(False, False), inner_wall="N"):
    """Cut a global tensor grid into blocks and connect them.

    ``xfaces``/``yfaces``/``zfaces``: global face coordinates. ``rects``: list of (x0, x1, y0, y1)
    global cell ranges (half-open) of the blocks. Faces shared by two blocks become ``"B"``
    connections; faces on the bounding box take ``wall_bc`` = {"x-","x+","y-","y+"} (or periodic
    wrap when ``periodic[axis]``); other physical faces (re-entrant corners of L-shapes) take
    ``inner_wall``. Every block spans all of z, with the z pair ``z_bc`` (``"P"`` for periodic).
    """
    xfaces, yfaces, zfaces = (np.asarray(a, dtype=np.float64) for a in (xfaces, yfaces, zfaces))
    NX, NY, NZ = len(xfaces) - 1, len(yfaces) - 1, len(zfaces) - 1
    wx, wy, wz = np.diff(xfaces), np.diff(yfaces), np.diff(zfaces)
    blocks = []
    for (x0, x1, y0, y1) in rects:
        blocks.append({"lo": (x0, y0, 0), "hi": (x1 - 1, y1 - 1, NZ - 1),
                       "dx": (wx[x0:x1].copy(), wy[y0:y1].copy(), wz.copy()),
                       "bc": [["?", "?"], ["?", "?"], [z_bc[0], z_bc[1]]],
                       "nbr": [[-1, -1], [-1, -1], [-1, -1]]})
    for b, (x0, x1, y0, y1) in enumerate(rects):
        lo = (x0, y0)
        hi = (x1, y1)
        for axis in range(2):
            o = 1 - axis
            olo, ohi = (y0, y1) if axis == 0 else (x0, x1)
            for side in range(2):
                pos = lo[axis] if side == 0 else hi[axis]
                found = -1
                for c, (cx0, cx1, cy0, cy1) in enumerate(rects):
                    clo, chi = (cx0, cy0), (cx1, cy1)
                    cpos = chi[axis] if side == 0 else clo[axis]
                    colo, cohi = (cy0, cy1) if axis == 0 else (cx0, cx1)
                    if c != b and cpos == pos and colo == olo and cohi == ohi:
                        found = c
                n_glob = NX if axis == 0 else NY
                on_box = pos == (0 if side == 0 else n_glob)
                if found >= 0:
                    blocks[b]["bc"][axis][side] = "B"
                    blocks[b]["nbr"][axis][side] = found
                elif on_box and periodic[axis]:
                    # wrap to the block on the opposite side of the bounding box
                    wrap = -1
                    for c, (cx0, cx1, cy0, cy1) in enumerate(rects):
                        clo, chi = (cx0, cy0), (cx1, cy1)
                        cpos = chi[axis] if side == 0 else clo[axis]
                        colo, cohi = (cy0, cy1) if axis == 0 else (cx0, cx1)
                        want = n_glob if side == 0 else 0
                        if cpos == want and colo == olo and cohi == ohi:
                            wrap = c
                    if wrap < 0:
                        raise ValueError("periodic wrap has no matching block face")
                    if wrap == b:
                        blocks[b]["bc"][axis][side] = "P"
                    else:
                        blocks[b]["bc"][axis][side] = "B"
                        blocks[b]["nbr"][axis][side] = wrap
                elif on_box:
                    blocks[b]["bc"][axis][side] = wall_bc[("x" if axis == 0 else "y") + ("-" if side == 0 else "+")]
                else:
                    blocks[b]["bc"][axis][side] = inner_wall
    for blk in blocks:
        blk["bc"] = tuple(tuple(p) for p in blk["bc"])
        blk["nbr"] = tuple(tuple(p) for p in blk["nbr"])
    return blocks


def block_sizes(blocks):
    return [tuple(int(blk["hi"][a] - blk["lo"][a] + 1) for a in range(3)) for blk in blocks]


def total_cells(blocks) -> int:
    return int(sum(nx * ny * nz for nx, ny, nz in block_sizes(blocks)))


def uniform_rhs(blocks, seed: int, remove_mean: bool = True) -> np.ndarray:
    """f ~ U[-1, 1] (numpy PCG64), with the volume-weighted mean removed if asked."""
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.uniform(-1.0, 1.0, total_cells(blocks))
    if remove_mean:
        vol = _cell_volumes(blocks)
        f -= np.dot(vol, f) / vol.sum()
    return f


def _cell_volumes(blocks) -> np.ndarray:
    out = []
    for blk in blocks:
        wx, wy, wz = blk["dx"]
        out.append((wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).ravel())
    return np.concatenate(out)


def divergence_rhs(blocks, seed: int, slope: float = -5.0 / 3.0, workers: int = -1) -> np.ndarray:
    """f = D u for a seeded random-phase face-velocity field u (right-hand side of Eq. 4, gamma*dt = 1).

    Each velocity component is a periodic random-phase field on the bounding box of the blocks,
    with a shell energy spectrum E(k) ~ k^slope on the index grid (amplitude |k|^((slope - 2)/2)
    in 3-D). The normal velocity is zero on every physical (Dirichlet or Neumann) face, so that the
    volume-weighted sum of f vanishes up to round-off. f is scaled to unit RMS.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = block_sizes(blocks)
    x0 = min(b["lo"][0] for b in blocks)
    y0 = min(b["lo"][1] for b in blocks)
    NX = max(b["hi"][0] for b in blocks) - x0 + 1
    NY = max(b["hi"][1] for b in blocks) - y0 + 1
    NZ = sizes[0][2]
    amp_exp = (slope - 2.0) / 2.0
    kz = scipy.fft.fftfreq(NZ, 1.0 / NZ)
    ky = scipy.fft.fftfreq(NY, 1.0 / NY)
    kx = scipy.fft.rfftfreq(NX, 1.0 / NX)
    f_blocks = [np.zeros((nz, ny, nx)) for (nx, ny, nz) in sizes]
    for comp in range(3):
        kk = np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)
        with np.errstate(divide="ignore"):
            amp = np.where(kk > 0, kk ** amp_exp, 0.0)
        del kk
        phase = rng.uniform(0.0, 2.0 * np.pi, amp.shape)
        spec = amp * np.exp(1j * phase)
        del amp, phase
        field = scipy.fft.irfftn(spec, s=(NZ, NY, NX), workers=workers)  # value i = face i - 1/2
        del spec
        field /= max(np.sqrt(np.mean(field ** 2)), 1e-300)
        for b, blk in enumerate(blocks):
            nx, ny, nz = sizes[b]
            bx, by = blk["lo"][0] - x0, blk["lo"][1] - y0
            wx, wy, wz = blk["dx"]
            if comp == 0:
                fl = np.empty((nz, ny, nx + 1))
                fl[:, :, :nx] = field[:, by:by + ny, bx:bx + nx]
                fl[:, :, nx] = field[:, by:by + ny, (bx + nx) % NX]
                if blk["bc"][0][0] in "DN":
                    fl[:, :, 0] = 0.0
                if blk["bc"][0][1] in "DN":
                    fl[:, :, nx] = 0.0
                f_blocks[b] += (fl[:, :, 1:] - fl[:, :, :-1]) / wx[None, None, :]
            elif comp == 1:
                fl = np.empty((nz, ny + 1, nx))
                fl[:, :ny, :] = field[:, by:by + ny, bx:bx + nx]
                fl[:, ny, :] = field[:, (by + ny) % NY, bx:bx + nx]
                if blk["bc"][1][0] in "DN":
                    fl[:, 0, :] = 0.0
                if blk["bc"][1][1] in "DN":
                    fl[:, ny, :] = 0.0
                f_blocks[b] += (fl[:, 1:, :] - fl[:, :-1, :]) / wy[None, :, None]
            else:
                fl = np.empty((nz + 1, ny, nx))
                fl[:nz] = field[:, by:by + ny, bx:bx + nx]
                fl[nz] = field[0, by:by + ny, bx:bx + nx]
                if blk["bc"][2][0] in "DN":
                    fl[0] = 0.0
                if blk["bc"][2][1] in "DN":
                    fl[nz] = 0.0
                f_blocks[b] += (fl[1:] - fl[:-1]) / wz[:, None, None]
            del fl
        del field
    f = np.concatenate([fb.ravel() for fb in f_blocks])
    f /= max(np.sqrt(np.mean(f ** 2)), 1e-300)
    return f


def _grid2x2(n, lx, ly, nz, lz, gy_type, gy_factor):
    xf = tanh_faces(2 * n, 0, 0.0, 0.0, lx)
    yf = tanh_faces(2 * n, gy_type, gy_factor, 0.0, ly)
    zf = np.linspace(0.0, lz, nz + 1)
    rects = [(0, n, 0, n), (n, 2 * n, 0, n), (0, n, n, 2 * n), (n, 2 * n, n, 2 * n)]
    return xf, yf, zf, rects


def config(name: str, seed: int = 0, scale: int = 1):
    """Blocks and right-hand side of a named workload.

    ``"c64"``: one block 64x64 (x Dirichlet-Dirichlet, y Neumann-Neumann, unit box) by n_z = 32
    periodic; f ~ U[-1, 1] with the mean removed.
    ``"mb2x2"``: a 2x2 layout of 256x256-cell blocks (x uniform on [0, 2], y two-sided tanh
    factor 1.5 on [0, 2]), all outer faces Neumann, n_z = 256 Neumann-Neumann on [0, 1];
    f = D u with a k^-5/3 spectrum.
    ``"mb2x2_z64"``: the same with n_z = 64 (a smaller case of the same kernels for profiling).
    ``"chan"``: one block 1024x512 (x uniform on [0, 2] Dirichlet-Dirichlet, y two-sided tanh
    factor 2.0 on [0, 1] Neumann-Neumann) by n_z = 512 periodic on [0, 1]; f = D u, k^-5/3.
    ``scale`` divides every cell count (and keeps the domain), giving small cases with the same
    structure.
    """
    if name == "c64":
        n, nz = 64 // scale, 32 // scale
        xf = np.linspace(0.0, 1.0, n + 1)
        zf = np.linspace(0.0, 1.0, nz + 1)
        blocks = make_blocks(xf, xf, zf, [(0, n, 0, n)],
                             {"x-": "D", "x+": "D", "y-": "N", "y+": "N"}, ("P", "P"))
        return blocks, uniform_rhs(blocks, seed, remove_mean=True)
    if name in ("mb2x2", "mb2x2_z64"):
        n, nz = 256 // scale, (256 if name == "mb2x2" else 64) // scale
        xf, yf, zf, rects = _grid2x2(n, 2.0, 2.0, nz, 1.0, 0, 1.5)
        blocks = make_blocks(xf, yf, zf, rects, {"x-": "N", "x+": "N", "y-": "N", "y+": "N"}, ("N", "N"))
        return blocks, divergence_rhs(blocks, seed)
    if name == "chan":
        nx, ny, nz = 1024 // scale, 512 // scale, 512 // scale
        xf = tanh_faces(nx, 0, 0.0, 0.0, 2.0)
        yf = tanh_faces(ny, 0, 2.0, 0.0, 1.0)
        zf = np.linspace(0.0, 1.0, nz + 1)
        blocks = make_blocks(xf, yf, zf, [(0, nx, 0, ny)],
                             {"x-": "D", "x+": "D", "y-": "N", "y+": "N"}, ("P", "P"))
        return blocks, divergence_rhs(blocks, seed)
    raise ValueError(f"unknown workload {name!r}")


def random_problem(rng, xy_exp=(5, 9), z_exp=(5, 8), rhs="divergence"):
    """One problem of the mixed workloads (many independent solves, or a stream of requests).

    Sizes are log-uniform per axis: n_x = 2^ex, n_y = 2^ey with ex, ey uniform in ``xy_exp``, and
    n_z = 2^ez with ez uniform in ``z_exp``; cubic cells of width 1/64. The x-y grid is cut into 1 to
    4 blocks (one block, halves along x or y, an L of three quarters, 2x2 quarters); every wall and
    the z pair (PP, NN, DD, ND, DN) are drawn at random. ``rhs``: ``"divergence"`` (f = D u,
    k^-5/3) or ``"uniform"`` (U[-1, 1]), compatible whenever the problem is singular.
    Returns (blocks, f, description)."""
    ex, ey = (int(v) for v in rng.integers(xy_exp[0], xy_exp[1] + 1, 2))
    ez = int(rng.integers(z_exp[0], z_exp[1] + 1))
    nx, ny, nz = 2 ** ex, 2 ** ey, 2 ** ez
    hx, hy = nx // 2, ny // 2
    nblk = int(rng.integers(1, 5))
    if nblk == 1:
        rects = [(0, nx, 0, ny)]
    elif nblk == 2:
        rects = [(0, hx, 0, ny), (hx, nx, 0, ny)] if rng.random() < 0.5 else [(0, nx, 0, hy), (0, nx, hy, ny)]
    elif nblk == 3:
        rects = [(0, hx, 0, hy), (hx, nx, 0, hy), (0, hx, hy, ny)]
    else:
        rects = [(0, hx, 0, hy), (hx, nx, 0, hy), (0, hx, hy, ny), (hx, nx, hy, ny)]
    zp = str(rng.choice(["PP", "NN", "DD", "ND", "DN"]))
    walls = {k: ("D" if rng.random() < 0.5 else "N") for k in ("x-", "x+", "y-", "y+")}
    h = 1.0 / 64.0
    blocks = make_blocks(np.arange(nx + 1) * h, np.arange(ny + 1) * h, np.arange(nz + 1) * h, rects, walls,
                         ("P", "P") if zp == "PP" else (zp[0], zp[1]), inner_wall="N")
    singular = zp in ("PP", "NN") and "D" not in walls.values()
    seed = int(rng.integers(0, 2 ** 31))
    f = divergence_rhs(blocks, seed) if rhs == "divergence" else uniform_rhs(blocks, seed, remove_mean=singular)
    desc = f"{nx}x{ny}x{nz} {len(rects)} block(s) z {zp} walls {''.join(walls.values())}"
    return blocks, f, desc


CONFIGS = {
    "c64": "1 block 64x64x32, x D-D / y N-N / z periodic (DFT), uniform unit box, f~U[-1,1]",
    "mb2x2": "2x2 blocks of 256x256, y tanh 1.5, Neumann walls, n_z=256 Neumann-Neumann (DCT-II), f=Du k^-5/3",
    "mb2x2_z64": "mb2x2 with n_z=64 (profiling size, 134 MB per field)",
    "chan": "1 block 1024x512, y tanh 2.0, x D-D / y N-N, n_z=512 periodic (DFT), f=Du k^-5/3",
}
