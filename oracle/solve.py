"""The whole solve: Algorithm 1 (Sec. 2) on a multi-block grid, plus a dense direct solve.

Test infrastructure only (see the package docstring).

``solve`` follows Algorithm 1 step by step: forward transform of every z column of the right-hand
side (Table 1, as an O(n^2) matrix product), one multigrid solve of the reduced equation (Eq. 9) per
wavenumber, backward transform of the solution divided by theta.

Singular problems (a zero eigenvalue along z -- periodic or Neumann-Neumann -- and no Dirichlet face
in x-y) are solvable only for a compatible right-hand side (volume-weighted sum zero). Reading used
on both sides of the parity tests: a sum within 1e-12 of sum(vol |f|) is round-off, and the
volume-weighted mean is removed from f before solving; a larger one is an error. Of the solutions
(defined up to a constant) the one with zero volume-weighted mean is returned.

``solve_dense`` solves the assembled 3-D system (Eq. 8) by Gaussian elimination with partial
pivoting (LAPACK via numpy); for singular problems it solves the bordered system
[A 1; vol^T 0], which yields the same zero-mean solution of the mean-removed problem.
"""
from __future__ import annotations

import numpy as np

from . import transforms
from .grid import Grid
from .mg import Multigrid


class IncompatibleRHS(ValueError):
    pass


def _compatibility(g: Grid, F: np.ndarray):
    tot = float((g.vol * F).sum())
    mag = float((g.vol * np.abs(F)).sum())
    if abs(tot) > 1e-12 * mag:
        raise IncompatibleRHS(f"volume-weighted sum {tot:.3e} vs {mag:.3e}")
    return tot / float(g.vol.sum())


def solve(blocks, f, rtol_mode=1e-13, nu1=2, nu2=2, max_cycles=100, modes=None, mg=None, shift=0.0):
    """Solve (A + shift I) p = f (shift = 0: Eq. 8). Returns (p in the caller layout, info dict).

    ``modes`` restricts the per-wavenumber solves to a subset (the others are left zero): used to
    time a bounded sample of a large problem. ``mg`` reuses a prepared Multigrid hierarchy."""
    g = Grid(blocks, shift)
    F = g.to_planes(f)
    info = {"removed_mean": 0.0, "singular": g.singular, "kind": g.kind}
    if g.singular:
        mean = _compatibility(g, F)
        F = F - mean
        info["removed_mean"] = mean
    # Algorithm 1, first loop: forward transform along the homogeneous direction
    Fh = transforms.forward(g.kind, F)
    lam = transforms.eigenvalues(g.kind, g.nz)
    mg = mg or Multigrid(g.plane, nu1, nu2)
    Ph = np.zeros_like(Fh)
    cycles = np.zeros(g.nz, dtype=np.int64)
    mode_res = np.zeros(g.nz)
    # Algorithm 1, second loop: one reduced 2-D solve per wavenumber
    for q in (range(g.nz) if modes is None else modes):
        sigma = lam[q] / (g.dz * g.dz) + g.shift
        Ph[q], cycles[q], mode_res[q] = mg.solve(sigma, Fh[q], singular=(g.singular and lam[q] == 0.0),
                                                 rtol=rtol_mode, max_cycles=max_cycles)
    # Algorithm 1, third loop: backward transform
    P = transforms.backward(g.kind, Ph)
    if g.singular:
        P = P - float((g.vol * P).sum()) / float(g.vol.sum())
    p = g.from_planes(P)
    if modes is None:
        r = g.from_planes((F - g.apply(P)))
        info["rel_res"] = float(np.linalg.norm(r) / max(np.linalg.norm(F), 1e-300))
    info["cycles"] = cycles
    info["mode_rel_res"] = mode_res
    info["levels"] = len(mg.levels)
    return p, info


def solve_dense(blocks, f, shift=0.0):
    """Dense direct solve of the assembled 3-D system (tiny grids only)."""
    g = Grid(blocks, shift)
    F = g.to_planes(f)
    A = g.matrix().toarray()
    n = A.shape[0]
    rhs = F.ravel()
    if g.singular:
        _compatibility(g, F)
        B = np.zeros((n + 1, n + 1))
        B[:n, :n] = A
        B[:n, n] = 1.0
        B[n, :n] = g.vol.ravel()
        x = np.linalg.solve(B, np.concatenate([rhs, [0.0]]))[:n]
    else:
        x = np.linalg.solve(A, rhs)
    return g.from_planes(x.reshape(g.nz, g.plane.n))


def apply_operator(blocks, p, shift=0.0):
    """(A + shift I) p (Eq. 8) in the caller's layout."""
    g = Grid(blocks, shift)
    return g.from_planes(g.apply(g.to_planes(p)))


def rel_residual(blocks, f, p, shift=0.0):
    """||f - (A + shift I) p|| / ||f|| (2-norm over all cells, rows per unit volume)."""
    g = Grid(blocks, shift)
    F = g.to_planes(f)
    r = F - g.apply(g.to_planes(p))
    return float(np.linalg.norm(r) / max(np.linalg.norm(F), 1e-300))
