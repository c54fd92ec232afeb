"""Textbook cell-centred geometric multigrid for the reduced 2-D equations (Eq. 9, Sec. 2).

Test infrastructure only (see the package docstring).

For wavenumber q the reduced equation is (A_xy + sigma_q I) u = f with sigma_q = lambda_q / dz^2
(Eq. 9 written with the synthesis direction last: the diagonal of the x-y operator shifted by the
eigenvalue of Table 1, which is <= 0). The paper leaves the multigrid to hypre (Sec. 3.3, PFMG with a
point smoother); the choices below are the free ones of a textbook V-cycle:

* hierarchy: every block halved along x and y (coarse faces = every other fine face), operator
  rediscretised on the coarse widths with the same face rules, the same shift on every level;
* smoother: red-black Gauss-Seidel, colour = parity of the global index-space position, nu1 sweeps
  before and nu2 after the coarse correction (red then black in each sweep);
* restriction: area-weighted average of the fine residual over the four children;
* prolongation: the affine (three-point) interpolation e_f = e_C + w_x (e_X - e_C) + w_y (e_Y - e_C),
  where C is the parent, X/Y the coarse neighbours on the fine cell's side and w = (distance from the
  fine centre to C's centre) / (distance between the two coarse centres); a physical face supplies the
  mirrored ghost (Dirichlet -e_C, Neumann +e_C). It needs no diagonal neighbour, so block corners
  (including re-entrant ones) need no special rule;
* coarsest level: a dense direct solve; when the x-y problem is singular (sigma = 0 and no Dirichlet
  face) the bordered system [A 1; area^T 0] picks the zero area-weighted-mean solution.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp

from .grid import Plane


def build_levels(plane: Plane, max_coarse: int = 64):
    levels = [plane]
    while levels[-1].n > max_coarse and levels[-1].can_coarsen():
        levels.append(levels[-1].coarsen())
    return levels


def restriction(fine: Plane, coarse: Plane) -> sp.csr_matrix:
    """R[c, f] = area_f / area_c for the four children f of coarse cell c."""
    rows, cols, vals = [], [], []
    for b in range(fine.nb):
        fi = fine.index_array(b)
        ci = coarse.index_array(b)
        parent = ci[np.arange(fine.ny[b])[:, None] // 2, np.arange(fine.nx[b])[None, :] // 2]
        rows.append(parent.ravel()); cols.append(fi.ravel())
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    vals = fine.area[cols] / coarse.area[rows]
    return sp.csr_matrix((vals, (rows, cols)), shape=(coarse.n, fine.n))


def prolongation(fine: Plane, coarse: Plane) -> sp.csr_matrix:
    """Affine three-point interpolation of a coarse correction to the fine cell centres."""
    rows, cols, vals = [], [], []
    cw = (coarse.wx, coarse.wy)
    for b in range(fine.nb):
        fi = fine.index_array(b)
        ci = coarse.index_array(b)
        jj, ii = np.meshgrid(np.arange(fine.ny[b]), np.arange(fine.nx[b]), indexing="ij")
        parent = ci[jj // 2, ii // 2].ravel()
        f = fi.ravel()
        rows.append(f); cols.append(parent); vals.append(np.ones(f.size))
        wfx = np.asarray(fine.blocks[b]["dx"][0], float)
        wfy = np.asarray(fine.blocks[b]["dx"][1], float)
        for axis, (pos, wf) in enumerate(((ii.ravel(), wfx), (jj.ravel(), wfy))):
            side = pos % 2                       # left/lower child looks at side 0, right/upper at 1
            sib = pos + np.where(side == 0, 1, -1)
            d = 0.5 * wf[sib]                    # fine centre to parent centre = half the sibling width
            nb = coarse.nbr[axis][side, parent]
            wc = cw[axis][parent]
            inner = nb >= 0
            H = np.where(inner, 0.5 * (wc + cw[axis][np.where(inner, nb, 0)]), wc)
            w = d / H
            # interior / block face: + w (e_nb - e_C)
            rows.append(f[inner]); cols.append(nb[inner]); vals.append(w[inner])
            rows.append(f[inner]); cols.append(parent[inner]); vals.append(-w[inner])
            # Dirichlet face: ghost -e_C gives -2 w e_C; Neumann face: ghost +e_C gives nothing
            dir_ = nb == -1
            rows.append(f[dir_]); cols.append(parent[dir_]); vals.append(-2.0 * w[dir_])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(fine.n, coarse.n))


class Multigrid:
    def __init__(self, plane: Plane, nu1: int = 2, nu2: int = 2, max_coarse: int = 64):
        self.levels = build_levels(plane, max_coarse)
        self.R = [restriction(self.levels[l], self.levels[l + 1]) for l in range(len(self.levels) - 1)]
        self.P = [prolongation(self.levels[l], self.levels[l + 1]) for l in range(len(self.levels) - 1)]
        self.nu1, self.nu2 = nu1, nu2
        self._coarse_cache = {}

    # ---- pieces of one cycle (also used one by one by the kernel parity tests)
    def operator(self, level: int, sigma: float, u: np.ndarray) -> np.ndarray:
        pl = self.levels[level]
        return pl.A @ u + sigma * u

    def residual(self, level, sigma, u, f):
        return f - self.operator(level, sigma, u)

    def half_sweep(self, level, sigma, u, f, red: bool):
        """Gauss-Seidel update of every cell of one colour (cells of one colour are not coupled)."""
        pl = self.levels[level]
        mask = pl.red if red else ~pl.red
        r = self.residual(level, sigma, u, f)
        u = u.copy()
        u[mask] += r[mask] / (pl.diag[mask] + sigma)
        return u

    def sweep(self, level, sigma, u, f):
        u = self.half_sweep(level, sigma, u, f, True)
        return self.half_sweep(level, sigma, u, f, False)

    def restrict(self, level, r):
        return self.R[level] @ r

    def prolong(self, level, e):
        return self.P[level] @ e

    def coarse_solve(self, sigma, f, singular):
        key = (sigma, singular)
        lv = self.levels[-1]
        if key not in self._coarse_cache:
            A = lv.A.toarray() + sigma * np.eye(lv.n)
            if singular:
                B = np.zeros((lv.n + 1, lv.n + 1))
                B[:lv.n, :lv.n] = A
                B[:lv.n, lv.n] = 1.0
                B[lv.n, :lv.n] = lv.area
                A = B
            self._coarse_cache[key] = scipy.linalg.lu_factor(A)
        rhs = np.concatenate([f, [0.0]]) if singular else f
        return scipy.linalg.lu_solve(self._coarse_cache[key], rhs)[:lv.n]

    def vcycle(self, level, sigma, u, f, singular):
        if level == len(self.levels) - 1:
            return self.coarse_solve(sigma, f, singular)
        for _ in range(self.nu1):
            u = self.sweep(level, sigma, u, f)
        rc = self.restrict(level, self.residual(level, sigma, u, f))
        ec = self.vcycle(level + 1, sigma, np.zeros(self.levels[level + 1].n), rc, singular)
        u = u + self.prolong(level, ec)
        for _ in range(self.nu2):
            u = self.sweep(level, sigma, u, f)
        return u

    def solve(self, sigma, f, singular=False, rtol=1e-13, max_cycles=100):
        """V-cycles from a zero guess until ||f - A u|| <= rtol ||f||, or until the residual stops
        falling (the FP64 floor). Returns (u, cycles, final relative residual)."""
        u = np.zeros_like(f)
        nf = np.linalg.norm(f)
        if nf == 0.0:
            return u, 0, 0.0
        prev = nf
        rel = 1.0
        for c in range(1, max_cycles + 1):
            u = self.vcycle(0, sigma, u, f, singular)
            rn = np.linalg.norm(self.residual(0, sigma, u, f))
            rel = rn / nf
            if rel <= rtol or (c >= 3 and rn > 0.7 * prev):
                return u, c, rel
            prev = rn
        return u, max_cycles, rel
