"""The oracle's per-wavenumber solves (Algorithm 1, second loop) spread over host processes.

Test infrastructure: the full-size parity tests need the oracle's solution of problems with 2.7e8
cells, whose 2-D multigrid solves take seconds each. The pool uses the ``spawn`` start method (a
process forked after CUDA has been initialised must not touch the GPU runtime), and each worker
builds the oracle's hierarchy once."""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_mg = None


def _init(blocks, nu1, nu2):
    global _mg
    from oracle import grid as ogrid
    from oracle import mg as omg
    _mg = omg.Multigrid(ogrid.Grid(blocks).plane, nu1, nu2)


def _solve_mode(task):
    q, sigma, fq, singular, rtol = task
    u, cycles, res = _mg.solve(sigma, fq, singular=singular, rtol=rtol)
    return q, u, cycles, res


def oracle_solve(blocks, f, rtol_mode=1e-13, nu1=2, nu2=2, workers=None, modes=None):
    """The oracle's solve (as ``oracle.solve.solve``) with the per-wavenumber solves in a pool.

    Returns (p in the caller layout, per-mode planes Ph, info). info holds the per-mode cycle counts
    and relative residuals and, for a full solve, the 3-D relative residual ||f - A p|| / ||f|| of the
    oracle's own solution (the acceptance number of its solve). With ``modes`` only those
    wavenumbers are solved (Ph is zero elsewhere and p is not formed)."""
    from oracle import grid as ogrid
    from oracle import solve as osv
    from oracle import transforms as T
    g = ogrid.Grid(blocks)
    F = g.to_planes(f)
    mean = 0.0
    if g.singular:
        mean = osv._compatibility(g, F)
        F = F - mean
    Fh = T.forward(g.kind, F)
    del F
    lam = T.eigenvalues(g.kind, g.nz)
    todo = list(range(g.nz)) if modes is None else list(modes)
    tasks = [(q, lam[q] / (g.dz * g.dz), Fh[q], bool(g.singular and lam[q] == 0.0), rtol_mode) for q in todo]
    workers = workers or min(16, os.cpu_count() or 1, len(tasks))
    Ph = np.zeros_like(Fh)
    cycles = np.zeros(g.nz, dtype=np.int64)
    mode_res = np.zeros(g.nz)
    ctx = mp.get_context("spawn")
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"   # one BLAS thread per worker process
    try:
        with ctx.Pool(workers, initializer=_init, initargs=(blocks, nu1, nu2)) as pool:
            for q, u, c, res in pool.imap_unordered(_solve_mode, tasks, chunksize=1):
                Ph[q] = u
                cycles[q] = c
                mode_res[q] = res
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    info = {"removed_mean": mean, "cycles": cycles, "mode_rel_res": mode_res, "singular": g.singular}
    if modes is not None:
        return None, Ph, info
    P = T.backward(g.kind, Ph)
    if g.singular:
        P = P - float((g.vol * P).sum()) / float(g.vol.sum())
    p = g.from_planes(P)
    del P
    info["rel_res"] = osv.rel_residual(blocks, f, p)
    return p, Ph, info
