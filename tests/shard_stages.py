"""Test infrastructure for the wavenumber-sharded solve (paper_2106_03583_gb300.shard).

* ``OracleStages``: the numerical steps of one rank computed by the CPU oracle, standing in for the
  library's kernels, so that the product's partitioning, packing and exchanges can run on gloo ranks
  without a GPU: the oracle's O(n^2) transforms of the pencil's columns, its multigrid solves of the
  slab's wavenumbers (each to 1e-13), its operator for the pencil residual, and the zero-mean shift
  of a singular problem written out from its definition.
* ``ThreadExchange``: ranks as threads of one process (host-side barriers; every rank's stream is
  synchronised before its data is handed over), for running the GPU stages of several ranks on one
  GPU without any kernel waiting on another rank's kernel."""
from __future__ import annotations

import threading

import numpy as np
import torch

from oracle import grid as ogrid
from oracle import mg as omg
from oracle import transforms as T


class OracleStages:
    device = "cpu"

    def __init__(self, blocks, q0: int, q1: int):
        self.g = ogrid.Grid(blocks)
        self.q0, self.q1 = q0, q1
        self.mg = omg.Multigrid(self.g.plane)
        self.lam = T.eigenvalues(self.g.kind, self.g.nz)

    def zeros(self, shape, inner: bool = False):
        return torch.zeros(shape, dtype=torch.float64)

    def setup(self, c0: int, ncols: int) -> np.ndarray:
        self.c0, self.c1 = c0, c0 + ncols
        nb = self.g.plane.nbr[:, :, c0:c0 + ncols].ravel()
        out = nb[(nb >= 0) & ((nb < c0) | (nb >= c0 + ncols))]
        self.halo = np.unique(out)
        return self.halo

    def residual(self, f, p_ext, r, fshift: float):
        g, c0, c1 = self.g, self.c0, self.c1
        P = np.zeros((g.nz, g.plane.n))
        pe = p_ext.numpy()
        P[:, c0:c1] = pe[:, :c1 - c0]
        P[:, self.halo] = pe[:, c1 - c0:]
        fv = f.numpy() - fshift
        rv = fv - g.apply(P)[:, c0:c1]
        r.copy_(torch.from_numpy(rv))
        vol = g.vol[:, c0:c1]
        return (float(np.sum(rv * rv)), float(np.sum(fv * fv)), float(np.sum(vol * P[:, c0:c1])),
                float(np.sum(vol * fv)), float(np.sum(vol * np.abs(fv))))

    def forward(self, x, modes):
        modes.copy_(torch.from_numpy(T.forward(self.g.kind, x.numpy())))

    def mode_solve(self, rhs, sol, target: float) -> int:
        g, cyc = self.g, 0
        for l, q in enumerate(range(self.q0, self.q1)):
            sigma = self.lam[q] / (g.dz * g.dz) + g.shift
            u, c, _ = self.mg.solve(sigma, rhs[l].numpy(), singular=bool(g.singular and self.lam[q] == 0.0),
                                    rtol=1e-13)
            sol[l].copy_(torch.from_numpy(u))
            cyc += int(c)
        return cyc

    def fix_mean(self, sol, sum_vp: float):
        """The updated p = p + F^-1(e) adds (dz n / theta) sum_xy area e_0 to sum V p (only wavenumber
        0 has a non-zero sum over z); shift e_0 by the constant that makes the new sum zero."""
        g = self.g
        if not g.singular or self.q0 != 0:
            return
        alpha = g.dz * g.nz / T.theta(g.kind, g.nz)
        area = g.plane.area
        e0 = sol[0].numpy()
        kappa = -(sum_vp + alpha * float(np.dot(area, e0))) / (alpha * float(area.sum()))
        sol[0].add_(kappa)

    def backward_update(self, modes, p):
        p.add_(torch.from_numpy(T.backward(self.g.kind, modes.numpy())))

    def sync(self):
        pass


class ThreadExchange:
    """All-to-all and sum between ranks that are threads of this process (shared state + barriers)."""

    class Hub:
        def __init__(self, world: int):
            self.world = world
            self.barrier = threading.Barrier(world)
            self.slots = {}

    def __init__(self, hub: "ThreadExchange.Hub", rank: int, sync=None):
        self.hub, self.rank, self.world = hub, rank, hub.world
        self.sync = sync or (lambda: None)

    def alltoallv(self, send: list, recv: list) -> None:
        self.sync()                                   # this rank's data is complete on its device
        for s in range(self.world):
            self.hub.slots[(self.rank, s)] = send[s]
        self.hub.barrier.wait()
        for r in range(self.world):
            if recv[r].numel():
                recv[r].copy_(self.hub.slots[(r, self.rank)])
        self.sync()
        self.hub.barrier.wait()                       # every rank has taken its parts

    def allreduce(self, t) -> None:
        self.sync()
        self.hub.slots[("sum", self.rank)] = t.clone()
        self.hub.barrier.wait()
        tot = sum(self.hub.slots[("sum", r)].to(t.device) for r in range(self.world))
        self.hub.barrier.wait()
        t.copy_(tot)
