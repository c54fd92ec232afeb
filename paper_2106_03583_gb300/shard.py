"""One Poisson solve sharded by wavenumber over several GPUs (App. A, Algorithm 3).

The reduced equations (Eq. 9) of different wavenumbers are independent, so a single problem spreads
over G ranks with one exchange each way per defect-correction step -- the paper's pencil <-> slab
redistribution:

* pencils: the x-y cells of the problem (the level-0 plane numbering: blocks in id order, [y][x]
  within a block) are split into G contiguous ranges by the paper's balanced split rule (the first
  n % G ranks take one cell more, Sec. 3.1); rank r holds its columns with every z plane, [z][c];
* slabs: the wavenumbers q = 0 .. n_z - 1 are split into G contiguous ranges, by that same rule on
  their count, or balanced by a predicted cost per wavenumber (App. B: the cycle count falls as |lambda_q|
  grows, so equal counts are not equal work);
* per step (one rank): outer FP64 residual of its pencil (the neighbouring columns of other ranks
  come in by a halo exchange), forward transform of its columns, all-to-all pencil -> slab, the
  reduced equations of its slab on a wavenumber-range plan, the mean fix of a singular problem on
  the rank holding q = 0, all-to-all slab -> pencil, backward transform and update of its columns.

Every numerical step runs in the stage object passed in (``GpuStages``: the library's CUDA kernels
through its C ABI); this module only partitions, packs, exchanges and unpacks. The exchanges are
grouped point-to-point transfers of torch.distributed (``TorchExchange``: NCCL between GPUs, gloo on
CPU), staged in buffers of the rank's own memory.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["d5_split", "ranges", "column_ranges", "mode_ranges", "predicted_mode_costs", "TorchExchange",
           "GpuStages", "ShardedSolver"]


def d5_split(n: int, m: int) -> list:
    """Counts of n points over m parts: the first n % m parts take n // m + 1 (Sec. 3.1)."""
    if m < 1 or n < 0:
        raise ValueError("need m >= 1 and n >= 0")
    return [n // m + (1 if k < n % m else 0) for k in range(m)]


def ranges(counts) -> list:
    """Contiguous [begin, end) ranges of the given counts."""
    out, b = [], 0
    for c in counts:
        out.append((b, b + c))
        b += c
    return out


def column_ranges(ncell: int, world: int) -> list:
    """The pencil of every rank: contiguous ranges of the plane's cells (balanced split rule)."""
    if ncell < world:
        raise ValueError("fewer plane cells than ranks")
    return ranges(d5_split(ncell, world))


def mode_ranges(nz: int, world: int, costs=None) -> list:
    """The slab of every rank: contiguous ranges of the wavenumbers. Without costs, the balanced
    split rule on their count; with a cost per wavenumber, cut where the running sum of the costs
    crosses k/world of the total (every rank keeps at least one wavenumber)."""
    if nz < world:
        raise ValueError("fewer wavenumbers than ranks")
    if costs is None:
        return ranges(d5_split(nz, world))
    c = np.asarray(costs, dtype=np.float64)
    if c.shape != (nz,) or not np.all(np.isfinite(c)) or np.any(c < 0):
        raise ValueError("costs must be n_z finite non-negative values")
    cum = np.concatenate([[0.0], np.cumsum(c)])
    cuts = [0]
    for k in range(1, world):
        want = cum[-1] * k / world
        q = int(np.searchsorted(cum, want))           # first q with cum[q] >= want
        if q > 0 and abs(cum[q - 1] - want) <= abs(cum[q] - want):
            q -= 1                                      # the nearer cut
        q = min(max(q, cuts[-1] + 1), nz - (world - k))
        cuts.append(q)
    cuts.append(nz)
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def _kind(blocks) -> str:
    lo, hi = blocks[0]["bc"][2]
    return "PP" if lo == "P" else lo + hi


def _lambda(kind: str, n: int, q: np.ndarray) -> np.ndarray:
    """Eigenvalue of the z operator for wavenumber slot q (Table 1), lambda_q = 2 (cos(kappa dl) - 1)."""
    m = {"PP": q, "NN": q / 2.0, "DD": (q + 1.0) / 2.0, "ND": (2.0 * q + 1.0) / 4.0,
         "DN": (2.0 * q + 1.0) / 4.0}[kind]
    return 2.0 * (np.cos(2.0 * np.pi * m / n) - 1.0)


def predicted_mode_costs(blocks, tol: float = 1e-10, rho0: float = 0.15) -> np.ndarray:
    """Predicted V-cycles per wavenumber (App. B: fewer cycles as |lambda_q| grows). Model: the
    cycle's contraction for mode q falls from rho0 by the diagonal dominance the shift adds,
    rho_q = rho0 / (1 + |sigma_q| / d), sigma_q = lambda_q / dz^2 and d the mean magnitude of the x-y
    operator's diagonal; cycles = log(tol) / log(rho_q). A cost model to balance slabs, not a bound."""
    nz = int(blocks[0]["hi"][2] - blocks[0]["lo"][2] + 1)
    dz = float(np.asarray(blocks[0]["dx"][2])[0])
    d, n = 0.0, 0
    for b in blocks:
        wx = np.asarray(b["dx"][0], dtype=np.float64)
        wy = np.asarray(b["dx"][1], dtype=np.float64)
        d += (2.0 / wx ** 2).sum() * len(wy) + (2.0 / wy ** 2).sum() * len(wx)
        n += len(wx) * len(wy)
    d /= n
    sigma = np.abs(_lambda(_kind(blocks), nz, np.arange(nz, dtype=np.float64))) / dz ** 2
    rho = rho0 / (1.0 + sigma / d)
    return np.maximum(1.0, np.ceil(np.log(tol) / np.log(rho)))


class TorchExchange:
    """The exchanges of a sharded solve over torch.distributed: grouped point-to-point transfers
    (one group per all-to-all; NCCL runs it as one grouped call, gloo pairwise) and a sum."""

    def __init__(self, group=None):
        import torch.distributed as td
        self.td = td
        self.group = group
        self.rank = td.get_rank(group)
        self.world = td.get_world_size(group)

    def alltoallv(self, send: list, recv: list) -> None:
        """send[s] goes to rank s, recv[r] comes from rank r (contiguous tensors; empty ones skipped)."""
        td = self.td
        ops = []
        for peer in range(self.world):
            if peer == self.rank:
                if recv[peer].numel():
                    recv[peer].copy_(send[peer])
                continue
            if send[peer].numel():
                ops.append(td.P2POp(td.isend, send[peer], peer, self.group))
            if recv[peer].numel():
                ops.append(td.P2POp(td.irecv, recv[peer], peer, self.group))
        if ops:
            for w in td.batch_isend_irecv(ops):
                w.wait()

    def allreduce(self, t) -> None:
        self.td.all_reduce(t, op=self.td.ReduceOp.SUM, group=self.group)


class GpuStages:
    """The numerical steps of one rank on its GPU: the library's kernels through its C ABI. The plan
    is a wavenumber-range plan holding this rank's slab (the pencil calls accept it too)."""

    def __init__(self, blocks, q0: int, q1: int, precision: str = "fp64", **plan_options):
        import torch
        from . import snac
        self.torch = torch
        self.plan = snac.Plan(blocks, precision=precision, modes=(q0, q1), **plan_options)
        self.nz, self.ncell = self.plan.nz, self.plan.ncell
        self.device = self.plan.device
        self.inner = self.plan.inner_dtype
        self.ncols = 0

    def zeros(self, shape, inner: bool = False):
        return self.torch.zeros(shape, dtype=self.inner if inner else self.torch.float64, device=self.device)

    def setup(self, c0: int, ncols: int) -> np.ndarray:
        self.ncols = ncols
        return self.plan.pencil_setup(c0, ncols)

    def residual(self, f, p_ext, r, fshift: float):
        return self.plan.pencil_residual(f, p_ext, r, fshift)

    def forward(self, x, modes):
        self.plan.pencil_forward(x, modes)

    def mode_solve(self, rhs, sol, target: float) -> int:
        info = self.plan.mode_solve(rhs, sol, target)
        return info["total_cycles"]

    def fix_mean(self, sol, sum_vp: float):
        self.plan.mode_fix_mean(sol, sum_vp)

    def backward_update(self, modes, p):
        self.plan.pencil_backward_update(modes, p)

    def sync(self):
        self.torch.cuda.current_stream(self.device).synchronize()

    def close(self):
        self.plan.close()


class ShardedSolver:
    """One rank of a solve sharded by wavenumber (App. A, Algorithm 3). ``stages`` computes,
    ``exchange`` moves data between ranks; this class partitions, packs and unpacks.

        ex = TorchExchange()
        cols = column_ranges(ncell, world); modes = mode_ranges(nz, world, predicted_mode_costs(blocks))
        st = GpuStages(blocks, *modes[rank], precision="mixed")
        sv = ShardedSolver(blocks, st, ex, cols, modes)
        info = sv.solve(f_pencil, p_pencil, tol=1e-10)     # [z][c] tensors of this rank's columns
    """

    def __init__(self, blocks, stages, exchange, cols=None, modes=None, inner_reduction: float = 1e-4,
                 max_outer: int = 20):
        self.blocks = blocks
        self.st = stages
        self.ex = exchange
        self.rank, self.world = exchange.rank, exchange.world
        self.nz = int(blocks[0]["hi"][2] - blocks[0]["lo"][2] + 1)
        self.ncell = int(sum((b["hi"][0] - b["lo"][0] + 1) * (b["hi"][1] - b["lo"][1] + 1) for b in blocks))
        self.cols = cols or column_ranges(self.ncell, self.world)
        self.modes = modes or mode_ranges(self.nz, self.world)
        if len(self.cols) != self.world or len(self.modes) != self.world:
            raise ValueError("one column range and one wavenumber range per rank")
        self.c0, self.c1 = self.cols[self.rank]
        self.q0, self.q1 = self.modes[self.rank]
        self.nc, self.nq = self.c1 - self.c0, self.q1 - self.q0
        self.inner_reduction = inner_reduction
        self.max_outer = max_outer
        kind = _kind(blocks)
        walls = [k for b in blocks for a in range(2) for k in b["bc"][a]]
        self.singular = kind in ("PP", "NN") and "D" not in walls
        vol = 0.0
        for b in blocks:
            vol += float(np.sum(b["dx"][0])) * float(np.sum(b["dx"][1])) * float(np.sum(b["dx"][2]))
        self.vol_total = vol
        # the halo: the columns of other ranks that this pencil's stencil reaches, ascending; since
        # the pencils are contiguous ranges, the part owned by each rank is a contiguous slice
        self.halo = stages.setup(self.c0, self.nc)
        owners = np.searchsorted(np.array([c1 for _, c1 in self.cols]), self.halo, side="right")
        self.halo_from = [np.nonzero(owners == s)[0] for s in range(self.world)]
        # tell every owner which of its columns this rank needs (counts, then the cell lists)
        import torch
        self.torch = torch
        need_n = [torch.tensor([len(ix)], dtype=torch.int64) for ix in self.halo_from]
        give_n = [torch.zeros(1, dtype=torch.int64) for _ in range(self.world)]
        self._exchange_cpu(need_n, give_n)
        need = [torch.from_numpy(self.halo[ix].astype(np.int64)) for ix in self.halo_from]
        give = [torch.zeros(int(n.item()), dtype=torch.int64) for n in give_n]
        self._exchange_cpu(need, give)
        # local column indices (in this rank's pencil) that each rank needs from it
        self.give_cols = [torch.as_tensor(g.numpy() - self.c0, dtype=torch.int64, device=self._device())
                          for g in give]
        self.nhalo = len(self.halo)

    def _device(self):
        return getattr(self.st, "device", "cpu")

    def _exchange_cpu(self, send, recv):
        """Small host-side exchanges of the setup (moved to the stages' device for the transfer)."""
        dev = self._device()
        s = [t.to(dev) for t in send]
        r = [t.to(dev) for t in recv]
        self.ex.alltoallv(s, r)
        for a, b in zip(recv, r):
            a.copy_(b.cpu())

    def _sum(self, values):
        t = self.torch.tensor(values, dtype=self.torch.float64, device=self._device())
        self.ex.allreduce(t)
        return t.cpu().numpy()

    # ---- exchanges ----
    def halo_exchange(self, p, p_ext):
        """p_ext [z][nc + nhalo] = this pencil's p, then the halo columns from their owners."""
        torch = self.torch
        p_ext[:, :self.nc].copy_(p.view(self.nz, self.nc))
        send = [p.view(self.nz, self.nc).index_select(1, g).contiguous() for g in self.give_cols]
        recv = [torch.empty((self.nz, len(ix)), dtype=p.dtype, device=p.device) for ix in self.halo_from]
        self.ex.alltoallv(send, recv)
        for ix, buf in zip(self.halo_from, recv):
            if len(ix):
                p_ext[:, self.nc + int(ix[0]):self.nc + int(ix[-1]) + 1].copy_(buf)

    def pencil_to_slab(self, modes, slab):
        """modes [n_z][nc] of this pencil -> slab [nq][ncell] of this rank's wavenumbers."""
        torch = self.torch
        m = modes.view(self.nz, self.nc)
        send = [m[a:b] for a, b in self.modes]                     # contiguous rows
        recv = [torch.empty((self.nq, c1 - c0), dtype=modes.dtype, device=modes.device) for c0, c1 in self.cols]
        self.ex.alltoallv(send, recv)
        sl = slab.view(self.nq, self.ncell)
        for (c0, c1), buf in zip(self.cols, recv):
            sl[:, c0:c1].copy_(buf)

    def slab_to_pencil(self, slab, modes):
        """slab [nq][ncell] -> modes [n_z][nc] of this pencil."""
        sl = slab.view(self.nq, self.ncell)
        m = modes.view(self.nz, self.nc)
        send = [sl[:, c0:c1].contiguous() for c0, c1 in self.cols]
        recv = [m[a:b] for a, b in self.modes]                     # contiguous rows
        self.ex.alltoallv(send, recv)

    # ---- the solve ----
    def solve(self, f, p, tol: float = 1e-10, mixed: bool = False) -> dict:
        """Solve A p = f to ||f - A p|| <= tol ||f|| over all ranks. f, p: this rank's pencil [z][nc]
        (p: initial guess in, solution out). Returns the solve's statistics (the same on every rank)."""
        st, nz, nc = self.st, self.nz, self.nc
        p_ext = st.zeros((nz, nc + self.nhalo))
        r = st.zeros((nz, nc))
        modes = st.zeros((nz, nc), inner=True)
        slab_rhs = st.zeros((self.nq, self.ncell), inner=True)
        slab_sol = st.zeros((self.nq, self.ncell), inner=True)
        self.halo_exchange(p, p_ext)
        sums = self._sum(list(st.residual(f, p_ext, r, 0.0)))
        fshift = 0.0
        if self.singular:
            if abs(sums[3]) > 1e-12 * sums[4]:
                raise ValueError("singular problem: the volume-weighted sum of the right-hand side is not zero")
            fshift = sums[3] / self.vol_total
            if fshift != 0.0:
                sums = self._sum(list(st.residual(f, p_ext, r, fshift)))
        fn = math.sqrt(sums[1])
        info = {"status": 0, "outer_iters": 0, "cycles": 0, "removed_mean": fshift}
        if fn == 0.0:
            p.zero_()
            info["rel_res"] = 0.0
            return info
        prev = math.inf
        for k in range(self.max_outer + 1):
            rn = math.sqrt(sums[0])
            rel = rn / fn
            info.update(outer_iters=k, rel_res=rel)
            if not math.isfinite(rel):
                info["status"] = -6
                return info
            if rel <= tol:
                return info
            if k == self.max_outer or rel >= prev:
                info["status"] = -5
                return info
            prev = rel
            target = 0.5 * tol * fn
            if mixed:
                target = max(target, self.inner_reduction * rn)
            st.forward(r, modes)                                   # Algorithm 3, first loop
            self.pencil_to_slab(modes, slab_rhs)                   # pencil -> slab
            info["cycles"] += int(self._sum([st.mode_solve(slab_rhs, slab_sol, target)])[0])
            if self.singular:
                st.fix_mean(slab_sol, float(sums[2]))              # on the rank holding q = 0
            self.slab_to_pencil(slab_sol, modes)                   # slab -> pencil
            st.backward_update(modes, p)                           # Algorithm 3, last loop
            self.halo_exchange(p, p_ext)
            sums = self._sum(list(st.residual(f, p_ext, r, fshift)))
        return info
