"""The wavenumber-sharded solve with the library's kernels (GpuStages: pencil transforms, pencil
residual, wavenumber-range plans), ranks emulated as threads of one process on one GPU
(tests/shard_stages.ThreadExchange: the host hands data between ranks after synchronising each
rank's stream, so no kernel ever waits on another rank's kernel). The assembled solution must match
the oracle's solve of the whole problem within 1e-9 at relative residual 1e-10, FP64 and mixed."""
import threading

import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import solve as osv
from paper_2106_03583_gb300 import inputs, shard

from gpu_util import ensure_built, rel
from layouts import make
from shard_stages import ThreadExchange

pytestmark = pytest.mark.gpu


def _problem(name):
    if name == "mb2x2":
        return inputs.config("mb2x2", seed=5, scale=8)
    if name == "chan":
        return inputs.config("chan", seed=5, scale=8)
    blocks = make("L", n=16, nz=10, zpair="DN", walls=("D", "N", "N", "N"), stretched=True)
    return blocks, inputs.uniform_rhs(blocks, 3, remove_mean=False)


def _run_ranks(blocks, f, world, precision, costs):
    import torch
    ensure_built()
    g = ogrid.Grid(blocks)
    F = g.to_planes(f)
    cols = shard.column_ranges(g.plane.n, world)
    modes = shard.mode_ranges(g.nz, world, shard.predicted_mode_costs(blocks) if costs else None)
    hub = ThreadExchange.Hub(world)
    out, errors = [None] * world, []

    def run(rank):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                st = shard.GpuStages(blocks, *modes[rank], precision=precision)
                ex = ThreadExchange(hub, rank, sync=s.synchronize)
                sv = shard.ShardedSolver(blocks, st, ex, cols, modes)
                c0, c1 = cols[rank]
                fp = torch.from_numpy(np.ascontiguousarray(F[:, c0:c1])).cuda()
                p = torch.zeros_like(fp)
                info = sv.solve(fp, p, tol=1e-10, mixed=precision == "mixed")
                s.synchronize()
                out[rank] = (c0, c1, p.cpu().numpy(), info)
                st.close()
        except BaseException as e:  # report, and release the other ranks
            errors.append(e)
            hub.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in th:
        t.start()
    for t in th:
        t.join(timeout=300)
    if errors:
        raise errors[0]
    P = np.zeros((g.nz, g.plane.n))
    for c0, c1, pp, info in out:
        assert info["status"] == 0 and info["rel_res"] <= 1e-10, info
        P[:, c0:c1] = pp
    return g.from_planes(P), out[0][3]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,world,costs", [("mb2x2", 2, True), ("chan", 3, False), ("L", 2, False)])
def test_sharded_gpu_solve_matches_the_oracle(name, world, costs, precision):
    blocks, f = _problem(name)
    p, info = _run_ranks(blocks, f, world, precision, costs)
    ref, _ = osv.solve(blocks, f)
    assert osv.rel_residual(blocks, f, p) <= 1.01e-10
    assert rel(p, ref) <= 1e-9
    g = ogrid.Grid(blocks)
    if g.singular:
        vol = g.from_planes(g.vol)
        assert abs(np.dot(vol, p)) <= 1e-12 * np.dot(vol, np.abs(p))


def test_one_rank_sharded_solve_equals_the_plain_solve():
    """With one rank the pencil is the whole plane and the slab every wavenumber: the stages are the
    plain solve's kernels, so the result matches the plain solve to rounding."""
    import torch
    from gpu_util import dev, host, plan
    blocks, f = _problem("mb2x2")
    p1, _ = _run_ranks(blocks, f, 1, "fp64", False)
    pl = plan(blocks)
    p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
    pl.solve(dev(f), p, tol=1e-10)
    assert rel(p1, host(p)) <= 1e-11


def test_range_plan_holds_only_its_wavenumbers():
    """A wavenumber-range plan refuses the 3-D calls; its mode solve of a slab equals the slab of
    the full plan's mode solve (same kernels, same per-mode stopping rule)."""
    import torch
    from gpu_util import dev, plan
    from paper_2106_03583_gb300 import snac
    blocks, f = _problem("mb2x2")
    full = plan(blocks)
    part = plan(blocks, modes=(5, 17))
    n3 = len(f)
    with pytest.raises(snac.SnacError) as e:
        part.solve(dev(f), torch.zeros(n3, dtype=torch.float64, device="cuda"))
    assert e.value.name == "INVALID_ARG"
    g = ogrid.Grid(blocks)
    rhs = torch.from_numpy(np.random.default_rng(2).standard_normal((g.nz, g.plane.n))).cuda()
    sol_full = torch.empty_like(rhs)
    full.mode_solve(rhs, sol_full, target=1e-6)
    sol_part = torch.empty((12, g.plane.n), dtype=torch.float64, device="cuda")
    part.mode_solve(rhs[5:17].contiguous(), sol_part, target=1e-6)
    assert rel(sol_part.cpu().numpy(), sol_full[5:17].cpu().numpy()) <= 1e-13
    assert list(part.mode_cycles()) == list(full.mode_cycles()[5:17])
