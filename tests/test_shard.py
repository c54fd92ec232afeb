"""The wavenumber-sharded solve (App. A, Algorithm 3) on CPU ranks: gloo process groups at
127.0.0.1, as torchrun starts them.

Each rank runs the product's partitioning, halo and pencil <-> slab exchanges and the defect-
correction loop (paper_2106_03583_gb300.shard), with the CPU oracle's transforms, multigrid solves
and operator standing in for the CUDA kernels (tests/shard_stages.py). The assembled solution must
equal the oracle's single-rank solve of the whole problem to 1e-13: the sharding moves data and
nothing else. Also: the balanced split rule, and slabs balanced by predicted cost."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(name):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from paper_2106_03583_gb300 import inputs
    from layouts import make
    if name == "mb2x2":
        return inputs.config("mb2x2", seed=4, scale=16)          # 2x2 blocks of 16x16, NN z, singular
    if name == "L":
        blocks = make("L", n=8, nz=12, zpair="DD", walls=("D", "N", "N", "D"), stretched=True)
    else:                                                         # periodic x-wrap across two blocks
        blocks = make("2x2", n=8, nz=8, zpair="PP", walls=("N", "N", "N", "N"), stretched=True,
                      periodic=(True, False))
    from oracle import grid as ogrid
    g = ogrid.Grid(blocks)
    return blocks, inputs.uniform_rhs(blocks, 9, remove_mean=g.singular)


def _rank(rank, world, port, name, costs, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as td
    from oracle import grid as ogrid
    from paper_2106_03583_gb300 import shard
    from shard_stages import OracleStages
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        blocks, f = _problem(name)
        g = ogrid.Grid(blocks)
        F = g.to_planes(f)
        cols = shard.column_ranges(g.plane.n, world)
        modes = shard.mode_ranges(g.nz, world, shard.predicted_mode_costs(blocks) if costs else None)
        sv = shard.ShardedSolver(blocks, OracleStages(blocks, *modes[rank]), shard.TorchExchange(), cols, modes)
        c0, c1 = cols[rank]
        p = torch.zeros((g.nz, c1 - c0), dtype=torch.float64)
        info = sv.solve(torch.from_numpy(np.ascontiguousarray(F[:, c0:c1])), p, tol=1e-12)
        q.put((rank, c0, c1, p.numpy(), info, modes, len(sv.halo)))
    finally:
        td.destroy_process_group()


@pytest.mark.parametrize("name,world,costs", [("mb2x2", 2, False), ("mb2x2", 3, True), ("L", 2, True),
                                              ("periodic", 3, False)])
def test_sharded_solve_equals_the_single_rank_oracle(name, world, costs):
    import torch.multiprocessing as mp
    from oracle import grid as ogrid
    from oracle import solve as osv
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, name, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    blocks, f = _problem(name)
    g = ogrid.Grid(blocks)
    P = np.zeros((g.nz, g.plane.n))
    for rank, c0, c1, pp, info, modes, nh in res:
        assert info["status"] == 0 and info["rel_res"] <= 1e-12, info
        assert nh > 0                                   # the pencils really need each other's columns
        P[:, c0:c1] = pp
    assert [m for m in res[0][5]] == [tuple(m) for m in res[-1][5]]
    ref, _ = osv.solve(blocks, f)
    got = g.from_planes(P)
    assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
    if g.singular:
        assert abs(float((g.vol * P).sum())) <= 1e-12 * float((g.vol * np.abs(P)).sum())


def test_split_rules():
    sys.path.insert(0, ROOT)
    from paper_2106_03583_gb300 import shard
    assert shard.d5_split(10, 3) == [4, 3, 3]
    assert shard.d5_split(9, 3) == [3, 3, 3]
    assert shard.column_ranges(11, 4) == [(0, 3), (3, 6), (6, 9), (9, 11)]
    assert shard.mode_ranges(8, 3) == [(0, 3), (3, 6), (6, 8)]
    # costs falling with q (App. B): equal counts give unequal work; the cost split evens it out
    costs = np.array([40, 30, 20, 10, 6, 5, 4, 3, 3, 3, 3, 3], dtype=float)
    by_count = shard.mode_ranges(12, 3)
    by_cost = shard.mode_ranges(12, 3, costs)
    spread = lambda rs: max(costs[a:b].sum() for a, b in rs) / costs.sum()
    assert spread(by_cost) < spread(by_count)
    assert by_cost[0][0] == 0 and by_cost[-1][1] == 12 and all(b > a for a, b in by_cost)
    assert all(by_cost[k][1] == by_cost[k + 1][0] for k in range(2))
    with pytest.raises(ValueError):
        shard.mode_ranges(2, 3)


def test_predicted_costs_fall_with_the_eigenvalue():
    sys.path.insert(0, ROOT)
    from paper_2106_03583_gb300 import inputs, shard
    blocks, _ = inputs.config("mb2x2", seed=0, scale=8)      # NN: |lambda_q| grows with q
    c = shard.predicted_mode_costs(blocks)
    assert c[0] >= c[-1] and np.all(np.diff(c) <= 0) and c.min() >= 1
