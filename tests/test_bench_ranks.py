"""The multi-rank path of bench.py on CPU: two gloo ranks (127.0.0.1), as torchrun would start them.

Every rank solves its own seeded problem (independent replicas, no collective on the data path); the
job's time is the slowest rank's, and the whole-job rate counts every rank's solves. The reference
arm runs on rank 0 only; the other ranks exit without output."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as td
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist()
        times = [12.5, 20.0]                      # this rank's timed region, ms
        mx = bench.max_over_ranks(times[r], w, "cpu")
        rate = bench.whole_job_rate(w, 10, mx)
        td.barrier()
        out.put((r, w, mx, rate, bench.rank_seed(7, r)))
    finally:
        td.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_torchrun():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for r, w, mx, rate, seed in res:
        assert w == 2
        assert mx == 20.0                          # the slowest rank's time on every rank
        assert rate == pytest.approx(2 * 10 / 0.020)
    assert [s for *_, s in res] == [7, 8]           # each rank its own problem


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(bench.argparse.Namespace(workload="c64", seed=0, steps=1, warmup=1))
    assert buf.getvalue() == ""


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(1, 4, 1000.0) == pytest.approx(4.0)


def test_reference_arm_line_has_the_gpu_arms_config(capsys):
    """The reference arm (the CPU oracle on bounded samples) prints one line on the same config dict,
    metric and unit as the GPU arm, with its step time and the oracle's cpu_baseline record."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_03583_gb300 import inputs
    args = bench.argparse.Namespace(workload="c64", seed=0, steps=2, warmup=1, tol=1e-10, precisions="mixed,fp64")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    blocks, _ = inputs.config("c64", seed=0)
    assert line["config"] == bench.workload_config("c64", blocks, 1e-10, "mixed", 1)
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_reports_single_thread_and_all_cores():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2106_03583_gb300 import inputs
    blocks, f = inputs.config("c64", seed=0)
    cb = bench.cpu_baseline(blocks, f)
    assert cb["kind"] == "oracle" and cb["single_thread"]["cores"] == 1
    assert cb["cores"] == cb["all_cores"]["cores"] >= 1 and cb["value"] == cb["all_cores"]["value"] > 0
    assert cb["single_thread"]["value"] > 0
