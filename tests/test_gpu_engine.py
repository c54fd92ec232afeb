"""The serving engine (include/snac_engine.h) through the C ABI: each request's solution is the same
alone and in a concurrent mix, admission respects the device-memory budget, plans are reused, and a
failed request does not disturb the others."""
import numpy as np
import pytest

from oracle import solve as osv
from paper_2106_03583_gb300 import inputs, snac

from gpu_util import dev, ensure_built, host, rel
from layouts import make

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _mix():
    """Problems of different layouts, boundary pairs, sizes and precisions (some repeated)."""
    out = []
    specs = [("2x2", 16, 8, "NN", ("N", "N", "N", "N"), "mixed"),
             ("L", 16, 16, "DD", ("N", "D", "D", "N"), "fp64"),
             ("1", 32, 8, "PP", ("D", "D", "N", "N"), "mixed"),
             ("1x2", 16, 12, "ND", ("D", "N", "N", "N"), "fp64"),
             ("2x1", 12, 10, "DN", ("N", "N", "D", "D"), "mixed"),
             ("2x2", 16, 8, "NN", ("N", "N", "N", "N"), "mixed"),   # same problem as the first
             ("1", 24, 16, "PP", ("N", "N", "N", "N"), "fp64"),
             ("L", 16, 16, "DD", ("N", "D", "D", "N"), "fp64")]     # same problem as the second
    for k, (layout, n, nz, zp, walls, prec) in enumerate(specs):
        blocks = make(layout, n=n, nz=nz, zpair=zp, walls=walls, stretched=True)
        f = inputs.divergence_rhs(blocks, 10 + k)
        out.append((blocks, f, prec))
    return out


def _alone(blocks, f, prec):
    import torch
    ensure_built()
    pl = snac.Plan(blocks, precision=prec)
    p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
    info = pl.solve(dev(f), p, tol=TOL)
    pl.close()
    return host(p), info


def test_same_alone_and_in_the_mix():
    mix = _mix()
    alone = [_alone(*m) for m in mix]
    ensure_built()
    with snac.Engine(workers=4, hbm_budget=8e9) as eng:
        tickets = [eng.submit(b, f, tol=TOL, precision=prec) for b, f, prec in mix]
        results = [eng.wait(t) for t in tickets]
        st = eng.stats()
    for (p_alone, info_alone), (p, info, times) in zip(alone, results):
        assert info["status"] == 0 and info["rel_res"] <= TOL
        assert info["rel_res"] == info_alone["rel_res"]
        assert np.array_equal(p, p_alone)             # identical, not merely close
        assert times["t_submit"] <= times["t_admit"] <= times["t_start"] <= times["t_done"]
    # repeated problems reused a resident plan once it was idle, or got their own while it was busy
    assert st["plans_built"] <= len(mix) and st["completed"] == len(mix)
    assert st["bytes_peak"] <= 8e9
    # and the mix agrees with the oracle
    for k in (0, 3):
        b, f, _ = mix[k]
        po, _ = osv.solve(b, f)
        assert rel(results[k][0], po) <= 1e-9


def test_budget_admission_and_eviction():
    """A budget that holds about one request at a time: requests wait, idle plans are evicted, the
    accounted peak stays within the budget and every result is still the alone result."""
    mix = _mix()[:5]
    alone = [_alone(*m) for m in mix]
    biggest = max(len(f) for _, f, _ in mix)
    budget = 16 * biggest + 64 * biggest + (64 << 20) + 1   # one request's buffers + one FP64 plan estimate
    with snac.Engine(workers=3, hbm_budget=budget, max_cached_plans=8) as eng:
        tickets = [eng.submit(b, f, tol=TOL, precision=prec) for b, f, prec in mix]
        results = [eng.wait(t) for t in tickets]
        st = eng.stats()
    assert st["bytes_peak"] <= budget
    assert st["plans_evicted"] >= 1
    for (p_alone, _), (p, info, _) in zip(alone, results):
        assert info["status"] == 0 and np.array_equal(p, p_alone)


def test_plan_reuse_and_errors():
    blocks = make("2x2", n=8, nz=8, zpair="NN", walls=("N", "N", "N", "N"))
    f = inputs.uniform_rhs(blocks, 1, remove_mean=True)
    with snac.Engine(workers=2, hbm_budget=4e9) as eng:
        _, i1, t1 = eng.wait(eng.submit(blocks, f, tol=TOL))
        _, i2, t2 = eng.wait(eng.submit(blocks, f, tol=TOL))
        assert t1["plan_reused"] == 0 and t2["plan_reused"] == 1
        # a singular problem with an incompatible right-hand side fails alone; the engine serves on
        bad = eng.submit(blocks, f + 1.0, tol=TOL)
        good = eng.submit(blocks, f, tol=TOL)
        with pytest.raises(snac.SnacError) as e:
            eng.wait(bad)
        assert e.value.name == "INCOMPATIBLE_RHS"
        p, info, _ = eng.wait(good)
        assert info["status"] == 0 and info["rel_res"] <= TOL
        # a request larger than the whole budget is refused at submission
    with snac.Engine(workers=1, hbm_budget=1 << 20) as small:
        with pytest.raises(snac.SnacError) as e:
            small.submit(blocks, f, tol=TOL)
        assert e.value.name == "OOM"
        with pytest.raises(snac.SnacError) as e:
            small.wait(12345)
        assert e.value.name == "INVALID_ARG"


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_picks_a_converging_schedule(precision):
    """snac_autotune times candidate schedules on the problem itself; the chosen one is no slower
    than the starting options and solves to the tolerance."""
    import torch
    ensure_built()
    blocks = make("2x2", n=32, nz=16, zpair="NN", walls=("N", "N", "N", "N"), stretched=True)
    f = inputs.divergence_rhs(blocks, 2)
    chosen, rep = snac.autotune(blocks, dev(f), tol=TOL, precision=precision)
    assert rep["trials"] >= 6 and rep["best_ms"] <= rep["base_ms"]
    pl = snac.Plan(blocks, **chosen)
    p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
    info = pl.solve(dev(f), p, tol=TOL)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    po, _ = osv.solve(blocks, f)
    assert rel(host(p), po) <= 1e-9


def test_engine_autotune_once_per_problem():
    blocks = make("L", n=16, nz=8, zpair="DD", walls=("N", "D", "D", "N"), stretched=True)
    f = inputs.divergence_rhs(blocks, 3)
    po, _ = osv.solve(blocks, f)
    with snac.Engine(workers=2, hbm_budget=4e9, autotune=True) as eng:
        res = [eng.wait(eng.submit(blocks, f, tol=TOL, precision="mixed")) for _ in range(3)]
    (p1, i1, t1), (p2, i2, t2), (p3, i3, t3) = res
    assert t1["tuned"] == 1 and t2["tuned"] == 0 and t3["tuned"] == 0
    assert t2["plan_reused"] == 1 and t3["plan_reused"] == 1
    assert np.array_equal(p2, p3)                 # the same tuned plan, the same result
    for p, info in ((p1, i1), (p2, i2)):
        assert info["status"] == 0 and info["rel_res"] <= TOL and rel(p, po) <= 1e-9


def test_concurrent_plans_with_different_transform_lengths():
    """Plans whose transforms have different lengths share the same transform kernels; their
    launches interleave on the engine's streams. Every request must still succeed (the kernels'
    shared-memory limit is a function-wide attribute, never lowered by a shorter plan)."""
    probs = []
    for nz, seed in ((8, 1), (512, 2)):
        blocks = make("1", n=8, nz=nz, zpair="NN", walls=("D", "D", "N", "N"))
        probs.append((blocks, inputs.uniform_rhs(blocks, seed, remove_mean=False)))
    fails = []
    with snac.Engine(workers=4, hbm_budget=8e9) as eng:
        tickets = [eng.submit(*probs[k % 2], tol=TOL, precision="mixed" if k % 4 < 2 else "fp64") for k in range(400)]
        for k, t in enumerate(tickets):
            _, info, times = eng.wait(t, raise_on_error=False)
            if info["status"] != 0:
                fails.append((k, info["status_name"], times["error"]))
    assert not fails, fails[:5]


def test_small_requests_merge_into_batched_solves():
    """Requests of resident on-chip plans that are ready together are solved as one batched solve
    (continuous batching). Each result is still the alone result, bitwise; a failing request in a
    group fails alone; requests whose plans are not on chip never join a group."""
    import torch
    ensure_built()
    specs = [("2x2", 16, 8, "NN", ("N", "N", "N", "N"), "mixed"),
             ("L", 16, 16, "DD", ("N", "D", "D", "N"), "fp64"),
             ("1", 32, 8, "PP", ("D", "D", "N", "N"), "mixed"),
             ("1x2", 16, 12, "ND", ("D", "N", "N", "N"), "fp64"),
             ("2x1", 12, 10, "DN", ("N", "N", "D", "D"), "mixed"),
             ("1", 24, 16, "PP", ("N", "N", "N", "N"), "fp64"),
             ("1", 16, 8, "DD", ("D", "N", "D", "N"), "mixed"),
             ("2x2", 8, 6, "PP", ("D", "D", "D", "D"), "fp64")]
    mix = []
    for k, (layout, n, nz, zp, walls, prec) in enumerate(specs):
        blocks = make(layout, n=n, nz=nz, zpair=zp, walls=walls, stretched=True)
        mix.append((blocks, inputs.divergence_rhs(blocks, 40 + k), prec, True))
    level = make("1", n=16, nz=8, zpair="DD", walls=("D", "D", "N", "N"), stretched=True)
    mix.append((level, inputs.divergence_rhs(level, 60), "mixed", False))     # level-by-level plan
    alone = []
    for blocks, f, prec, oc in mix:
        pl = snac.Plan(blocks, precision=prec, onchip=oc)
        p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
        pl.solve(dev(f), p, tol=TOL)
        ks = pl.kernel_stats()
        assert (ks["onchip"]["launches"] + ks["fwd_onchip"]["launches"] > 0) == oc
        alone.append(host(p))
        pl.close()
    # a singular problem of its own (periodic z, Neumann walls): a compatible f caches its plan, an
    # incompatible one fails inside a group
    sing = make("1", n=20, nz=8, zpair="PP", walls=("N", "N", "N", "N"), stretched=True)
    f_sing = inputs.divergence_rhs(sing, 61)
    with snac.Engine(workers=1, hbm_budget=8e9, max_group=16) as eng:
        for blocks, f, prec, oc in mix + [(sing, f_sing, "mixed", True)]:   # build and cache every plan
            eng.wait(eng.submit(blocks, f, tol=TOL, precision=prec, onchip=oc))
        for _ in range(3):
            tickets = [eng.submit(b, f, tol=TOL, precision=prec, onchip=oc) for b, f, prec, oc in mix]
            tickets.append(eng.submit(sing, f_sing + 1.0, tol=TOL, precision="mixed"))
            res = [eng.wait(t, raise_on_error=False) for t in tickets]
            if res[-1][2]["group"] > 1:
                break
    groups = [t["group"] for _, _, t in res]
    assert res[-1][2]["group"] > 1, groups                   # the failing request ran in a group
    assert res[-1][1]["status_name"] == "INCOMPATIBLE_RHS"
    assert res[len(mix) - 1][2]["group"] == 1                 # the level-by-level plan ran alone
    for p_alone, (p, info, times) in zip(alone, res):
        assert info["status"] == 0 and info["rel_res"] <= TOL, (info, times)
        assert np.array_equal(p, p_alone)
        assert times["plan_reused"] == 1
