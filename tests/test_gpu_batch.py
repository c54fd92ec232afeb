"""Whole-wavenumber solves on chip and many problems in one batch (snac_poisson_solve_batch).

* A plan whose multigrid hierarchy fits in one CTA's shared memory solves each wavenumber in one
  CTA, V-cycling until the mode's own stopping rule holds, decided on the device: one launch per
  defect-correction step. Its solution must match the oracle's (1e-9 at rel. residual 1e-10) and
  the level-by-level path's.
* snac_poisson_solve_batch runs several problems in lock-step, the on-chip wavenumber solves of all
  of them in one persistent launch per precision. Every result must be bitwise identical to the
  same plan solving the same problem alone (the batch changes the schedule, not the arithmetic)."""
import numpy as np
import pytest

from oracle import solve as osv
from paper_2106_03583_gb300 import inputs, snac

from gpu_util import dev, host, plan, rel
from layouts import make

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["c64", "mb2x2_8", "L_dn"])
def test_onchip_solve_matches_oracle_and_level_path(name, precision):
    import torch
    if name == "c64":
        blocks, f = inputs.config("c64", seed=1)
    elif name == "mb2x2_8":
        blocks, f = inputs.config("mb2x2", seed=1, scale=8)
    else:
        blocks = make("L", n=24, nz=12, zpair="DN", walls=("D", "N", "N", "D"), stretched=True)
        f = inputs.uniform_rhs(blocks, 4, remove_mean=False)
    ref, _ = osv.solve(blocks, f)
    sols = {}
    for onchip in (True, False):
        pl = plan(blocks, precision=precision, onchip=onchip)
        p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
        pl.reset_stats()
        info = pl.solve(dev(f), p, tol=1e-10)
        st = pl.kernel_stats()
        assert info["status"] == 0 and info["rel_res"] <= 1e-10
        if onchip:
            # one launch per defect-correction step (forward transform and on-chip solves together),
            # no level-by-level cycle and no separate forward transform
            assert st["fwd_onchip"]["launches"] == info["outer_iters"] >= 1
            assert st["forward_transform"]["launches"] == 0
            assert st["smooth"]["launches"] == 0 and st["fused_up"]["launches"] == 0
        else:
            assert st["fwd_onchip"]["launches"] == 0 and st["onchip"]["launches"] == 0
        sols[onchip] = host(p)
        assert osv.rel_residual(blocks, f, sols[onchip]) <= 1.01e-10
        assert rel(sols[onchip], ref) <= 1e-9
        pl.close()
    assert rel(sols[True], sols[False]) <= 2e-9


def _batch_problems():
    probs = [inputs.config("c64", seed=3), inputs.config("mb2x2", seed=3, scale=8)]
    b = make("1x2", n=16, nz=8, zpair="PP", walls=("N", "N", "D", "N"), stretched=True)
    probs.append((b, inputs.uniform_rhs(b, 7, remove_mean=False)))
    b = make("2x2", n=24, nz=6, zpair="NN", walls=("N", "N", "N", "N"), stretched=True)
    probs.append((b, inputs.uniform_rhs(b, 8, remove_mean=True)))
    probs.append(inputs.config("mb2x2", seed=3, scale=4))     # 128x128 plane: too large for on chip
    return probs


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_each_problem_alone(precision):
    import torch
    probs = _batch_problems()
    plans = [plan(b, precision=precision) for b, _ in probs]
    fs = [dev(f) for _, f in probs]
    alone = []
    for pl, f in zip(plans, fs):
        p = torch.zeros_like(f)
        info = pl.solve(f, p, tol=1e-10)
        alone.append((host(p), info))
    ps = [torch.zeros_like(f) for f in fs]
    for pl in plans:
        pl.reset_stats()
    infos = snac.solve_batch(plans, fs, ps, tol=1e-10)
    for (b, f), pl, p, info, (pa, ia) in zip(probs, plans, ps, infos, alone):
        assert info["status"] == 0 and info["rel_res"] <= 1e-10
        assert np.array_equal(host(p), pa)                       # bitwise: same arithmetic
        assert info["outer_iters"] == ia["outer_iters"] and info["total_cycles"] == ia["total_cycles"]
        assert osv.rel_residual(b, f, host(p)) <= 1.01e-10
    # the on-chip plans' transforms and wavenumber solves shared one launch per step
    onchip = [pl for pl in plans if pl.kernel_stats()["fwd_onchip"]["launches"]]
    assert len(onchip) >= 3
    for pl in plans:
        pl.close()


def test_batch_reports_each_problems_status():
    """An incompatible right-hand side fails its own problem only; the others still converge."""
    import torch
    probs = _batch_problems()[:3]
    blocks, f = inputs.config("mb2x2", seed=3, scale=8)         # singular: a mean makes it incompatible
    probs.append((blocks, f + 1.0))
    plans = [plan(b) for b, _ in probs]
    fs = [dev(f) for _, f in probs]
    ps = [torch.zeros_like(f) for f in fs]
    infos = snac.solve_batch(plans, fs, ps, tol=1e-10, raise_on_error=False)
    assert [i["status_name"] for i in infos] == ["OK", "OK", "OK", "INCOMPATIBLE_RHS"]
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bounded_wait_gives_up_and_the_context_stays_usable(precision):
    """The on-chip solves wait on the device for their plan's transform chunks. The self-test makes
    that wait impossible (one chunk more than the launch has): every wait must give up after the
    limit and the call return TIMEOUT without trapping; the same plan then solves normally."""
    import time
    import torch
    blocks, f = inputs.config("c64", seed=5)
    pl = plan(blocks, precision=precision)
    t0 = time.time()
    assert pl.test_wait_timeout(0.05) == "TIMEOUT"
    assert time.time() - t0 < 10.0
    p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
    info = pl.solve(dev(f), p, tol=1e-10)
    assert info["status"] == 0
    ref, _ = osv.solve(blocks, f)
    assert rel(host(p), ref) <= 1e-9
    pl.close()
    lvl = plan(blocks, precision=precision, onchip=False)   # level by level: no on-chip wait to test
    assert lvl.test_wait_timeout(0.05) == "INVALID_ARG"
    lvl.close()
