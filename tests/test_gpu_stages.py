"""Stage-by-stage parity of the CUDA library with the oracle, through the C ABI.

Tolerances: FP64 stages agree with the oracle up to rounding (1e-13 relative for the operator and
the residual, 1e-12 for transforms of length up to 1024, 1e-11 for one V-cycle, whose smoother uses a
Newton-refined reciprocal of the diagonal). FP32 stages (mixed plans) agree to 2e-6 relative."""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import mg as omg
from oracle import transforms as T
from paper_2106_03583_gb300 import inputs

from gpu_util import dev, host, plan, rel
from layouts import make

pytestmark = pytest.mark.gpu

CASES = [
    ("1", 8, 8, "PP", ("D", "D", "N", "N"), False),
    ("2x2", 8, 16, "NN", ("N", "N", "N", "N"), True),
    ("L", 8, 6, "DD", ("N", "D", "D", "N"), True),
    ("1x2", 12, 10, "ND", ("D", "N", "N", "N"), True),
    ("2x1", 6, 34, "DN", ("N", "N", "D", "D"), True),
]
PERIODIC = [("2x2", 8, 8, "PP", ("N", "N", "N", "N"), True, (True, False))]


def _blocks(case):
    layout, n, nz, zp, walls, st = case[:6]
    per = case[6] if len(case) > 6 else (False, False)
    return make(layout, n=n, nz=nz, zpair=zp, walls=walls, stretched=st, periodic=per)


@pytest.mark.parametrize("case", CASES + PERIODIC)
def test_operator_and_residual(case):
    import torch
    blocks = _blocks(case)
    N = inputs.total_cells(blocks)
    rng = np.random.default_rng(1)
    p, f = rng.standard_normal(N), rng.standard_normal(N)
    pl = plan(blocks)
    out = torch.empty(N, dtype=torch.float64, device="cuda")
    pl.apply_operator(dev(p), out)
    g = ogrid.Grid(blocks)
    ref = g.from_planes(g.apply(g.to_planes(p)))
    assert rel(host(out), ref) <= 1e-13
    r = torch.empty_like(out)
    r2, f2 = pl.residual(dev(f), dev(p), r)
    assert rel(host(r), f - ref) <= 1e-13
    assert abs(r2 - np.sum((f - ref) ** 2)) <= 1e-12 * r2
    assert abs(f2 - np.sum(f ** 2)) <= 1e-12 * f2


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-6)])
@pytest.mark.parametrize("zpair", ["PP", "NN", "DD", "ND", "DN"])
@pytest.mark.parametrize("nz", [2, 4, 6, 8, 34, 64, 256, 512, 1024])
def test_transforms(precision, tol, zpair, nz):
    import torch
    n = 4 if nz >= 256 else 8
    blocks = make("1x2", n=n, nz=nz, zpair=zpair, walls=("N", "N", "N", "N"))
    N = inputs.total_cells(blocks)
    g = ogrid.Grid(blocks)
    x = np.random.default_rng(nz).standard_normal(N)
    pl = plan(blocks, precision=precision)
    modes = torch.empty(N, dtype=pl.inner_dtype, device="cuda")
    pl.forward_transform(dev(x), modes)
    ref = T.forward(g.kind, g.to_planes(x))
    assert rel(host(modes).reshape(nz, -1), ref) <= tol
    # backward: p += F^-1 X
    X = np.random.default_rng(nz + 1).standard_normal(N)
    p0 = np.random.default_rng(nz + 2).standard_normal(N)
    p = dev(p0)
    pl.backward_update(dev(X, pl.inner_dtype), p)
    upd = g.from_planes(T.backward(g.kind, X.reshape(nz, -1)))
    assert rel(host(p) - p0, upd) <= tol


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("mixed", 2e-6)])
@pytest.mark.parametrize("case", CASES + PERIODIC)
def test_mode_operator(precision, tol, case):
    import torch
    blocks = _blocks(case)
    N = inputs.total_cells(blocks)
    g = ogrid.Grid(blocks)
    mg = omg.Multigrid(g.plane)
    lam = T.eigenvalues(g.kind, g.nz) / g.dz ** 2
    U = np.random.default_rng(3).standard_normal((g.nz, g.plane.n))
    pl = plan(blocks, precision=precision)
    out = torch.empty(N, dtype=pl.inner_dtype, device="cuda")
    pl.mode_operator(dev(U.ravel(), pl.inner_dtype), out)
    ref = np.stack([mg.operator(0, lam[q], U[q]) for q in range(g.nz)])
    assert rel(host(out).reshape(g.nz, -1), ref) <= tol


@pytest.mark.parametrize("case", CASES + PERIODIC + [("2x2", 16, 8, "NN", ("N", "N", "N", "N"), True)])
def test_vcycle_matches_oracle(case):
    """Two V(2,2) cycles of every wavenumber from a random iterate equal the oracle's cycles."""
    blocks = _blocks(case)
    g = ogrid.Grid(blocks)
    mg = omg.Multigrid(g.plane, 2, 2, max_coarse=64)
    lam = T.eigenvalues(g.kind, g.nz)
    rng = np.random.default_rng(5)
    Fh = rng.standard_normal((g.nz, g.plane.n))
    U0 = rng.standard_normal((g.nz, g.plane.n))
    ref = np.empty_like(U0)
    for q in range(g.nz):
        u = U0[q]
        sing = g.singular and lam[q] == 0.0
        if sing:      # singular modes: a compatible right-hand side
            Fh[q] -= np.dot(g.plane.area, Fh[q]) / g.plane.area.sum()
        for _ in range(2):
            u = mg.vcycle(0, lam[q] / g.dz ** 2, u, Fh[q], sing)
        ref[q] = u
    pl = plan(blocks, precision="fp64", max_coarse=64)
    assert pl.info()["levels"] == len(mg.levels)
    u = dev(U0.ravel())
    pl.mode_vcycles(dev(Fh.ravel()), u, 2)
    got = host(u).reshape(g.nz, -1)
    for q in range(g.nz):
        if g.singular and lam[q] == 0.0:   # the null-space component is free: compare mean-free parts
            a = g.plane.area
            got[q] -= np.dot(a, got[q]) / a.sum()
            ref[q] -= np.dot(a, ref[q]) / a.sum()
    assert rel(got, ref) <= 1e-11
