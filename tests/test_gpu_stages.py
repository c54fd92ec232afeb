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
@pytest.mark.parametrize("nz", [2, 4, 6, 8, 34, 64, 90, 150, 194, 256, 512, 576, 1024, 2048, 4096])
def test_transforms(precision, tol, zpair, nz):
    """Every even length: half-lengths with factors 2 and 4 (Stockham radix 4/2), 3 and 5 (90: 45 =
    3^2 5, 150: 75 = 3 5^2, 576: 288 = 2^5 3^2) and a prime (194: 97), up to 4096 (fewer columns per
    CTA beyond 1024)."""
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


FUSED_CASES = [
    ("2x2", 32, 8, "NN", ("N", "N", "N", "N"), True),      # fused levels 0..2 (blocks 32, 16, 8)
    ("L", 24, 6, "DD", ("N", "D", "D", "N"), True),        # ragged 24x24 tiles, re-entrant corner
    ("1", 40, 4, "ND", ("D", "N", "N", "N"), True),        # 80x80: ragged 64+16 tiles, four fused levels
    ("2x2", 24, 8, "PP", ("N", "N", "N", "N"), True, (True, True)),   # periodic wrap across blocks
    ("1x2", 20, 10, "DN", ("D", "D", "N", "N"), False),   # 20x40 blocks
]


def _two_cycles(blocks, Fh, U0, precision, fused, nu=(2, 2)):
    pl = plan(blocks, precision=precision, max_coarse=64, fused=fused, nu1=nu[0], nu2=nu[1])
    u = dev(U0.ravel(), pl.inner_dtype)
    pl.mode_vcycles(dev(Fh.ravel(), pl.inner_dtype), u, 2)
    got = host(u).reshape(U0.shape)
    pl.close()
    return got


def _oracle_two_cycles(g, mg, Fh, U0):
    lam = T.eigenvalues(g.kind, g.nz)
    ref = np.empty_like(U0)
    for q in range(g.nz):
        u = U0[q]
        sing = g.singular and lam[q] == 0.0
        for _ in range(2):
            u = mg.vcycle(0, lam[q] / g.dz ** 2, u, Fh[q], sing)
        ref[q] = u
    return ref


def _mean_free(g, X):
    lam = T.eigenvalues(g.kind, g.nz)
    X = X.copy()
    for q in range(g.nz):
        if g.singular and lam[q] == 0.0:   # the null-space component is free
            X[q] -= np.dot(g.plane.area, X[q]) / g.plane.area.sum()
    return X


@pytest.mark.parametrize("case", FUSED_CASES)
def test_vcycle_fused_matches_oracle(case):
    """The fused tile kernels (levels whose blocks are >= 8 wide; each tile reads one iterate
    buffer and writes the other) reproduce the oracle's V(2,2) cycles: to rounding when run in FP64
    from a random iterate, and in FP32 from a zero iterate as accurately as the per-colour FP32
    kernels do (the FP32 error itself grows with the conditioning of the low modes)."""
    blocks = _blocks(case)
    g = ogrid.Grid(blocks)
    mg = omg.Multigrid(g.plane, 2, 2, max_coarse=64)
    lam = T.eigenvalues(g.kind, g.nz)
    rng = np.random.default_rng(6)
    Fh = rng.standard_normal((g.nz, g.plane.n))
    for q in range(g.nz):
        if g.singular and lam[q] == 0.0:
            Fh[q] -= np.dot(g.plane.area, Fh[q]) / g.plane.area.sum()
    U0 = rng.standard_normal((g.nz, g.plane.n))
    ref = _mean_free(g, _oracle_two_cycles(g, mg, Fh, U0))
    got = _mean_free(g, _two_cycles(blocks, Fh, U0, "fp64", 1))
    assert rel(got, ref) <= 1e-11
    Z = np.zeros_like(U0)
    ref0 = _mean_free(g, _oracle_two_cycles(g, mg, Fh, Z))
    err_fused = rel(_mean_free(g, _two_cycles(blocks, Fh, Z, "mixed", 1)), ref0)
    err_colour = rel(_mean_free(g, _two_cycles(blocks, Fh, Z, "mixed", 0)), ref0)
    assert err_colour <= 2e-4
    assert err_fused <= max(2e-5, 4.0 * err_colour), (err_fused, err_colour)


@pytest.mark.parametrize("nu", [(1, 1), (2, 1), (1, 2)])
@pytest.mark.parametrize("case", FUSED_CASES[:3])
def test_vcycle_fused_other_schedules(case, nu):
    """The fused kernels with the other sweep counts the autotuner may choose: exact (FP64, 1e-11)
    against the oracle's V(nu1, nu2) cycles, and in FP32 as accurate as the per-colour kernels."""
    blocks = _blocks(case)
    g = ogrid.Grid(blocks)
    mg = omg.Multigrid(g.plane, nu[0], nu[1], max_coarse=64)
    lam = T.eigenvalues(g.kind, g.nz)
    rng = np.random.default_rng(7)
    Fh = rng.standard_normal((g.nz, g.plane.n))
    for q in range(g.nz):
        if g.singular and lam[q] == 0.0:
            Fh[q] -= np.dot(g.plane.area, Fh[q]) / g.plane.area.sum()
    U0 = rng.standard_normal((g.nz, g.plane.n))
    ref = _mean_free(g, _oracle_two_cycles(g, mg, Fh, U0))
    assert rel(_mean_free(g, _two_cycles(blocks, Fh, U0, "fp64", 1, nu)), ref) <= 1e-11
    Z = np.zeros_like(U0)
    ref0 = _mean_free(g, _oracle_two_cycles(g, mg, Fh, Z))
    err_fused = rel(_mean_free(g, _two_cycles(blocks, Fh, Z, "mixed", 1, nu)), ref0)
    err_colour = rel(_mean_free(g, _two_cycles(blocks, Fh, Z, "mixed", 0, nu)), ref0)
    assert err_fused <= max(2e-5, 4.0 * err_colour), (err_fused, err_colour)


def _abs_operator(g, p):
    """|A| |p| with the oracle's assembled 3-D operator (the scale of the cancellation in f - A p)."""
    A = g.matrix().tocsr()
    A.data = np.abs(A.data)
    return g.from_planes((A @ np.abs(g.to_planes(p)).ravel()).reshape(g.nz, g.plane.n))


def _check_ff(pl, g, f, p, norms=True):
    """The float-float residual against the oracle's FP64 residual, cell by cell, within the bound
    2^-24 |r| (rounding to FP32) + 16 * 2^-47 (|f| + |A||p|) + |A| 2^-103 (operands below 2^-103
    count as zero); the norms against the sums of the same values."""
    import torch
    N = len(f)
    r = torch.empty(N, dtype=torch.float32, device="cuda")
    r2, f2 = pl.residual_ff(dev(f), dev(p), r)
    ref = f - g.from_planes(g.apply(g.to_planes(p)))
    got = host(r)
    bound = 2.0 ** -24 * np.abs(ref) + 16 * 2.0 ** -47 * (np.abs(f) + _abs_operator(g, p)) + \
        _abs_operator(g, np.ones(N)) * 2.0 ** -103
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / bound))
    if norms:
        assert r2 == pytest.approx(float(np.sum(got.astype(np.float64) ** 2)), rel=1e-5)
        assert f2 == pytest.approx(float(np.sum(f ** 2)), rel=1e-5)
    return got, ref


@pytest.mark.parametrize("case", CASES + PERIODIC)
def test_float_float_residual_random(case):
    """Random f and p of unit size on every layout and z pair (no cancellation: the bound is the
    FP32 rounding of r)."""
    blocks = _blocks(case)
    N = inputs.total_cells(blocks)
    rng = np.random.default_rng(5)
    _check_ff(plan(blocks, precision="mixed"), ogrid.Grid(blocks), rng.standard_normal(N), rng.standard_normal(N))


@pytest.mark.parametrize("name,scale", [("mb2x2", 4), ("chan", 8), ("c64", 2)])
def test_float_float_residual_near_the_solution(name, scale):
    """p within 1e-9 of the solution, where A p cancels f to nine digits and more: the residual is
    resolved far below |A||p| (the float-float bound), and its norm matches the FP64 residual's."""
    from oracle import solve as osv
    blocks, f = inputs.config(name, seed=2, scale=scale)
    ps, _ = osv.solve(blocks, f)
    rng = np.random.default_rng(6)
    p = ps * (1.0 + 1e-9 * rng.standard_normal(len(ps)))
    g = ogrid.Grid(blocks)
    got, ref = _check_ff(plan(blocks, precision="mixed"), g, f, p)
    assert np.linalg.norm(ref) <= 1e-6 * np.linalg.norm(_abs_operator(g, p))  # the cancellation is real
    assert rel(got, ref) <= 1e-3


def test_float_float_residual_special_operands():
    """Zeros, negative zeros, operands below 2^-103 (taken as zero), all-ones mantissas, large values,
    and a NaN (which must reach the norm). Values of 1e30 stay within the elementwise bound, but their
    squares overflow the FP32 sums of this stage call (which has no scaling), so the norms are
    checked with values of 1e12."""
    import torch
    blocks = _blocks(CASES[1])
    N = inputs.total_cells(blocks)
    rng = np.random.default_rng(7)
    p = rng.standard_normal(N)
    p[::7] = 0.0
    p[1::7] = -0.0
    p[2::7] = 1e-200
    p[3::7] = -3e-33
    p[4::7] = np.nextafter(2.0, 0.0) * np.sign(rng.standard_normal(len(p[4::7])))
    p[5::7] = 1e30 * rng.standard_normal(len(p[5::7]))
    f = rng.standard_normal(N)
    f[::5] = 0.0
    pl = plan(blocks, precision="mixed")
    g = ogrid.Grid(blocks)
    _check_ff(pl, g, f, p, norms=False)
    p[5::7] = 1e12 * rng.standard_normal(len(p[5::7]))
    _check_ff(pl, g, f, p)
    p[10] = np.nan
    r = torch.empty(N, dtype=torch.float32, device="cuda")
    r2, _ = pl.residual_ff(dev(f), dev(p), r)
    assert not np.isfinite(r2)


def test_mixed_solve_runs_float_float_passes_and_decides_in_fp64():
    """A mixed solve from zero: the intermediate residual passes are the float-float kernel, the
    convergence check an FP64 pass; the result still meets the tolerance under the oracle's operator."""
    import torch
    from oracle import solve as osv
    blocks, f = inputs.config("chan", seed=1, scale=8)
    pl = plan(blocks, precision="mixed")
    p = torch.zeros(len(f), dtype=torch.float64, device="cuda")
    pl.reset_stats()
    info = pl.solve(dev(f), p, tol=1e-10)
    st = pl.kernel_stats()
    assert info["status"] == 0 and info["outer_iters"] >= 2
    assert st["field3d_ff"]["launches"] >= 1
    assert st["field3d"]["launches"] >= 2          # the pre-pass and at least one FP64 check
    assert osv.rel_residual(blocks, f, host(p)) <= 1.01e-10


@pytest.mark.parametrize("zpair", ["PP", "NN"])
def test_fp32_transforms_of_extreme_values(zpair):
    """The FP32 transforms convert between FP64 and FP32 with integer operations (round to nearest
    even; exact the other way): zeros, signs, values across the FP32 range and values above it (which
    must come out infinite, not garbage) in the 3-D field and in the modes."""
    import torch
    nz = 16
    blocks = make("1x2", n=8, nz=nz, zpair=zpair, walls=("N", "N", "N", "N"))
    N = inputs.total_cells(blocks)
    g = ogrid.Grid(blocks)
    rng = np.random.default_rng(9)
    mags = 10.0 ** rng.uniform(-30, 30, N)
    x = np.where(rng.random(N) < 0.5, -1.0, 1.0) * mags
    x[::11] = 0.0
    x[1::11] = -0.0
    pl = plan(blocks, precision="mixed")
    modes = torch.empty(N, dtype=torch.float32, device="cuda")
    pl.forward_transform(dev(x), modes)
    got = host(modes).reshape(nz, -1)
    ref = T.forward(g.kind, g.to_planes(x.astype(np.float32).astype(np.float64)))
    # column by column, relative to the column's largest input (FP32 transform accuracy)
    scale = np.abs(g.to_planes(x)).max(axis=0) * nz
    assert np.all(np.abs(got - ref) <= 1e-5 * scale + 1e-37)
    # beyond the FP32 range: an infinity or NaN reaches the modes, nothing finite and wrong
    x[5] = 1e300
    pl.forward_transform(dev(x), modes)
    col = int(np.argmax(np.abs(g.to_planes(x)).max(axis=0) >= 1e300))
    assert not np.all(np.isfinite(host(modes).reshape(nz, -1)[:, col]))
    # backward: modes of all sizes into an FP64 field, exactly converted before the update
    X = (np.where(rng.random(N) < 0.5, -1.0, 1.0) * 10.0 ** rng.uniform(-30, 30, N)).astype(np.float32)
    X[::7] = 0.0
    p = torch.zeros(N, dtype=torch.float64, device="cuda")
    pl.backward_update(dev(X.astype(np.float64), torch.float32), p)
    upd = g.from_planes(T.backward(g.kind, X.astype(np.float64).reshape(nz, -1)))
    scale_b = g.from_planes(np.broadcast_to(np.abs(X.astype(np.float64).reshape(nz, -1)).max(axis=0), (nz, g.plane.n)))
    assert np.all(np.abs(host(p) - upd) <= 1e-5 * scale_b + 1e-37)
