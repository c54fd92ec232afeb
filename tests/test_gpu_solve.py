"""End-to-end parity of the CUDA solve with the oracle, through the C ABI.

The bar: at relative residual 1e-10 the GPU solution matches the oracle's (solved to 1e-13 per
wavenumber) within 1e-9 relative L2, for FP64 and mixed-precision plans. The residual is re-checked
with the oracle's own operator."""
import numpy as np
import pytest

from oracle import grid as ogrid
from oracle import solve as osv
from paper_2106_03583_gb300 import inputs, snac

from gpu_util import dev, host, plan, rel
from layouts import homogeneous_along, make

pytestmark = pytest.mark.gpu

TOL = 1e-10
PARITY = 1e-9


def gpu_solve(blocks, f, precision="fp64", tol=TOL, p0=None, **kw):
    import torch
    pl = plan(blocks, precision=precision, **kw)
    p = dev(p0) if p0 is not None else torch.zeros(len(f), dtype=torch.float64, device="cuda")
    info = pl.solve(dev(f), p, tol=tol)
    return host(p), info, pl


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("layout", ["1", "1x2", "L", "2x2"])
@pytest.mark.parametrize("zpair", ["PP", "NN", "DD", "ND", "DN"])
@pytest.mark.parametrize("walls", [("D", "D", "N", "N"), ("N", "N", "N", "N")])
def test_tiny_grids_vs_dense_lu(precision, layout, zpair, walls):
    blocks = make(layout, n=4, nz=6, zpair=zpair, walls=walls, stretched=True)
    g = ogrid.Grid(blocks)
    f = inputs.uniform_rhs(blocks, 21, remove_mean=g.singular)
    pd = osv.solve_dense(blocks, f)
    p, info, _ = gpu_solve(blocks, f, precision)
    assert info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, p) <= 1.01 * TOL
    assert rel(p, pd) <= PARITY


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,scale", [("c64", 1), ("mb2x2", 4), ("chan", 4), ("chan", 8)])
def test_workloads_vs_oracle(precision, name, scale):
    """The three workload shapes (ragged-free but multi-level, multi-block, stretched)."""
    blocks, f = inputs.config(name, seed=0, scale=scale)
    po, oinfo = osv.solve(blocks, f)
    p, info, pl = gpu_solve(blocks, f, precision)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, p) <= 1.01 * TOL
    assert rel(p, po) <= PARITY, (rel(p, po), info)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("bottom_cells", [512, 2048, -1])
def test_bottom_start_vs_oracle(precision, bottom_cells):
    """Where the bottom sub-cycle starts (an autotuner dimension) changes only the launch shape: the
    solution still matches the oracle, and -1 (no sub-cycle: every level level by level and the
    dense coarsest solve) runs no bottom launch."""
    blocks, f = inputs.config("mb2x2", seed=0, scale=4)
    po, _ = osv.solve(blocks, f)
    p, info, pl = gpu_solve(blocks, f, precision, bottom_cells=bottom_cells)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, p) <= 1.01 * TOL
    assert rel(p, po) <= PARITY, (rel(p, po), info)
    if bottom_cells == -1:
        assert pl.kernel_stats()["bottom"]["launches"] == 0


def _table2_blocks(refine, nz, z_bc):
    """The four-block layout of Table 2 (its index-space corners, from the golden fixture), refined."""
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "table2_blocks.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                c = [t.split() for t in line.split("|")]
                rows.append((tuple(map(int, c[1])), tuple(map(int, c[2]))))
    x0, y0 = min(lo[0] for lo, _ in rows), min(lo[1] for lo, _ in rows)
    rects = [((lo[0] - x0) * refine, (hi[0] - x0 + 1) * refine, (lo[1] - y0) * refine, (hi[1] - y0 + 1) * refine)
             for lo, hi in rows]
    NX, NY = max(r[1] for r in rects), max(r[3] for r in rects)
    return inputs.make_blocks(inputs.tanh_faces(NX, 0, 1.0, 0.0, 4.0), inputs.tanh_faces(NY, 0, 1.0, 0.0, 2.0),
                              np.linspace(0.0, 0.1 * nz / 2, nz + 1), rects,
                              {"x-": "D", "x+": "N", "y-": "N", "y+": "N"}, z_bc)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("z_bc", [("N", "N"), ("P", "P")])
def test_table2_layout_vs_oracle(precision, z_bc):
    """The paper's four-block T-shaped example (Table 2, Fig. 1) refined 4x (blocks 80x40 and three
    40x40, n_z = 16): fused levels across the T junction, a coarsest level with odd block sizes."""
    blocks = _table2_blocks(4, 16, z_bc)
    f = inputs.divergence_rhs(blocks, 4)
    po, _ = osv.solve(blocks, f)
    p, info, _ = gpu_solve(blocks, f, precision)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, p) <= 1.01 * TOL
    assert rel(p, po) <= PARITY


def test_ragged_tiles_and_periodic_xy():
    """Blocks whose sizes are not multiples of the 32x8 tile, periodic in x and y (singular)."""
    xf = inputs.tanh_faces(40, 0, 1.2, 0.0, 1.0)
    yf = inputs.tanh_faces(24, 1, 0.8, 0.0, 1.0)
    zf = np.linspace(0, 1, 11)
    blocks = inputs.make_blocks(xf, yf, zf, [(0, 20, 0, 24), (20, 40, 0, 24)], {}, ("N", "N"),
                                periodic=(True, True))
    f = inputs.uniform_rhs(blocks, 2, remove_mean=True)
    po, _ = osv.solve(blocks, f)
    for prec in ("fp64", "mixed"):
        p, info, _ = gpu_solve(blocks, f, prec)
        assert rel(p, po) <= PARITY
        vol = ogrid.Grid(blocks).from_planes(ogrid.Grid(blocks).vol)
        assert abs(np.dot(vol, p)) <= 1e-12 * np.dot(vol, np.abs(p))


def test_zero_rhs_gives_zero():
    blocks = make("2x2", n=8, nz=8, zpair="NN", walls=("N", "N", "N", "N"))
    f = np.zeros(inputs.total_cells(blocks))
    p, info, _ = gpu_solve(blocks, f, p0=np.ones_like(f))
    assert info["status"] == 0 and np.all(p == 0.0)


def test_warm_start_and_constant_shift():
    """The latest solution as initial guess needs no correction; a constant added to the guess of a
    singular problem does not change the returned (zero-mean) solution."""
    blocks = make("L", n=8, nz=8, zpair="PP", walls=("N", "N", "N", "N"), stretched=True)
    f = inputs.divergence_rhs(blocks, 3)
    p1, info1, pl = gpu_solve(blocks, f)
    import torch
    p = dev(p1)
    info2 = pl.solve(dev(f), p, tol=TOL)
    assert info2["outer_iters"] == 0 and rel(host(p), p1) <= 1e-15
    p = dev(p1 + 3.0)
    pl.solve(dev(f), p, tol=TOL)
    assert rel(host(p), p1) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("zpair,walls", [("NN", ("N", "N", "N", "N")), ("DD", ("D", "N", "N", "N"))])
def test_zero_guess_shortcut_matches_residual_path(precision, zpair, walls):
    """A zero initial guess skips the first residual pass (r = f - mean). The returned solution and
    ||f - mean|| agree with a run whose guess is a tiny nonzero vector (the full residual path), and
    a guess of negative zeros counts as zero."""
    import torch
    blocks = make("2x2", n=16, nz=8, zpair=zpair, walls=walls, stretched=True)
    g = ogrid.Grid(blocks)
    f = inputs.divergence_rhs(blocks, 5)
    vol = g.from_planes(g.vol)
    mean = np.dot(vol, f) / vol.sum() if g.singular else 0.0
    p0, info0, pl = gpu_solve(blocks, f, precision)
    assert info0["status"] == 0 and info0["rel_res"] <= TOL
    assert abs(info0["rhs_norm"] - np.linalg.norm(f - mean)) <= 1e-12 * np.linalg.norm(f)
    tiny = np.zeros_like(f)
    tiny[7] = 1e-300
    p = dev(tiny)
    info1 = pl.solve(dev(f), p, tol=TOL)
    assert abs(info1["rhs_norm"] - info0["rhs_norm"]) <= 1e-13 * info0["rhs_norm"]
    assert rel(host(p), p0) <= 1e-9
    p = torch.full((len(f),), -0.0, dtype=torch.float64, device="cuda")
    info2 = pl.solve(dev(f), p, tol=TOL)
    assert info2["outer_iters"] == info0["outer_iters"] and rel(host(p), p0) <= 1e-15


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("layout,zpair,walls", [("2x2", "NN", ("N", "N", "N", "N")), ("L", "PP", ("N", "N", "N", "N")),
                                                ("1x2", "DD", ("D", "N", "N", "N")), ("1", "ND", ("D", "D", "N", "N"))])
def test_helmholtz_vs_oracle(precision, layout, zpair, walls):
    """(A + s I) p = f, s < 0 (the Helmholtz form of Sec. 3.3): regular even where s = 0 would be
    singular, so a right-hand side with a nonzero mean is solved as it is."""
    import torch
    blocks = make(layout, n=16, nz=8, zpair=zpair, walls=walls, stretched=True)
    f = inputs.uniform_rhs(blocks, 9, remove_mean=False) + 0.25
    s = -40.0
    po, _ = osv.solve(blocks, f, shift=s)
    p, info, pl = gpu_solve(blocks, f, precision, shift=s)
    assert info["status"] == 0 and info["rel_res"] <= TOL and info["removed_mean"] == 0.0
    assert osv.rel_residual(blocks, f, p, shift=s) <= 1.01 * TOL
    assert rel(p, po) <= PARITY
    out = torch.empty(len(f), dtype=torch.float64, device="cuda")
    pl.apply_operator(dev(p), out)
    assert rel(host(out), osv.apply_operator(blocks, p, shift=s)) <= 1e-13


@pytest.mark.parametrize("homog", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("layout,zpair,walls", [("L", "DN", ("D", "N", "N", "N")), ("2x2", "NN", ("N", "N", "N", "N")),
                                                ("1x2", "PP", ("D", "D", "N", "N"))])
def test_homogeneous_axis_x_or_y(homog, precision, layout, zpair, walls):
    """The same problems with the homogeneous direction along caller x or y (the plan transforms
    along that axis and runs the multigrid on the other two): identical to the oracle's solve of
    the z-homogeneous original once the caller layout is transposed back."""
    import torch
    blocks = make(layout, n=8, nz=8, zpair=zpair, walls=walls, stretched=True)
    f = inputs.divergence_rhs(blocks, 6)
    po, _ = osv.solve(blocks, f)
    rb, rf, back = homogeneous_along(blocks, f, homog)
    p, info, pl = gpu_solve(rb, rf, precision, homog_axis=homog)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, back(p)) <= 1.01 * TOL
    assert rel(back(p), po) <= PARITY
    q = np.random.default_rng(1).standard_normal(len(f))
    out = torch.empty(len(f), dtype=torch.float64, device="cuda")
    pl.apply_operator(dev(homogeneous_along(blocks, q, homog)[1]), out)
    assert rel(back(host(out)), osv.apply_operator(blocks, q)) <= 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graph_replay_matches_direct_launches(precision):
    """Without profiling the V-cycle rounds are replayed from captured CUDA graphs; with profiling
    they are launched one by one. Same kernels, same order: bitwise identical solutions and the same
    launch counts."""
    import torch
    blocks, f = inputs.config("mb2x2", seed=1, scale=8)
    pl = plan(blocks, precision=precision, onchip=False)  # the level-by-level rounds are what is replayed
    fd = dev(f)
    out = {}
    for prof in (True, False, False):
        pl.set_profiling(prof)
        pl.reset_stats()
        p = torch.zeros_like(fd)
        info = pl.solve(fd, p, tol=TOL)
        launches = sum(v["launches"] for v in pl.kernel_stats().values())
        out.setdefault(prof, []).append((host(p), info, launches))
    pl.set_profiling(False)
    (pd, idirect, ld), = out[True]
    assert idirect["graph_rounds"] == 0
    for pg, igraph, lg in out[False]:
        assert np.array_equal(pg, pd) and lg == ld
        assert igraph["graph_rounds"] > 0 and igraph["rel_res"] == idirect["rel_res"]


def test_errors():
    import torch
    blocks = make("2x2", n=8, nz=8, zpair="NN", walls=("N", "N", "N", "N"))
    N = inputs.total_cells(blocks)
    pl = plan(blocks)
    p = torch.zeros(N, dtype=torch.float64, device="cuda")
    f = inputs.uniform_rhs(blocks, 1, remove_mean=True)
    with pytest.raises(snac.SnacError) as e:
        pl.solve(dev(f + 1.0), p)
    assert e.value.name == "INCOMPATIBLE_RHS"
    assert torch.all(p == 0)
    fn = f.copy()
    fn[5] = np.nan
    with pytest.raises(snac.SnacError) as e:
        pl.solve(dev(fn), p)
    assert e.value.name == "NONFINITE"
    pl1 = plan(blocks, max_outer=1, max_cycles=1)
    p = torch.zeros(N, dtype=torch.float64, device="cuda")
    info = pl1.solve(dev(f), p, tol=1e-14, raise_on_error=False)
    assert info["status_name"] == "NOT_CONVERGED" and info["rel_res"] < 1.0
    with pytest.raises(ValueError):
        pl.solve(dev(f).float(), p)
    with pytest.raises(ValueError):
        pl.solve(dev(f)[:-1], p)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_stalled_solve_returns_its_best_iterate(precision):
    """A tolerance below the floating-point floor of the FP64 outer residual: the defect correction
    stops at the first step that does not lower the residual (instead of running max_outer steps),
    takes that step back and returns NOT_CONVERGED with the better iterate. The reported residual is
    that of the returned solution (re-evaluated independently here), it sits at the floor, and the
    solution still matches the oracle's."""
    import torch
    blocks, f = inputs.config("mb2x2", seed=3, scale=8)
    pref, _ = osv.solve(blocks, f)
    pl = plan(blocks, precision=precision, max_outer=20)
    fd = dev(f)
    p = torch.zeros_like(fd)
    info = pl.solve(fd, p, tol=1e-19, raise_on_error=False)
    assert info["status_name"] == "NOT_CONVERGED"
    assert info["outer_iters"] < 20                       # stopped by the stall, not by max_outer
    r = torch.empty_like(fd)
    r2, f2 = pl.residual(fd, p, r)
    # (the solve's residual is that of f minus its round-off mean, about 1e-17: hence rel=1e-3)
    assert info["rel_res"] == pytest.approx(np.sqrt(r2 / f2), rel=1e-3)
    assert info["rel_res"] <= 1e-12
    assert osv.rel_residual(blocks, f, host(p)) <= 1e-12
    assert rel(host(p), pref) <= PARITY
    # the same solve asked for a reachable tolerance converges to it: the stall is the floor
    p2 = torch.zeros_like(fd)
    info2 = pl.solve(fd, p2, tol=1e-11)
    assert info2["status"] == 0 and info2["outer_iters"] <= info["outer_iters"]
    pl.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nz,zpair", [(96, "PP"), (150, "NN"), (194, "DN"), (2048, "DD")])
def test_general_lengths_solve(nz, zpair, precision):
    """Homogeneous lengths that are not powers of two (the square-cylinder case of Sec. 4.2 uses
    n_z = 576; here 96 = 2^5 3, 150 = 2 3 5^2 and 194 = 2 97) and a long axis (2048), solved
    end to end against the oracle."""
    from layouts import make
    blocks = make("1x2", n=8 if nz < 1000 else 4, nz=nz, zpair=zpair, walls=("D", "N", "N", "N"), stretched=True)
    f = inputs.uniform_rhs(blocks, 12, remove_mean=False)
    ref, _ = osv.solve(blocks, f)
    p, info, _ = gpu_solve(blocks, f, precision)
    assert info["status"] == 0 and info["rel_res"] <= TOL
    assert osv.rel_residual(blocks, f, p) <= 1.01 * TOL
    assert rel(p, ref) <= PARITY
