"""Pins of the oracle's whole solve (Algorithm 1): dense LU, closed forms, invariants."""
import numpy as np
import pytest
import scipy.fft

from oracle import grid as ogrid
from oracle import mg as omg
from oracle import solve as osv
from oracle import transforms as T
from paper_2106_03583_gb300 import inputs

from layouts import make

LAYOUTS = ["1", "1x2", "2x1", "L", "2x2"]
ZPAIRS = ["PP", "NN", "DD", "ND", "DN"]


@pytest.mark.parametrize("layout", LAYOUTS)
@pytest.mark.parametrize("zpair", ZPAIRS)
@pytest.mark.parametrize("walls", [("D", "D", "N", "N"), ("N", "N", "N", "N"), ("N", "D", "D", "N")])
@pytest.mark.parametrize("stretched", [False, True])
def test_matches_dense_lu(layout, zpair, walls, stretched):
    blocks = make(layout, n=4, nz=6, zpair=zpair, walls=walls, stretched=stretched)
    assert inputs.total_cells(blocks) <= 2000
    g = ogrid.Grid(blocks)
    f = inputs.uniform_rhs(blocks, 11, remove_mean=g.singular)
    p, info = osv.solve(blocks, f)
    pd = osv.solve_dense(blocks, f)
    assert np.linalg.norm(p - pd) <= 1e-11 * np.linalg.norm(pd)
    assert info["rel_res"] <= 1e-12


@pytest.mark.parametrize("zpair", ZPAIRS)
def test_manufactured_eigenfunction(zpair):
    """p = X_a(x) Y_b(y) Z_q(z) from the 1-D bases of each axis gives
    f = (lambda_a/dx^2 + lambda_b/dy^2 + lambda_q/dz^2) p exactly (Table 1, Eq. 8)."""
    nx, ny, nz = 16, 8, 8
    dx, dy, dz = 1.0 / nx, 2.0 / ny, 0.5 / nz
    xf, yf, zf = np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, np.arange(nz + 1) * dz
    blocks = inputs.make_blocks(xf, yf, zf, [(0, nx, 0, ny)], {"x-": "D", "x+": "D", "y-": "N", "y+": "D"},
                                make.__globals__["Z_PAIRS"][zpair])
    for (a, b, q) in [(0, 0, 0), (3, 5, 1), (nx - 1, ny - 1, nz - 1), (7, 2, nz // 2)]:
        X = T.basis_vector("DD", nx, a)
        Y = T.basis_vector("ND", ny, b)
        Z = T.basis_vector(zpair, nz, q)
        lam = (T.eigenvalues("DD", nx)[a] / dx ** 2 + T.eigenvalues("ND", ny)[b] / dy ** 2
               + T.eigenvalues(zpair, nz)[q] / dz ** 2)
        ph = (Z[:, None, None] * Y[None, :, None] * X[None, None, :]).ravel()
        p, _ = osv.solve(blocks, lam * ph)
        assert np.linalg.norm(p - ph) <= 1e-11 * np.linalg.norm(ph)


def test_triple_transform_closed_form():
    """Uniform box, x Dirichlet-Dirichlet (DST-II), y Neumann-Neumann (DCT-II), z periodic (DFT):
    the exact solve by transforms in all three directions (the direct-solver special case of Sec. 2)."""
    nx, ny, nz = 32, 16, 24
    lx, ly, lz = 1.0, 0.5, 2.0
    dx, dy, dz = lx / nx, ly / ny, lz / nz
    blocks = inputs.make_blocks(np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, np.arange(nz + 1) * dz,
                                [(0, nx, 0, ny)], {"x-": "D", "x+": "D", "y-": "N", "y+": "N"}, ("P", "P"))
    f = np.random.default_rng(2).uniform(-1, 1, (nz, ny, nx))
    F = scipy.fft.dst(scipy.fft.dct(np.fft.fft(f, axis=0), type=2, axis=1), type=2, axis=2)
    lx_ = 2 * (np.cos(np.pi * (np.arange(nx) + 1) / nx) - 1) / dx ** 2
    ly_ = 2 * (np.cos(np.pi * np.arange(ny) / ny) - 1) / dy ** 2
    lz_ = 2 * (np.cos(2 * np.pi * np.arange(nz) / nz) - 1) / dz ** 2
    P = F / (lz_[:, None, None] + ly_[None, :, None] + lx_[None, None, :])
    pex = np.fft.ifft(scipy.fft.idct(scipy.fft.idst(P, type=2, axis=2), type=2, axis=1), axis=0).real
    p, info = osv.solve(blocks, f.ravel())
    assert np.linalg.norm(p - pex.ravel()) <= 1e-12 * np.linalg.norm(pex)
    assert info["cycles"].max() > 1          # the multigrid really ran (several levels)
    assert info["levels"] >= 3


@pytest.mark.parametrize("layout", ["1", "L", "2x2"])
@pytest.mark.parametrize("zpair", ["PP", "NN"])
def test_zero_mean_invariant(layout, zpair):
    blocks = make(layout, n=4, nz=6, zpair=zpair, walls=("N", "N", "N", "N"), stretched=True)
    g = ogrid.Grid(blocks)
    assert g.singular
    vol = g.from_planes(g.vol)
    f = inputs.uniform_rhs(blocks, 3, remove_mean=True)
    p, info = osv.solve(blocks, f)
    assert abs(np.dot(vol, p)) <= 1e-13 * np.dot(vol, np.abs(p))
    # a round-off-sized incompatibility is removed and reported
    f2 = f + 1e-14
    p2, info2 = osv.solve(blocks, f2)
    assert abs(info2["removed_mean"] - 1e-14) < 1e-15
    assert np.linalg.norm(p2 - p) <= 1e-11 * np.linalg.norm(p)
    # a real one is an error
    with pytest.raises(osv.IncompatibleRHS):
        osv.solve(blocks, f + 1e-3)


def test_partition_invariance():
    """A 2x2 layout of n x n blocks equals one 2n x 2n block with the same outer faces (Sec. 4.1)."""
    n, nz = 16, 8
    for zpair in ("NN", "DD"):
        one = make("1", n=n, nz=nz, zpair=zpair, walls=("N", "D", "N", "N"), stretched=True)
        four = make("2x2", n=n, nz=nz, zpair=zpair, walls=("N", "D", "N", "N"), stretched=True)
        f1 = inputs.uniform_rhs(one, 9, remove_mean=False)
        # the same field, rearranged into the block layout
        F = f1.reshape(nz, 2 * n, 2 * n)
        f4 = np.concatenate([F[:, y0:y1, x0:x1].ravel() for (x0, x1, y0, y1) in
                             [(0, n, 0, n), (n, 2 * n, 0, n), (0, n, n, 2 * n), (n, 2 * n, n, 2 * n)]])
        p1, _ = osv.solve(one, f1)
        p4, _ = osv.solve(four, f4)
        P1 = p1.reshape(nz, 2 * n, 2 * n)
        p1r = np.concatenate([P1[:, y0:y1, x0:x1].ravel() for (x0, x1, y0, y1) in
                              [(0, n, 0, n), (n, 2 * n, 0, n), (0, n, n, 2 * n), (n, 2 * n, n, 2 * n)]])
        assert np.linalg.norm(p4 - p1r) <= 1e-12 * np.linalg.norm(p1r)


def test_divergence_free_projection():
    """u - G p is divergence-free when p solves L p = D u (Eqs. 4-5, the check of Sec. 4.1)."""
    blocks = make("L", n=8, nz=8, zpair="NN", walls=("N", "N", "N", "N"), stretched=True)
    f = inputs.divergence_rhs(blocks, seed=4)       # f = D u, unit RMS
    p, info = osv.solve(blocks, f)
    # the divergence of G p is A p; D(u - G p) = f - A p
    r = f - osv.apply_operator(blocks, p)
    assert np.linalg.norm(r) <= 1e-12 * np.linalg.norm(f)
    vol = ogrid.Grid(blocks).from_planes(ogrid.Grid(blocks).vol)
    assert abs(np.dot(vol, f)) <= 1e-13 * np.dot(vol, np.abs(f))   # walls carry no flux


def test_cycles_fall_with_eigenvalue():
    """Modes with larger |lambda_q| converge in fewer cycles (Sec. 3.3, App. B), up to one cycle."""
    blocks = make("1", n=16, nz=32, zpair="NN", walls=("D", "D", "N", "N"), stretched=False)
    f = inputs.uniform_rhs(blocks, 1, remove_mean=False)
    _, info = osv.solve(blocks, f)
    c = info["cycles"]
    assert all(c[q + 1] <= c[q] + 1 for q in range(len(c) - 1))
    assert c[-1] < c[0]


def test_planted_mistakes_are_caught(monkeypatch):
    """A wrong eigenvalue (NN read as PP) or a dropped Dirichlet ghost term in the oracle makes the
    closed-form pins fail: they are sensitive to the plausible mistakes."""
    blocks = make("1", n=4, nz=8, zpair="NN", walls=("D", "D", "N", "N"))
    f = inputs.uniform_rhs(blocks, 2, remove_mean=False)
    good = osv.solve_dense(blocks, f)
    real = T.eigenvalues
    monkeypatch.setattr(T, "eigenvalues", lambda kind, n: real("PP" if kind == "NN" else kind, n))
    bad, _ = osv.solve(blocks, f)
    assert np.linalg.norm(bad - good) > 1e-3 * np.linalg.norm(good)
    monkeypatch.setattr(T, "eigenvalues", real)
    orig = ogrid.Plane._build_operator

    def dropped(self):
        orig(self)
        fix = np.zeros(self.n)
        for axis, w in ((0, self.wx), (1, self.wy)):
            for side in range(2):
                d = self.nbr[axis, side] == -1
                fix[d] += 2.0 / w[d] ** 2            # remove the Dirichlet ghost contribution
        self.diag = self.diag + fix
        self.A = (self.offdiag + ogrid.sp.diags(self.diag)).tocsr()
    monkeypatch.setattr(ogrid.Plane, "_build_operator", dropped)
    from test_oracle_operator import staggered_div_grad
    p = np.random.default_rng(0).standard_normal(f.size)
    assert not np.allclose(osv.apply_operator(blocks, p), staggered_div_grad(blocks, p), rtol=1e-6)


@pytest.mark.parametrize("zpair", ZPAIRS)
def test_manufactured_eigenfunction_helmholtz(zpair):
    """Helmholtz form (A + s I) p = f (Sec. 3.3, footnote): the same eigenfunctions, with every
    eigenvalue shifted by s."""
    nx, ny, nz = 16, 8, 8
    dx, dy, dz = 1.0 / nx, 2.0 / ny, 0.5 / nz
    xf, yf, zf = np.arange(nx + 1) * dx, np.arange(ny + 1) * dy, np.arange(nz + 1) * dz
    blocks = inputs.make_blocks(xf, yf, zf, [(0, nx, 0, ny)], {"x-": "N", "x+": "N", "y-": "N", "y+": "N"},
                                make.__globals__["Z_PAIRS"][zpair])
    s = -37.5
    for (a, b, q) in [(0, 0, 0), (3, 5, 1), (nx - 1, ny - 1, nz - 1)]:
        X = T.basis_vector("NN", nx, a)
        Y = T.basis_vector("NN", ny, b)
        Z = T.basis_vector(zpair, nz, q)
        lam = (T.eigenvalues("NN", nx)[a] / dx ** 2 + T.eigenvalues("NN", ny)[b] / dy ** 2
               + T.eigenvalues(zpair, nz)[q] / dz ** 2 + s)
        ph = (Z[:, None, None] * Y[None, :, None] * X[None, None, :]).ravel()
        p, info = osv.solve(blocks, lam * ph, shift=s)
        assert not info["singular"]
        assert np.linalg.norm(p - ph) <= 1e-11 * np.linalg.norm(ph)


@pytest.mark.parametrize("layout", ["1", "L", "2x2"])
@pytest.mark.parametrize("zpair", ["PP", "NN", "DD", "DN"])
def test_helmholtz_matches_dense_lu(layout, zpair):
    """All-Neumann walls with a periodic or Neumann z would be singular; with a shift the problem is
    regular, any right-hand side is admissible, and the solve equals the dense solution."""
    blocks = make(layout, n=4, nz=6, zpair=zpair, walls=("N", "N", "N", "N"), stretched=True)
    f = inputs.uniform_rhs(blocks, 5, remove_mean=False) + 0.5
    for s in (-1.0, -250.0):
        p, info = osv.solve(blocks, f, shift=s)
        pd = osv.solve_dense(blocks, f, shift=s)
        assert info["removed_mean"] == 0.0
        assert np.linalg.norm(p - pd) <= 1e-11 * np.linalg.norm(pd)
        assert osv.rel_residual(blocks, f, p, shift=s) <= 1e-12


def test_helmholtz_shift_sign():
    blocks = make("1", n=4, nz=6, zpair="NN", walls=("N", "N", "N", "N"))
    f = inputs.uniform_rhs(blocks, 1, remove_mean=True)
    with pytest.raises(ValueError):
        osv.solve(blocks, f, shift=1.0)
    # shift 0 is Eq. 8 itself
    p0, _ = osv.solve(blocks, f)
    p1, _ = osv.solve(blocks, f, shift=0.0)
    assert np.array_equal(p0, p1)
