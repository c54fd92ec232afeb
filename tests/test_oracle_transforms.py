"""Pins of the oracle's transforms and eigenvalues (Table 1) against library routines, the printed
table and closed forms."""
import os
import re

import numpy as np
import pytest
import scipy.fft

from oracle import grid as ogrid
from oracle import transforms as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NS = [2, 4, 6, 8, 16, 32, 34]


@pytest.mark.parametrize("n", NS)
def test_forward_matches_scipy(n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n)
    assert np.allclose(T.forward("NN", x), scipy.fft.dct(x, type=2), rtol=0, atol=1e-12 * n)
    assert np.allclose(T.forward("DD", x), scipy.fft.dst(x, type=2), rtol=0, atol=1e-12 * n)
    assert np.allclose(T.forward("ND", x), scipy.fft.dct(x, type=4), rtol=0, atol=1e-12 * n)
    assert np.allclose(T.forward("DN", x), scipy.fft.dst(x, type=4), rtol=0, atol=1e-12 * n)
    h = T.forward("PP", x)
    c = np.fft.rfft(x)
    assert np.allclose(h[: n // 2 + 1], c.real, atol=1e-12 * n)
    k = np.arange(1, n // 2)
    assert np.allclose(h[n - k], c.imag[k], atol=1e-12 * n)


@pytest.mark.parametrize("n", NS)
def test_backward_matches_scipy(n):
    rng = np.random.default_rng(100 + n)
    X = rng.standard_normal(n)
    B = lambda kind: T.backward_matrix(kind, n) @ X
    assert np.allclose(B("NN"), scipy.fft.dct(X, type=3), atol=1e-12 * n)
    assert np.allclose(B("DD"), scipy.fft.dst(X, type=3), atol=1e-12 * n)
    assert np.allclose(B("ND"), scipy.fft.dct(X, type=4), atol=1e-12 * n)
    assert np.allclose(B("DN"), scipy.fft.dst(X, type=4), atol=1e-12 * n)
    # half-complex -> real: numpy irfft of the packed spectrum, times n
    c = np.zeros(n // 2 + 1, dtype=complex)
    c.real = X[: n // 2 + 1]
    k = np.arange(1, n // 2)
    c.imag[k] = X[n - k]
    assert np.allclose(B("PP"), n * np.fft.irfft(c, n), atol=1e-12 * n)


@pytest.mark.parametrize("kind", T.KINDS)
@pytest.mark.parametrize("n", NS)
def test_round_trip_theta(kind, n):
    M = T.backward_matrix(kind, n) @ T.forward_matrix(kind, n)
    assert np.allclose(M, T.theta(kind, n) * np.eye(n), atol=1e-11 * n)


@pytest.mark.parametrize("kind", T.KINDS)
@pytest.mark.parametrize("n", NS)
def test_eigenvalues_closed_form(kind, n):
    """The 1-D staggered operator with the face ghosts of the pair maps every basis vector v_q to
    lambda_q v_q, lambda_q from Table 1."""
    D = ogrid.dzz_matrix(kind, n, 1.0)
    lam = T.eigenvalues(kind, n)
    for q in range(n):
        v = T.basis_vector(kind, n, q)
        assert np.linalg.norm(v) > 0.5
        assert np.allclose(D @ v, lam[q] * v, atol=1e-12 * max(1.0, np.abs(lam).max()))


@pytest.mark.parametrize("kind", T.KINDS)
def test_transform_diagonalises_operator(kind):
    """F (D_zz x) = Lambda F x for random x: the synthesis of Eq. 8 into Eq. 9."""
    n = 16
    rng = np.random.default_rng(7)
    x = rng.standard_normal(n)
    D = ogrid.dzz_matrix(kind, n, 0.25)
    lhs = T.forward(kind, D @ x)
    rhs = T.eigenvalues(kind, n) / 0.25 ** 2 * T.forward(kind, x)
    assert np.allclose(lhs, rhs, atol=1e-10 * np.abs(rhs).max())


def test_periodic_eigenvalue_example():
    """The periodic case in closed form: lambda_k / dz^2 = 2 (cos(2 pi k / N) - 1) / dz^2."""
    n, dz = 12, 0.1
    k = np.arange(n)
    assert np.allclose(T.eigenvalues("PP", n) / dz ** 2, 2 * (np.cos(2 * np.pi * k / n) - 1) / dz ** 2)


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_operators.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([c.strip() for c in line.split("|")])
    return rows


def _expr(s):
    """Printed arithmetic ("2q+1", "2n") as a Python expression."""
    return re.sub(r"(\d)([a-z(])", r"\1*\2", s)


def test_table1_golden():
    """Table 1 as printed: kappa_q/(2 pi/l), F, theta*F^-1 and theta for every pair."""
    lib = {"DFT": None, "DCT-II": (scipy.fft.dct, 2), "DST-II": (scipy.fft.dst, 2),
           "DCT-III": (scipy.fft.dct, 3), "DST-III": (scipy.fft.dst, 3), "DCT-IV": (scipy.fft.dct, 4)}
    rows = _table1()
    assert [r[0] for r in rows] == ["PP", "NN", "DD", "ND"]
    for pair, kappa, fwd, bwd, th in rows:
        for n in (4, 8, 10):
            q = np.arange(n, dtype=float)
            m = eval(_expr(kappa), {"q": q})          # kappa_q / (2 pi / l)
            lam = 2.0 * (np.cos(2.0 * np.pi * m / n) - 1.0)   # kappa dl = 2 pi m / n
            assert np.allclose(T.eigenvalues(pair, n), lam, atol=1e-14)
            assert T.theta(pair, n) == eval(_expr(th), {"n": n})
            x = np.random.default_rng(n).standard_normal(n)
            if lib[fwd] is not None:
                fn, t = lib[fwd]
                assert np.allclose(T.forward(pair, x), fn(x, type=t), atol=1e-12)
                fn, t = lib[bwd]
                assert np.allclose(T.backward_matrix(pair, n) @ x, fn(x, type=t), atol=1e-12)
