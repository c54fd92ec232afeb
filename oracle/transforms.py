"""Real-to-real transforms along the homogeneous direction, from their definitions (Table 1, Sec. 2).

Test infrastructure only (see the package docstring).

Every forward transform F and scaled backward transform theta*F^-1 is written out as an explicit
n x n matrix of cosines/sines and applied by a matrix product: O(n^2) per column, no FFT. The
conventions are the unnormalised real-to-real ones of the FFTW library the paper uses (Sec. 3.3.2):

  PP  (periodic)          F = real DFT, half-complex order   theta*F^-1 = its inverse (x n)   theta = n
  NN  (Neumann-Neumann)   F = DCT-II                         theta*F^-1 = DCT-III             theta = 2n
  DD  (Dirichlet-Dirichlet) F = DST-II                       theta*F^-1 = DST-III             theta = 2n
  ND  (Neumann at 0, Dirichlet at L) F = DCT-IV              theta*F^-1 = DCT-IV              theta = 2n
  DN  (Dirichlet at 0, Neumann at L) F = DST-IV              theta*F^-1 = DST-IV              theta = 2n

DN does not appear in Table 1; it is the mirror image of ND (the same eigenvalues, sine instead of
cosine basis).

Eigenvalues (Table 1): lambda_q = 2 (cos(kappa_q dl) - 1), q = 0..n-1, dl = l/n, with
kappa_q / (2 pi / l) = q (PP), q/2 (NN), (q+1)/2 (DD), (2q+1)/4 (ND and DN).
For PP in half-complex order, slot q holds wavenumber min(q, n-q); the cosine is the same for q and
n-q, so the formula applies slot by slot.
"""
from __future__ import annotations

import numpy as np

KINDS = ("PP", "NN", "DD", "ND", "DN")


def kind_from_bc(lo: str, hi: str) -> str:
    """Transform kind for a pair of z boundary conditions ("P", "N", "D")."""
    if lo == "P" or hi == "P":
        if lo != hi:
            raise ValueError("periodic z needs both faces periodic")
        return "PP"
    return lo + hi


def theta(kind: str, n: int) -> float:
    """Normalisation theta of Table 1: theta*F^-1 F = theta * identity."""
    return float(n) if kind == "PP" else 2.0 * n


def eigenvalues(kind: str, n: int) -> np.ndarray:
    """lambda_q = 2 (cos(kappa_q dl) - 1), Table 1, written as 2 (cos(2 pi m_q / n) - 1)."""
    q = np.arange(n, dtype=np.float64)
    m = {"PP": q, "NN": q / 2.0, "DD": (q + 1.0) / 2.0, "ND": (2.0 * q + 1.0) / 4.0,
         "DN": (2.0 * q + 1.0) / 4.0}[kind]
    return 2.0 * (np.cos(2.0 * np.pi * m / n) - 1.0)


def forward_matrix(kind: str, n: int) -> np.ndarray:
    """Matrix of the forward transform F (rows: output index k, columns: input index j)."""
    j = np.arange(n, dtype=np.float64)[None, :]
    k = np.arange(n, dtype=np.float64)[:, None]
    if kind == "PP":
        if n % 2:
            raise ValueError("the real DFT in half-complex order needs an even n")
        M = np.zeros((n, n))
        kk = np.arange(n // 2 + 1)
        # real parts r_k = sum_j x_j cos(2 pi j k / n), k = 0..n/2, stored at slot k
        M[kk, :] = np.cos(2.0 * np.pi * kk[:, None] * j / n)
        # imaginary parts i_k = -sum_j x_j sin(2 pi j k / n), k = 1..n/2-1, stored at slot n-k
        ki = np.arange(1, n // 2)
        M[n - ki, :] = -np.sin(2.0 * np.pi * ki[:, None] * j / n)
        return M
    if kind == "NN":   # DCT-II: Y_k = 2 sum_j x_j cos(pi (j + 1/2) k / n)
        return 2.0 * np.cos(np.pi * (j + 0.5) * k / n)
    if kind == "DD":   # DST-II: Y_k = 2 sum_j x_j sin(pi (j + 1/2) (k + 1) / n)
        return 2.0 * np.sin(np.pi * (j + 0.5) * (k + 1.0) / n)
    if kind == "ND":   # DCT-IV: Y_k = 2 sum_j x_j cos(pi (j + 1/2) (k + 1/2) / n)
        return 2.0 * np.cos(np.pi * (j + 0.5) * (k + 0.5) / n)
    if kind == "DN":   # DST-IV: Y_k = 2 sum_j x_j sin(pi (j + 1/2) (k + 1/2) / n)
        return 2.0 * np.sin(np.pi * (j + 0.5) * (k + 0.5) / n)
    raise ValueError(kind)


def backward_matrix(kind: str, n: int) -> np.ndarray:
    """Matrix of theta*F^-1 (rows: output index j, columns: input index k)."""
    jj = np.arange(n, dtype=np.float64)[:, None]
    k = np.arange(n, dtype=np.float64)[None, :]
    if kind == "PP":   # x_j = H_0 + (-1)^j H_{n/2} + 2 sum_{k=1}^{n/2-1} (H_k cos - H_{n-k} sin)(2 pi j k / n)
        M = np.zeros((n, n))
        M[:, 0] = 1.0
        M[:, n // 2] = np.cos(np.pi * jj[:, 0])
        ki = np.arange(1, n // 2)
        M[:, ki] = 2.0 * np.cos(2.0 * np.pi * jj * ki[None, :] / n)
        M[:, n - ki] = -2.0 * np.sin(2.0 * np.pi * jj * ki[None, :] / n)
        return M
    if kind == "NN":   # DCT-III: x_j = X_0 + 2 sum_{k>=1} X_k cos(pi k (j + 1/2) / n)
        M = 2.0 * np.cos(np.pi * k * (jj + 0.5) / n)
        M[:, 0] = 1.0
        return M
    if kind == "DD":   # DST-III: x_j = (-1)^j X_{n-1} + 2 sum_{k<n-1} X_k sin(pi (k + 1) (j + 1/2) / n)
        M = 2.0 * np.sin(np.pi * (k + 1.0) * (jj + 0.5) / n)
        M[:, n - 1] = np.cos(np.pi * jj[:, 0])
        return M
    if kind in ("ND", "DN"):   # DCT-IV and DST-IV are their own inverses up to 2n
        return forward_matrix(kind, n).T.copy()
    raise ValueError(kind)


def forward(kind: str, x: np.ndarray) -> np.ndarray:
    """F applied along axis 0 of x (shape (n, ...))."""
    n = x.shape[0]
    return (forward_matrix(kind, n) @ x.reshape(n, -1)).reshape(x.shape)


def backward(kind: str, X: np.ndarray) -> np.ndarray:
    """F^-1 applied along axis 0 (theta*F^-1 divided by theta)."""
    n = X.shape[0]
    return (backward_matrix(kind, n) @ X.reshape(n, -1)).reshape(X.shape) / theta(kind, n)


def basis_vector(kind: str, n: int, q: int) -> np.ndarray:
    """Eigenvector v_q of the 1-D staggered operator for the pair (continuous eigenfunction sampled
    at cell centres j + 1/2): the function whose discrete eigenvalue is lambda_q."""
    j = np.arange(n, dtype=np.float64) + 0.5
    if kind == "PP":   # any phase is an eigenvector on a periodic grid; use the cell index
        m = min(q, n - q)
        jp = j - 0.5
        return np.cos(2.0 * np.pi * m * jp / n) if q <= n // 2 else np.sin(2.0 * np.pi * m * jp / n)
    if kind == "NN":
        return np.cos(np.pi * q * j / n)
    if kind == "DD":
        return np.sin(np.pi * (q + 1) * j / n)
    if kind == "ND":
        return np.cos(np.pi * (2 * q + 1) * j / (2 * n))
    if kind == "DN":
        return np.sin(np.pi * (2 * q + 1) * j / (2 * n))
    raise ValueError(kind)
