"""Unrestarted GMRES with modified Gram-Schmidt (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The boundary system of Section 3.4, eq. [double_bae], is solved in the paper
by "vanilla GMRES with no preconditioner and a zero initial guess"
(Section 4.1). This is the textbook method (Saad and Schultz 1986): Arnoldi
with modified Gram-Schmidt, Givens rotations on the Hessenberg matrix, stop
when the least-squares residual estimate |g_{j+1}| <= tol ||b||.

Parity: pinned in tests/test_oracle_gmres.py: solution equals a direct
solve, and the iteration count equals the number of distinct eigenvalues of
a diagonalisable matrix (minimal-polynomial property).
"""
from __future__ import annotations

import math

import numpy as np


def gmres(matvec, b: np.ndarray, tol: float = 1e-10, maxiter: int = 500):
    """Returns (x, iterations, residual_estimates)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    beta = float(np.linalg.norm(b))
    if beta == 0.0:
        return np.zeros(n), 0, [0.0]
    m = min(maxiter, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    cs = np.zeros(m)
    sn = np.zeros(m)
    g = np.zeros(m + 1)
    g[0] = beta
    V[0] = b / beta
    hist = [1.0]
    j_done = 0
    for j in range(m):
        w = np.asarray(matvec(V[j]), dtype=np.float64).copy()
        for i in range(j + 1):
            H[i, j] = float(V[i] @ w)
            w -= H[i, j] * V[i]
        H[j + 1, j] = float(np.linalg.norm(w))
        if H[j + 1, j] > 0.0:
            V[j + 1] = w / H[j + 1, j]
        for i in range(j):  # apply earlier rotations to the new column
            a, c = H[i, j], H[i + 1, j]
            H[i, j] = cs[i] * a + sn[i] * c
            H[i + 1, j] = -sn[i] * a + cs[i] * c
        r = math.hypot(H[j, j], H[j + 1, j])
        cs[j], sn[j] = H[j, j] / r, H[j + 1, j] / r
        H[j, j] = r
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        j_done = j + 1
        hist.append(abs(g[j + 1]) / beta)
        if abs(g[j + 1]) <= tol * beta or r == 0.0:
            break
    y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
    x = V[:j_done].T @ y
    return x, j_done, hist
