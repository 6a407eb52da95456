"""Pins of the oracle's GMRES and of the sparse finite-difference route."""
import numpy as np
import pytest

import workloads as W
from oracle import fd, grid
from oracle.gmres import gmres


def test_gmres_matches_direct_solve():
    rng = np.random.default_rng(0)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    x, it, hist = gmres(lambda v: A @ v, b, tol=1e-13)
    assert np.linalg.norm(A @ x - b) <= 2e-13 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=0, atol=1e-11)
    assert hist[-1] <= 1e-13


def test_gmres_minimal_polynomial_iterations():
    # a diagonalisable matrix with k distinct eigenvalues: exact convergence
    # after k Arnoldi steps
    rng = np.random.default_rng(1)
    n, k = 40, 5
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.repeat(np.arange(1, k + 1, dtype=float), n // k)
    A = Q @ np.diag(lam) @ Q.T
    b = rng.standard_normal(n)
    x, it, _ = gmres(lambda v: A @ v, b, tol=1e-10)
    assert it == k
    assert np.linalg.norm(A @ x - b) < 1e-9 * np.linalg.norm(b)


def test_fd_recovers_discrete_function():
    # pick u on N+, build f and g from the discrete equations, solve, recover u
    P = W.torus_helmholtz(24)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    h, s = P.grid.h, P.kappa2 * P.grid.h ** 2
    A, np_idx, pos = fd.assemble(cls, s)
    u = np.random.default_rng(2).standard_normal(np_idx.size)
    b = A @ u
    f = np.zeros(cls.N ** 3)
    f[cls.mp_idx] = b[pos[cls.mp_idx]] / (h * h)
    g = b[pos[cls.gm_idx]]
    got = fd.solve_fd(cls, f.reshape(P.phi.shape), g, h, s).reshape(-1)[np_idx]
    assert np.max(np.abs(got - u)) < 1e-10


def test_fd_row_is_seven_point_operator():
    P = W.sphere_exp(12)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    A, np_idx, pos = fd.assemble(cls, 0.5)
    r = pos[cls.mp_idx[0]]
    row = A.getrow(r)
    assert row.nnz == 7
    assert sorted(row.data) == [-1.0] * 6 + [6.5]
