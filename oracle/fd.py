"""The discrete problem as a sparse finite-difference system (oracle route B).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.1, eq. [discrete]: L_h u = -Lap_h u + sigma u = f on M+ with the
7-point Laplacian; multiplied by h^2 this is
    (6 + s) u(x) - sum_{6 neighbours y} u(y) = h^2 f(x),   x in M+, s = sigma h^2.
Every neighbour of an M+ node lies in N+ = M+ u gamma-, so the unknowns are
u on N+; the system is closed by one Dirichlet row per gamma- node, the same
closure the BAE uses (oracle/grid.py):
    t(m) u(m) + (1 - t(m)) u(p(m)) = g(x*(m)).
The BAE solution restricted to N+ is exactly this discrete solution (the
equivalence theorems of Sections 2.2 and 3.2), which makes this route an
LGF-free check of the whole chain.

Parity: pinned in tests/test_oracle_fd.py by recovering a random discrete
function from its own right-hand side, and by second-order convergence to
smooth exact solutions.
"""
from __future__ import annotations

import numpy as np
from scipy import sparse
from scipy.sparse import linalg as splinalg

from .grid import DIRS, Classification


def assemble(cls: Classification, s: float):
    """Sparse matrix over the N+ unknowns (lexicographic order) and the
    map from grid linear index to unknown number."""
    N = cls.N
    shape = (N, N, N)
    np_idx = np.flatnonzero(cls.nplus)
    pos = -np.ones(N ** 3, dtype=np.int64)
    pos[np_idx] = np.arange(np_idx.size)
    rows, cols, vals = [], [], []
    mp = cls.mp_idx
    r_mp = pos[mp]
    rows.append(r_mp); cols.append(r_mp); vals.append(np.full(mp.size, 6.0 + s))
    ijk = np.stack(np.unravel_index(mp, shape), axis=1)
    for d in DIRS:
        nb = np.ravel_multi_index((ijk + np.array(d)).T, shape)
        assert np.all(pos[nb] >= 0)
        rows.append(r_mp); cols.append(pos[nb]); vals.append(-np.ones(mp.size))
    r_gm = pos[cls.gm_idx]
    rows.append(r_gm); cols.append(r_gm); vals.append(cls.t.copy())
    rows.append(r_gm); cols.append(pos[cls.partner]); vals.append(1.0 - cls.t)
    A = sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(np_idx.size, np_idx.size))
    return A, np_idx, pos


def rhs(cls: Classification, f: np.ndarray, g: np.ndarray, h: float, pos) -> np.ndarray:
    b = np.zeros(int(cls.nplus.sum()))
    b[pos[cls.mp_idx]] = (h * h) * np.asarray(f).reshape(-1)[cls.mp_idx]
    b[pos[cls.gm_idx]] = g
    return b


def solve_fd(cls: Classification, f: np.ndarray, g: np.ndarray, h: float, s: float) -> np.ndarray:
    """u on the N^3 grid (zero off N+) solving the closed FD system."""
    A, np_idx, pos = assemble(cls, s)
    b = rhs(cls, f, g, h, pos)
    x = splinalg.spsolve(A.tocsc(), b)
    u = np.zeros(cls.N ** 3)
    u[np_idx] = x
    return u.reshape((cls.N,) * 3)


def harmonic_extension(cls: Classification, s: float, values_gm: np.ndarray) -> np.ndarray:
    """u on N+ with (6+s)u - sum u_nbr = 0 on M+ and u = values on gamma-
    (the gamma- -> gamma+ map that S+S-^{-1} and D+D-^{-1} represent)."""
    N = cls.N
    shape = (N, N, N)
    np_idx = np.flatnonzero(cls.nplus)
    pos = -np.ones(N ** 3, dtype=np.int64)
    pos[np_idx] = np.arange(np_idx.size)
    rows, cols, vals = [], [], []
    mp = cls.mp_idx
    rows.append(pos[mp]); cols.append(pos[mp]); vals.append(np.full(mp.size, 6.0 + s))
    ijk = np.stack(np.unravel_index(mp, shape), axis=1)
    for d in DIRS:
        nb = np.ravel_multi_index((ijk + np.array(d)).T, shape)
        rows.append(pos[mp]); cols.append(pos[nb]); vals.append(-np.ones(mp.size))
    rows.append(pos[cls.gm_idx]); cols.append(pos[cls.gm_idx]); vals.append(np.ones(cls.gm_idx.size))
    A = sparse.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(np_idx.size, np_idx.size))
    b = np.zeros(np_idx.size)
    b[pos[cls.gm_idx]] = values_gm
    x = splinalg.spsolve(A.tocsc(), b)
    u = np.zeros(N ** 3)
    u[np_idx] = x
    return u
