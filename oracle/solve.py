"""Algorithm 1 (unfitted BAE) end to end (oracle route A).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Steps, in the order of Algorithm 1:
  1. LGF table G_s, s = kappa^2 h^2 (oracle/lgf.py).
  2. Point sets and closure from the phi samples (oracle/grid.py).
  3. Particular solution u_p = G_h[chi_{M+} f] on N+ (eq. [ps]).
  4. b = g - Phi u_p at the boundary points (Section 3.4, definition of b).
  5. A = Phi+ K+ + Phi- K- applied matrix-free, K = D (double layer,
     eq. [double_bae]) or S (single layer); one closure row per gamma- node:
        (A q)_m = t(m) (Kq)(m) + (1 - t(m)) (Kq)(p(m)).
  6. q = GMRES(A, b), zero initial guess, no preconditioner.
  7. u = u_p + K q on N+ (discrete generalized Green's formula,
     eq. [discrete_green], with the layer potential as the density term).

Readings: by default the particular solution is the free-lattice
convolution with G_s rather than the finite-box FFT solve of eq. [aux];
the discrete solution on N+ is unique, so u on N+ is the same (only q
differs). `particular="box"` takes the finite-box solve of eq. [aux]
(potentials.box_particular) as Algorithm 1 prints it. Sign convention: f
is the paper's, -Lap u + kappa^2 u = f.

`potential="direct"` evaluates every potential by direct summation over the
sources (small grids); `potential="fft"` uses the zero-padded FFT
convolution (the timed CPU baseline).

Parity: route A against route B (oracle/fd.py) in tests/test_oracle_solve.py.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import fd, gmres as gm, grid, lgf, potentials as pot


@dataclasses.dataclass
class Result:
    q: np.ndarray           # density on gamma-
    u: np.ndarray           # N^3, u on N+ (zero elsewhere)
    iterations: int
    residuals: list
    cls: grid.Classification
    seconds: dict


def boundary_rhs(cls, up_flat, g):
    return g - (cls.t * up_flat[cls.gm_idx] + (1.0 - cls.t) * up_flat[cls.partner])


def closure_apply(cls, v_flat):
    return cls.t * v_flat[cls.gm_idx] + (1.0 - cls.t) * v_flat[cls.partner]


def solve(phi, h, origin, f, g_fn, kappa2, layer="double", tol=1e-10, maxiter=500,
          potential="direct", table=None, spectrum=None, workers=1, particular="lattice") -> Result:
    """g_fn(xstar (n,3)) -> Dirichlet data at the boundary points."""
    sec = {}
    t0 = time.perf_counter()
    N = phi.shape[0]
    s = kappa2 * h * h
    cls = grid.classify(phi, h, origin)
    g = np.asarray(g_fn(cls.xstar), dtype=np.float64)
    nplus_idx = np.flatnonzero(cls.nplus)
    sec["classify"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    if potential == "fft":
        if spectrum is None:
            if table is None:
                table = lgf.LGFTable(N, s)
            spectrum = pot.lgf_spectrum(table)
    elif table is None:
        table = lgf.LGFTable(N, s)
    sec["lgf"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    fmask = np.where(cls.inside, np.asarray(f, dtype=np.float64), 0.0)
    if particular == "box":
        up = pot.box_particular(np.asarray(f, dtype=np.float64), h, s, cls.inside).reshape(-1)
    elif particular != "lattice":
        raise ValueError(particular)
    elif potential == "fft":
        up = pot.fft_convolve((h * h) * fmask, spectrum=spectrum, workers=workers).reshape(-1)
    else:
        up = np.zeros(N ** 3)
        up[nplus_idx] = pot.direct_particular(table, cls, f, h, nplus_idx)
    b = boundary_rhs(cls, up, g)
    sec["particular"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    if potential == "fft":
        def K_full(q):
            return pot.fft_convolve(pot.source_density(cls, q, layer), spectrum=spectrum, workers=workers).reshape(-1)

        def matvec(q):
            return closure_apply(cls, K_full(q))
    else:
        rows = np.concatenate([cls.gm_idx, cls.partner])
        K = pot.layer_matrix(table, cls, rows, layer)
        n = cls.gm_idx.size
        A = cls.t[:, None] * K[:n] + (1.0 - cls.t)[:, None] * K[n:]

        def matvec(q):
            return A @ q
    q, iters, hist = gm.gmres(matvec, b, tol=tol, maxiter=maxiter)
    sec["gmres"] = time.perf_counter() - t0

    t0 = time.perf_counter()
    u = np.zeros(N ** 3)
    if potential == "fft":
        u[nplus_idx] = (up + K_full(q))[nplus_idx]
    else:
        u[nplus_idx] = up[nplus_idx] + pot.direct_potential(table, cls, q, nplus_idx, layer)
    sec["reconstruct"] = time.perf_counter() - t0
    return Result(q=q, u=u.reshape((N,) * 3), iterations=iters, residuals=hist, cls=cls, seconds=sec)


def solve_fd(phi, h, origin, f, g_fn, kappa2):
    """Route B: the same discrete solution by a sparse direct solve."""
    cls = grid.classify(phi, h, origin)
    g = np.asarray(g_fn(cls.xstar), dtype=np.float64)
    return fd.solve_fd(cls, f, g, h, kappa2 * h * h), cls
