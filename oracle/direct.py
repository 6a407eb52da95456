"""The direct formulation of the boundary equations (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.2 (eq. [dp], the Theorem with eq. [bep] and its reduced form eq.
[rbep]) and Section 3 (eq. [direct_sys]): the unknown is u on
gamma = gamma- u gamma+. The difference potential of a grid function w on
gamma is
    P w = G_h [chi_{M-} L_h w];
on the free lattice with G_h = h^2 G_s and h^2 L_h = (6 + s) - (sum of the
six neighbours), it is the convolution of G_s with the source
    rho(n) = (6 + s) w(n) - sum_{y ~ n} w(y)   for n in M- (zero on M+),
w being zero off gamma. The closed system (eq. [inhom]: eq. [direct_sys]
with the particular solution on the right-hand side):
    u(p) - (P u)(p) = u_p(p)                          p in gamma+
    t(m) u(m) + (1 - t(m)) u(p(m)) = g(x*(m))          m in gamma-
and the solution on M+ is u = P u_gamma + u_p (eq. [discrete_green]).
Unknown order: gamma- (the lexicographic gm list), then gamma+
(lexicographic). Every closure partner p(m), an M+ neighbour of an M- node,
is a gamma+ node.

Parity: pinned in tests/test_oracle_direct.py by the Green's formula of the
Theorem (a discrete solution of eq. [discrete] equals u_p + P u_gamma on M+,
so it solves the gamma+ rows exactly), agreement of the solve with the
sparse finite-difference solve (oracle/fd.py), and the matrix-free apply
against its dense column-by-column assembly.
"""
from __future__ import annotations

import numpy as np

from . import gmres as gm, grid, lgf, potentials as pot


def unknown_nodes(cls: grid.Classification) -> np.ndarray:
    """Grid linear index of every unknown: gamma-, then gamma+."""
    return np.concatenate([cls.gm_idx, cls.gp_idx])


def partner_unknown(cls: grid.Classification) -> np.ndarray:
    """Unknown number of each closure partner p(m) (in the gamma+ block)."""
    k = np.searchsorted(cls.gp_idx, cls.partner)
    assert np.all(cls.gp_idx[np.minimum(k, cls.gp_idx.size - 1)] == cls.partner), "partner outside gamma+"
    return cls.gm_idx.size + k


def _neighbour_sum(a: np.ndarray) -> np.ndarray:
    """Sum of the six neighbours, zero outside the box."""
    out = np.zeros_like(a)
    for ax in range(3):
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(1, None)
        hi[ax] = slice(None, -1)
        out[tuple(lo)] += a[tuple(hi)]
        out[tuple(hi)] += a[tuple(lo)]
    return out


def source(cls: grid.Classification, w: np.ndarray, s: float) -> np.ndarray:
    """rho = chi_{M-} (6 + s - neighbour sum) w on the N^3 grid."""
    N = cls.N
    wg = np.zeros(N ** 3)
    wg[unknown_nodes(cls)] = w
    wg = wg.reshape((N,) * 3)
    lw = (6.0 + s) * wg - _neighbour_sum(wg)
    return np.where(cls.inside, 0.0, lw)


def difference_potential(cls, w, s, spectrum) -> np.ndarray:
    """P w on the N^3 grid (flat): the zero-padded FFT linear convolution."""
    return pot.fft_convolve(source(cls, w, s), spectrum=spectrum).reshape(-1)


def apply(cls, w, s, spectrum) -> np.ndarray:
    """The operator of the closed system: closure rows on gamma-, then
    w - P w on gamma+."""
    n = cls.gm_idx.size
    pw = difference_potential(cls, w, s, spectrum)
    out = np.empty_like(w)
    out[:n] = cls.t * w[:n] + (1.0 - cls.t) * w[partner_unknown(cls)]
    out[n:] = w[n:] - pw[cls.gp_idx]
    return out


def particular(cls, f, h, spectrum) -> np.ndarray:
    """u_p = G_s * (h^2 chi_{M+} f) on the N^3 grid (flat), eq. [ps]."""
    fmask = np.where(cls.inside, np.asarray(f, dtype=np.float64), 0.0)
    return pot.fft_convolve((h * h) * fmask, spectrum=spectrum).reshape(-1)


def rhs(cls, g, up) -> np.ndarray:
    return np.concatenate([np.asarray(g, dtype=np.float64), up[cls.gp_idx]])


def reconstruct(cls, w, s, up, spectrum) -> np.ndarray:
    """u on N+: u_p + P u_gamma on M+ (eq. [discrete_green]), u_gamma on
    gamma-; zero elsewhere (N^3)."""
    N = cls.N
    u = np.zeros(N ** 3)
    pw = difference_potential(cls, w, s, spectrum)
    u[cls.mp_idx] = up[cls.mp_idx] + pw[cls.mp_idx]
    u[cls.gm_idx] = w[: cls.gm_idx.size]
    return u.reshape((N,) * 3)


def solve(phi, h, origin, f, g_fn, kappa2, tol=1e-10, maxiter=2000, spectrum=None):
    """Direct-formulation solve: (u on N+ (N^3), u_gamma, iterations)."""
    N = phi.shape[0]
    s = kappa2 * h * h
    cls = grid.classify(phi, h, origin)
    if spectrum is None:
        spectrum = pot.lgf_spectrum(lgf.LGFTable(N, s))
    g = np.asarray(g_fn(cls.xstar), dtype=np.float64)
    up = particular(cls, f, h, spectrum)
    b = rhs(cls, g, up)
    w, iters, _ = gm.gmres(lambda v: apply(cls, v, s, spectrum), b, tol=tol, maxiter=maxiter)
    return reconstruct(cls, w, s, up, spectrum), w, iters
