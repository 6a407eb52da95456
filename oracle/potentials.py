"""Discrete layer potentials and the particular solution (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.2:
  single layer  S(m, n) = G_s(m - n)                          (eq. [single])
                v(m) = sum_{n in gamma-} S(m, n) q(n)          (eq. [single_potential])
  double layer  D(m, n) = sum_{k in D_n} [G_s(m - n) - G_s(m - k)]
                v(m) = sum_{n in gamma-} D(m, n) q(n)          (eq. [double_potential])
Section 2.1: particular solution u_p = G_h [chi_{M+} f] (eq. [ps]); on the free
lattice with G_h = h^2 G_s (Section 2.2, h = 1 scaling) this is
    u_p(m) = sum_{x in M+} G_s(m - x) h^2 f(x).

Reading (paper silent): a gamma- node whose D_n is empty would give an
identically zero double-layer column; such a column is replaced by the
single-layer column G_s(. - n), which is still lattice-harmonic on M+.

Both potentials are sums sum_x G_s(m - x) rho(x) over a source density rho
on the grid (rho = "B q"); `source_density` builds rho from q by the
definitions above, `direct_potential` does the sum term by term and
`fft_convolve` does the same linear convolution with a zero-padded (2N)^3
FFT (the "3D FFTs" of Section 2.2 and Algorithm 1).

Finite auxiliary box (eq. [aux] with eq. [ps], Algorithm 1's "u_p via FFT"
on the finite grid): `box_particular` solves L_h u = chi_{M+} f on the box
nodes M0 with u = 0 on the layer around them, by the sine basis that
diagonalizes the 7-point operator there. Reading (the paper does not fix
where the box boundary sits on the cell-centred grid): M0 = the nodes with
all indices in [1, N - 1], u = 0 on the layers of index 0 and N (the first
just inside the N^3 array, the second just outside it), so the basis
sin(pi k i / N), k = 1..N-1, has period 2N, the same as the zero-padded
free-lattice convolution. Pinned in tests/test_oracle_potentials.py by the
difference equation on M0, the zero layers, and a sparse direct solve.

Parity: pinned in tests/test_oracle_potentials.py by lattice harmonicity on
M+ (Propositions of Section 3.2), the lattice equation for u_p, agreement of
the direct and FFT routes, and the dense identities of Section 3.2.
"""
from __future__ import annotations

import numpy as np
from scipy import fft as sfft

from .grid import DIRS, Classification


def source_density(cls: Classification, q: np.ndarray, layer: str) -> np.ndarray:
    """rho on the N^3 grid such that v(m) = sum_x G_s(m - x) rho(x)."""
    N = cls.N
    rho = np.zeros(N ** 3)
    shape = (N, N, N)
    ijk = np.stack(np.unravel_index(cls.gm_idx, shape), axis=1)
    c = cls.count.reshape(-1)[cls.gm_idx]
    if layer == "single":
        np.add.at(rho, cls.gm_idx, q)
        return rho.reshape(shape)
    if layer != "double":
        raise ValueError(layer)
    nplus = cls.nplus.reshape(-1)
    coef = np.where(c > 0, c, 1).astype(np.float64)
    np.add.at(rho, cls.gm_idx, coef * q)
    for d in DIRS:
        k = ijk + np.array(d)
        lin = np.ravel_multi_index(k.T, shape)
        out = ~nplus[lin]           # k in D_n
        np.add.at(rho, lin[out], -q[out])
    return rho.reshape(shape)


def layer_matrix(table, cls: Classification, targets: np.ndarray, layer: str) -> np.ndarray:
    """Dense K[t, n] = S(m_t, n) or D(m_t, n) for target nodes (linear
    indices) and all source nodes n in gamma-, column by column."""
    N = cls.N
    shape = (N, N, N)
    tg = np.stack(np.unravel_index(np.asarray(targets), shape), axis=1)
    src = np.stack(np.unravel_index(cls.gm_idx, shape), axis=1)
    nplus = cls.nplus
    K = np.zeros((len(tg), len(src)))
    for col, n in enumerate(src):
        g_mn = table(tg - n)
        if layer == "single":
            K[:, col] = g_mn
            continue
        Dn = [n + np.array(d) for d in DIRS if not nplus[tuple(n + np.array(d))]]
        if not Dn:
            K[:, col] = g_mn
            continue
        acc = np.zeros(len(tg))
        for k in Dn:
            acc += g_mn - table(tg - k)
        K[:, col] = acc
    return K


def direct_potential(table, cls: Classification, q: np.ndarray, targets: np.ndarray, layer: str) -> np.ndarray:
    """v at the target nodes by the plain sum over the nonzero source nodes."""
    N = cls.N
    shape = (N, N, N)
    rho = source_density(cls, q, layer).reshape(-1)
    nz = np.flatnonzero(rho)
    src = np.stack(np.unravel_index(nz, shape), axis=1)
    tg = np.stack(np.unravel_index(np.asarray(targets), shape), axis=1)
    out = np.zeros(len(tg))
    for a in range(len(nz)):
        out += table(tg - src[a]) * rho[nz[a]]
    return out


def direct_particular(table, cls: Classification, f: np.ndarray, h: float, targets: np.ndarray) -> np.ndarray:
    """u_p at the target nodes: sum over x in M+ of G_s(m - x) h^2 f(x)."""
    N = cls.N
    shape = (N, N, N)
    src = np.stack(np.unravel_index(cls.mp_idx, shape), axis=1)
    w = (h * h) * np.asarray(f, dtype=np.float64).reshape(-1)[cls.mp_idx]
    tg = np.stack(np.unravel_index(np.asarray(targets), shape), axis=1)
    out = np.zeros(len(tg))
    for a in range(len(src)):
        out += table(tg - src[a]) * w[a]
    return out


def embedded_lgf(table) -> np.ndarray:
    """G_s on the (2N)^3 periodic box: offset a in [0, 2N) stands for a
    (a < N) or a - 2N (a > N); the unused offset a = N is set to 0."""
    N = table.N
    a = np.arange(2 * N)
    off = np.where(a < N, a, 2 * N - a)
    valid = a != N
    g = table.cube[np.ix_(np.clip(off, 0, N - 1), np.clip(off, 0, N - 1), np.clip(off, 0, N - 1))].copy()
    g[~valid, :, :] = 0.0
    g[:, ~valid, :] = 0.0
    g[:, :, ~valid] = 0.0
    return g


def lgf_spectrum(table) -> np.ndarray:
    """Real 3D DFT of the embedded G_s, (2N, 2N, N+1) half spectrum."""
    return np.real(sfft.rfftn(embedded_lgf(table)))


def fft_convolve(rho: np.ndarray, table=None, spectrum: np.ndarray | None = None, workers: int = 1) -> np.ndarray:
    """v(m) = sum_x G_s(m - x) rho(x) for all m in the N^3 grid by a
    zero-padded (2N)^3 real FFT in float64."""
    N = rho.shape[0]
    if spectrum is None:
        spectrum = lgf_spectrum(table)
    rf = sfft.rfftn(rho, s=(2 * N,) * 3, workers=workers)
    v = sfft.irfftn(rf * spectrum, s=(2 * N,) * 3, workers=workers)
    return v[:N, :N, :N]


def box_particular(f: np.ndarray, h: float, s: float, inside: np.ndarray) -> np.ndarray:
    """u = G_h[chi_{M+} f] on the finite auxiliary box (eqs. [aux], [ps]) in
    lattice units: (6 + s) u(m) - sum of the six neighbours = h^2 f(m) [m in
    M+] for m in M0 = [1, N-1]^3, u = 0 on the layers 0 and N. In the basis
    sin(pi k i / N) (k = 1..N-1 per axis; a type-I sine transform of length
    N - 1) the operator is diagonal with eigenvalue 6 + s - 2 sum_d cos(pi
    k_d / N). Returns the N^3 array (zero on the layer 0)."""
    N = f.shape[0]
    q = (h * h) * np.where(inside, np.asarray(f, dtype=np.float64), 0.0)[1:, 1:, 1:]
    Q = sfft.dstn(q, type=1)
    c = 2.0 * np.cos(np.pi * np.arange(1, N) / N)
    lam = (6.0 + s) - (c[:, None, None] + c[None, :, None] + c[None, None, :])
    u = np.zeros((N, N, N))
    u[1:, 1:, 1:] = sfft.idstn(Q / lam, type=1)
    return u
