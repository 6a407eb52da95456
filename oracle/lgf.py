"""Lattice Green's function of (6+s) - sum of the six neighbours (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Definition (Section 2.2, eq. [lgf] with h = 1, and Watson's transformation
eq. [lgf_bessel] generalised to sigma > 0): with s = sigma h^2,

    G_s(n) = int_0^inf exp(-s t) Ie_{n1}(2t) Ie_{n2}(2t) Ie_{n3}(2t) dt,

where Ie_n(x) = exp(-x) I_n(x) is the exponentially scaled modified Bessel
function, so that exp(-(6+s)t) I I I = exp(-s t) Ie Ie Ie. G_s solves
(6+s) G(n) - sum_{+-e_i} G(n +- e_i) = delta_{n,0} (eq. [lgf_delta] scaled by
h^2).

Evaluation follows the paper's split (Section 2.2): adaptive quadrature on a
finite range and the large-argument Bessel series (Abramowitz-Stegun 9.7.1,
with mu = 4n^2) beyond T_TAIL = 1e8, where the series is summed to 6 terms.
scipy's `ive` is used below T_TAIL (it returns NaN above about 1e9).

Readings (paper garbled or silent):
  * The paper's Gamma-function values of G_0(0) are twice the G defined by
    eqs. [lgf]/[lgf_bessel]; the pin here is half of them (0.2527310098587...).
  * The far-field expansion A_G^q is printed with the wrong overall sign; the
    correct one is +1/(4 pi |n|) + ..., used only as a test invariant.
  * In A_G^3 the coefficient printed as -288 (of k^2 l^2 j^4 + ...) is read as
    -228: with -228 the remainder G_0 - A_G^3 times |n|^7 stays below 0.35 in
    every direction tried (0.120 on the diagonal for |n| from 35 to 69); with
    -288 it grows like |n|^2 along the diagonal, i.e. the q = 3 expansion
    would only be O(|n|^-5) there.

Parity: pinned (tests/test_oracle_lgf.py): Watson closed form, lattice
identity, symmetry, far-field expansion, and for s > 0 the periodic
trapezoid sum of Section 2.2; the closed-form periodic spectrum against the
spectrum of the Bessel table where its applicability rule holds, and its
failure where it does not.
"""
from __future__ import annotations

import math
import warnings

import numpy as np
from scipy import integrate, special

T_TAIL = 1.0e8


def watson_g0() -> float:
    """G_0(0,0,0) from the Gamma-function closed form (Section 2.2), halved:
    sqrt(6)/(192 pi^3) Gamma(1/24) Gamma(5/24) Gamma(7/24) Gamma(11/24)."""
    g = math.gamma
    return math.sqrt(6.0) / (192.0 * math.pi ** 3) * g(1 / 24) * g(5 / 24) * g(7 / 24) * g(11 / 24)


def watson_g0_alt() -> float:
    """Second closed form of Section 2.2, halved:
    (sqrt(3) - 1)/(192 pi^3) [Gamma(1/24) Gamma(11/24)]^2."""
    g = math.gamma
    return (math.sqrt(3.0) - 1.0) / (192.0 * math.pi ** 3) * (g(1 / 24) * g(11 / 24)) ** 2


def ive_large(n, t, terms: int = 6):
    """exp(-2t) I_n(2t) by the large-argument series with mu = 4 n^2:
    (2 pi x)^(-1/2) [1 - (mu-1)/(8x) + (mu-1)(mu-9)/(2! (8x)^2) - ...], x=2t."""
    mu = 4.0 * np.asarray(n, dtype=np.float64) ** 2
    x = 2.0 * t
    term = np.ones_like(mu)
    total = np.ones_like(mu)
    for k in range(1, terms + 1):
        term = term * (-(mu - (2 * k - 1) ** 2) / (k * 8.0 * x))
        total = total + term
    return total / math.sqrt(2.0 * math.pi * x)


def _breakpoints(t_hi: float):
    pts = [0.0]
    k = 0
    while 4.0 ** k < t_hi:
        pts.append(4.0 ** k)
        k += 1
    pts.append(t_hi)
    return pts


def lgf_entry(n, s: float) -> float:
    """G_s(n) for one integer offset n by scipy.quad, panel by panel."""
    n1, n2, n3 = (abs(int(v)) for v in n)

    def body(t):
        return math.exp(-s * t) * special.ive(n1, 2 * t) * special.ive(n2, 2 * t) * special.ive(n3, 2 * t)

    def tail(w):  # t = T_TAIL / w^2, dt = 2 T_TAIL / w^3 dw
        if w == 0.0:
            return 0.0
        t = T_TAIL / (w * w)
        iv = ive_large(np.array([n1, n2, n3]), t)
        return math.exp(-s * t) * float(iv[0] * iv[1] * iv[2]) * 2.0 * T_TAIL / w ** 3

    total = 0.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", integrate.IntegrationWarning)
        pts = _breakpoints(T_TAIL)
        for a, b in zip(pts[:-1], pts[1:]):
            total += integrate.quad(body, a, b, epsabs=0.0, epsrel=1e-13, limit=500)[0]
        total += integrate.quad(tail, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=500)[0]
    return total


def sorted_triples(N: int) -> np.ndarray:
    """All (a, b, c) with N > a >= b >= c >= 0, lexicographic in (a, b, c)."""
    out = [(a, b, c) for a in range(N) for b in range(a + 1) for c in range(b + 1)]
    return np.array(out, dtype=np.int64).reshape(-1, 3)


def lgf_triples(tri: np.ndarray, s: float) -> np.ndarray:
    """G_s at many offsets at once: the same integral as lgf_entry, with
    scipy.quad_vec on the same panels. Each entry is scaled by a rough
    inverse magnitude 4 pi |n| exp(sqrt(s)|n|) inside the integral so that
    the shared max-norm error control acts per entry relatively; the scale is
    divided out afterwards."""
    tri = np.abs(np.asarray(tri, dtype=np.int64))
    nmax = int(tri.max()) + 1 if len(tri) else 1
    ns = np.arange(nmax)
    r = np.sqrt((tri.astype(np.float64) ** 2).sum(axis=1))
    wgt = 4.0 * math.pi * np.maximum(r, 1.0) * np.exp(math.sqrt(s) * r)
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]

    def body(t):
        iv = special.ive(ns, 2.0 * t)
        return math.exp(-s * t) * iv[a] * iv[b] * iv[c] * wgt

    def tail(w):
        if w == 0.0:
            return np.zeros(len(tri))
        t = T_TAIL / (w * w)
        iv = ive_large(ns, t)
        return math.exp(-s * t) * iv[a] * iv[b] * iv[c] * wgt * (2.0 * T_TAIL / w ** 3)

    total = np.zeros(len(tri))
    kw = dict(epsabs=1e-300, epsrel=2e-15, norm="max", limit=100000)
    pts = _breakpoints(T_TAIL)
    for lo, hi in zip(pts[:-1], pts[1:]):
        total += integrate.quad_vec(body, lo, hi, **kw)[0]
    total += integrate.quad_vec(tail, 0.0, 1.0, **kw)[0]
    return total / wgt


class LGFTable:
    """G_s(n) for 0 <= n_i < N, stored for sorted triples only (the 1/48
    symmetry of the numerical section), with lookup at any signed offset."""

    def __init__(self, N: int, s: float, values: np.ndarray | None = None):
        self.N, self.s = int(N), float(s)
        self.tri = sorted_triples(self.N)
        self.values = lgf_triples(self.tri, self.s) if values is None else np.asarray(values, np.float64)
        # dense cube view, G[|n1|, |n2|, |n3|] for 0 <= |n_i| < N
        self.cube = np.empty((self.N,) * 3)
        t = self.tri
        for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
            self.cube[t[:, perm[0]], t[:, perm[1]], t[:, perm[2]]] = self.values

    def __call__(self, d):
        """G_s at integer offsets d (..., 3), any sign, |d_i| < N."""
        d = np.abs(np.asarray(d, dtype=np.int64))
        return self.cube[d[..., 0], d[..., 1], d[..., 2]]


def far_field(n) -> float:
    """Three-term far-field expansion of G_0 (Section 2.2, after
    Martinsson-Rodin), with the overall sign fixed so that G_0 ~ +1/(4 pi|n|):
    1/(4 pi r) + T2/(16 pi r^7) + T3/(128 pi r^13), T3 with -228 (see header)."""
    j, k, l = (float(v) for v in n)
    r2 = j * j + k * k + l * l
    r = math.sqrt(r2)
    t2 = j ** 4 + k ** 4 + l ** 4 - 3 * (j * j * k * k + j * j * l * l + k * k * l * l)
    t3 = (-228 * (k * k * l * l * j ** 4 + k * k * l ** 4 * j * j + k ** 4 * l * l * j * j)
          + 621 * (j ** 4 * k ** 4 + l ** 4 * k ** 4 + j ** 4 * l ** 4)
          - 244 * (k * k * j ** 6 + l * l * j ** 6 + k ** 6 * j * j + l ** 6 * j * j + k * k * l ** 6 + k ** 6 * l * l)
          + 23 * (j ** 8 + k ** 8 + l ** 8))
    return 1.0 / (4 * math.pi * r) + t2 / (16 * math.pi * r ** 7) + t3 / (128 * math.pi * r ** 13)


def periodic_decay(s: float) -> float:
    """mu with cosh(mu) = 1 + s/2: G_s decays like exp(-mu |n|) along an
    axis (the slowest direction) for s > 0."""
    return math.acosh(1.0 + 0.5 * s) if s > 0 else 0.0


def periodic_spectrum_applies(N: int, s: float) -> bool:
    """The (2N)-periodic Green's function equals the even embedding of G_s
    on the (2N)^3 box up to the images at distance >= N: its deviation,
    summed over the box, is below (2N)^3 exp(-mu N); the closed form is used
    when that is below 1e-14 (Section 2.2, the sigma > 0 trapezoid rule
    with M = 2N)."""
    return s > 0 and (2 * N) ** 3 * math.exp(-periodic_decay(s) * N) < 1e-14


def periodic_spectrum(N: int, s: float) -> np.ndarray:
    """The real spectrum of the (2N)-periodic Green's function, i.e. the
    2N-point trapezoid rule of the Fourier integral eq. [lgf] read in
    frequency space: 1 / (6 + s - 2 sum_i cos(pi k_i / N)) on the (2N, 2N,
    N + 1) half spectrum (the layout of potentials.lgf_spectrum)."""
    k = np.arange(2 * N)
    c = np.cos(np.pi * k / N)
    c3 = c[: N + 1]
    sym = 6.0 + s - 2.0 * (c[:, None, None] + c[None, :, None] + c3[None, None, :])
    return 1.0 / sym


def periodic_trapezoid(M: int, s: float) -> np.ndarray:
    """The sigma > 0 approximation of Section 2.2: the M-point
    periodic trapezoid rule of the Fourier integral, i.e. an inverse DFT of
    1/(6 + s - 2 sum cos(2 pi p / M)). Returns the M^3 periodic array indexed
    by offset mod M. Accurate only where G_s decays well inside M/2."""
    th = 2.0 * math.pi * np.arange(M) / M
    c = np.cos(th)
    sym = 6.0 + s - 2.0 * (c[:, None, None] + c[None, :, None] + c[None, None, :])
    return np.real(np.fft.ifftn(1.0 / sym))
