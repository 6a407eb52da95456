"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds geometry and manufactured solutions only: level-set samples
phi on a cell-centred grid, exact solutions u, right-hand sides f in the
paper's sign convention (-Lap u + sigma u = f, Section 2, eq. (2.1)), and the
seeded random draws of the batched and serving workloads. It contains none of
the BAE method's arithmetic, so both the CUDA path and the CPU oracle may
import it.

Grid convention: node (i, j, k) sits at origin + (i, j, k) * h, C-order with k
fastest. For the box [lo, hi]^3 split into N cells per side the nodes are the
cell centres, origin = lo + h/2, h = (hi - lo)/N (the numerical section's
"N^3 degrees of freedom" on [-1-l, 1+l]^3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Grid:
    N: int
    h: float
    origin: float  # coordinate of node 0 on every axis

    def axis(self) -> np.ndarray:
        return self.origin + np.arange(self.N, dtype=np.float64) * self.h

    def mesh(self):
        a = self.axis()
        return np.meshgrid(a, a, a, indexing="ij")


def cell_centred(N: int, lo: float = -1.0, hi: float = 1.0) -> Grid:
    h = (hi - lo) / N
    return Grid(N=N, h=h, origin=lo + 0.5 * h)


# ---------------------------------------------------------------- geometries

def phi_sphere(x, y, z, radius=0.6, center=(0.0, 0.0, 0.0)):
    return (x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2 - radius ** 2


def phi_ellipsoid(x, y, z, a=1.0, b=0.8, c=0.4):
    return x ** 2 / a ** 2 + y ** 2 / b ** 2 + z ** 2 / c ** 2 - 1.0


def phi_torus(x, y, z, R=0.5, r=0.2):
    return (np.sqrt(x ** 2 + y ** 2) - R) ** 2 + z ** 2 - r ** 2


def phi_star(x, y, z, r0=0.6, amp=0.1, m_theta=5, m_phi=3):
    """Star-shaped body r = r0 + amp sin(m_theta theta) cos(m_phi varphi),
    theta the polar angle acos(z/r), varphi = atan2(y, x)."""
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    rs = np.where(r > 0, r, 1.0)
    theta = np.arccos(np.clip(z / rs, -1.0, 1.0))
    varphi = np.arctan2(y, x)
    return r - (r0 + amp * np.sin(m_theta * theta) * np.cos(m_phi * varphi))


# -------------------------------------------------------- exact solutions
# Each returns (u, f) where f is the right-hand side in the paper's sign,
# -Lap u + kappa2 u = f.

def sol_exp_sum(x, y, z, kappa2=0.0):
    u = np.exp(x + y + z)
    return u, (-3.0 + kappa2) * u


def sol_sin2x_cosy_expz(x, y, z, kappa2=10.0):
    u = np.sin(2 * x) * np.cos(y) * np.exp(z)
    return u, (4.0 + kappa2) * u


def sol_exp_dir(x, y, z, a, kappa2=0.0):
    a = np.asarray(a, dtype=np.float64)
    u = np.exp(a[0] * x + a[1] * y + a[2] * z)
    return u, (-float(a @ a) + kappa2) * u


def sol_quadratic(x, y, z, kappa2=0.0):
    u = x ** 2 + y ** 2 + z ** 2
    return u, -6.0 + kappa2 * u


def sol_sinx_cosy_sinz(x, y, z, kappa2=10.0):
    u = np.sin(x) * np.cos(y) * np.sin(z)
    return u, (3.0 + kappa2) * u


# ----------------------------------------------------------- problem sets

@dataclasses.dataclass
class Problem:
    """One synthetic Dirichlet problem: grid, phi samples, kappa^2, the exact
    solution as a callable, and f on every node (paper sign)."""
    name: str
    grid: Grid
    phi: np.ndarray
    kappa2: float
    layer: str
    exact: callable  # exact(x, y, z) -> (u, f)

    def f(self) -> np.ndarray:
        X, Y, Z = self.grid.mesh()
        return np.ascontiguousarray(self.exact(X, Y, Z)[1], dtype=np.float64)

    def u_exact(self) -> np.ndarray:
        X, Y, Z = self.grid.mesh()
        return self.exact(X, Y, Z)[0]

    def g_at(self, xyz: np.ndarray) -> np.ndarray:
        xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
        return np.ascontiguousarray(self.exact(xyz[:, 0], xyz[:, 1], xyz[:, 2])[0])


def _make(name, grid, phifn, kappa2, layer, exact):
    X, Y, Z = grid.mesh()
    phi = np.ascontiguousarray(phifn(X, Y, Z), dtype=np.float64)
    return Problem(name=name, grid=grid, phi=phi, kappa2=float(kappa2), layer=layer, exact=exact)


def sphere_exp(N=32, radius=0.6, kappa2=0.0, layer="double"):
    """Poisson, sphere of radius 0.6 in [-1,1]^3, u = exp(x+y+z)."""
    return _make(f"sphere{radius}_N{N}", cell_centred(N), lambda x, y, z: phi_sphere(x, y, z, radius),
                 kappa2, layer, lambda x, y, z: sol_exp_sum(x, y, z, kappa2))


def torus_helmholtz(N=128, kappa2=10.0, layer="double", R=0.5, r=0.2):
    """Modified Helmholtz kappa^2 = 10, torus R=0.5, r=0.2 in [-1,1]^3,
    u = sin(2x) cos(y) exp(z)."""
    return _make(f"torus_N{N}_k{kappa2:g}", cell_centred(N), lambda x, y, z: phi_torus(x, y, z, R, r),
                 kappa2, layer, lambda x, y, z: sol_sin2x_cosy_expz(x, y, z, kappa2))


def torus_batch_dirs(nrhs=64, seed=3):
    """Unit directions a_k of the batched workload u_k = exp(a_k . x)."""
    a = np.random.default_rng(seed).standard_normal((nrhs, 3))
    return a / np.linalg.norm(a, axis=1, keepdims=True)


def torus_poisson_dir(N, a, layer="double"):
    a = np.asarray(a, dtype=np.float64)
    return _make(f"torus_N{N}_dir", cell_centred(N), phi_torus, 0.0, layer,
                 lambda x, y, z: sol_exp_dir(x, y, z, a, 0.0))


def star(N=256, kappa2=0.0, layer="double"):
    a = np.array([1.0, 1.0, 1.0]) / math.sqrt(3.0)
    return _make(f"star_N{N}_k{kappa2:g}", cell_centred(N), phi_star, kappa2, layer,
                 lambda x, y, z: sol_exp_dir(x, y, z, a, kappa2))


def paper_ellipsoid(N=31, layer="double"):
    """Poisson in the ellipsoid (1, 0.8, 0.4), box [-1.25, 1.25]^3,
    u = x^2 + y^2 + z^2 (numerical section, first experiment)."""
    return _make(f"ellipsoid_N{N}", cell_centred(N, -1.25, 1.25), phi_ellipsoid, 0.0, layer,
                 lambda x, y, z: sol_quadratic(x, y, z, 0.0))


def paper_torus(N=31, layer="double"):
    """Modified Helmholtz sigma = 10 in the torus R=0.6, r=0.3, box
    [-1.1, 1.1]^3, u = sin x cos y sin z (numerical section, second experiment)."""
    return _make(f"ptorus_N{N}", cell_centred(N, -1.1, 1.1), lambda x, y, z: phi_torus(x, y, z, 0.6, 0.3),
                 10.0, layer, lambda x, y, z: sol_sinx_cosy_sinz(x, y, z, 10.0))


def random_density(n, seed=0):
    return np.random.default_rng(seed).standard_normal(n)


def serving_trace(n_requests=2000, seed=5, sizes=(32, 64, 128, 256), kappa2s=(0.0, 10.0)):
    """Request mix of the serving workload: N uniform over `sizes`, kappa^2
    uniform over `kappa2s`, geometry uniform over sphere / ellipsoid / torus
    centred at 0 (sphere radius U[0.3,0.8], ellipsoid semi-axes U[0.3,0.8],
    torus R U[0.35,0.6], r U[0.1,0.25] with R + r <= 0.8), exact solution
    exp(a . x) with a a random unit vector. Returns a list of dicts."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_requests):
        N = int(rng.choice(sizes))
        k2 = float(rng.choice(kappa2s))
        kind = ["sphere", "ellipsoid", "torus"][int(rng.integers(3))]
        if kind == "sphere":
            params = (float(rng.uniform(0.3, 0.8)),)
        elif kind == "ellipsoid":
            params = tuple(float(v) for v in rng.uniform(0.3, 0.8, size=3))
        else:
            while True:
                R, r = float(rng.uniform(0.35, 0.6)), float(rng.uniform(0.1, 0.25))
                if R + r <= 0.8:
                    break
            params = (R, r)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        out.append(dict(N=N, kappa2=k2, kind=kind, params=params, a=a))
    return out


def trace_problem(req, layer="double"):
    N, k2, kind, params, a = req["N"], req["kappa2"], req["kind"], req["params"], req["a"]
    if kind == "sphere":
        fn = lambda x, y, z: phi_sphere(x, y, z, params[0])
    elif kind == "ellipsoid":
        fn = lambda x, y, z: phi_ellipsoid(x, y, z, *params)
    else:
        fn = lambda x, y, z: phi_torus(x, y, z, *params)
    return _make(f"{kind}_N{N}", cell_centred(N), fn, k2, layer,
                 lambda x, y, z: sol_exp_dir(x, y, z, a, k2))


def trace_tensors(req, device="cuda"):
    """phi and f (paper sign) of a serving-trace request as float64 torch
    tensors computed on `device`, with the formulas of trace_problem (for
    benchmarks that must not spend host time evaluating N^3 samples)."""
    import torch
    N, k2, kind, params, a = req["N"], req["kappa2"], req["kind"], req["params"], req["a"]
    g = cell_centred(N)
    ax = g.origin + torch.arange(N, dtype=torch.float64, device=device) * g.h
    x, y, z = ax.view(N, 1, 1), ax.view(1, N, 1), ax.view(1, 1, N)
    if kind == "sphere":
        phi = x * x + y * y + z * z - params[0] ** 2
    elif kind == "ellipsoid":
        phi = x * x / params[0] ** 2 + y * y / params[1] ** 2 + z * z / params[2] ** 2 - 1.0
    else:
        phi = (torch.sqrt(x * x + y * y) - params[0]) ** 2 + z * z - params[1] ** 2
    u = torch.exp(float(a[0]) * x + float(a[1]) * y + float(a[2]) * z)
    f = (-float(np.dot(a, a)) + k2) * u
    return phi.expand(N, N, N).contiguous(), f.expand(N, N, N).contiguous()
