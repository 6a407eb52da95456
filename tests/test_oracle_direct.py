"""Pins of the oracle's direct formulation (eq. [direct_sys] with eq. [inhom],
difference potentials eq. [dp], discrete Green's formula eq.
[discrete_green]) against things other than itself:

* the Green's formula of the Theorem: a solution of the discrete problem
  (the sparse FD route, no LGF) equals u_p + P u_gamma on all of M+, so it
  solves the gamma+ rows of the direct system exactly;
* the direct solve reproduces the sparse FD solution on N+;
* the matrix-free apply equals its dense column-by-column assembly, and a
  dense solve of that matrix gives the FD solution to rounding.
"""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import fd, grid, lgf, potentials as pot


def _setup(P):
    g = P.grid
    s = P.kappa2 * g.h * g.h
    cls = grid.classify(P.phi, g.h, g.origin)
    spec = pot.lgf_spectrum(lgf.LGFTable(g.N, s))
    return cls, s, spec


@pytest.mark.parametrize("make", [lambda: W.sphere_exp(16), lambda: W.torus_helmholtz(20, kappa2=10.0),
                                  lambda: W.star(20, kappa2=1.0)])
def test_green_formula_on_fd_solution(make):
    P = make()
    cls, s, spec = _setup(P)
    g = P.g_at(cls.xstar)
    ufd = fd.solve_fd(cls, P.f(), g, P.grid.h, s).reshape(-1)
    w = ufd[D.unknown_nodes(cls)]
    up = D.particular(cls, P.f(), P.grid.h, spec)
    pw = D.difference_potential(cls, w, s, spec)
    scale = np.max(np.abs(ufd))
    # u = u_p + P u_gamma on M+ (eq. [discrete_green])
    assert np.max(np.abs(up[cls.mp_idx] + pw[cls.mp_idx] - ufd[cls.mp_idx])) < 1e-11 * scale
    # hence every row of the direct system holds for the FD solution
    res = D.apply(cls, w, s, spec) - D.rhs(cls, g, up)
    assert np.max(np.abs(res)) < 1e-11 * scale


def test_green_formula_fails_for_a_non_solution():
    # the identity is not automatic: perturb the FD solution at one gamma- node
    P = W.sphere_exp(16)
    cls, s, spec = _setup(P)
    g = P.g_at(cls.xstar)
    ufd = fd.solve_fd(cls, P.f(), g, P.grid.h, s).reshape(-1)
    w = ufd[D.unknown_nodes(cls)].copy()
    w[3] += 1e-3
    res = D.apply(cls, w, s, spec) - D.rhs(cls, g, D.particular(cls, P.f(), P.grid.h, spec))
    assert np.max(np.abs(res[cls.gm_idx.size:])) > 1e-6


@pytest.mark.parametrize("make", [lambda: W.sphere_exp(16), lambda: W.torus_helmholtz(24, kappa2=10.0)])
def test_direct_solve_equals_fd(make):
    P = make()
    g = P.grid
    u, w, iters = D.solve(P.phi, g.h, g.origin, P.f(), P.g_at, P.kappa2, tol=1e-12)
    cls = grid.classify(P.phi, g.h, g.origin)
    ufd = fd.solve_fd(cls, P.f(), P.g_at(cls.xstar), g.h, P.kappa2 * g.h * g.h)
    m = cls.nplus
    assert np.max(np.abs(u[m] - ufd[m])) < 1e-9 * np.max(np.abs(ufd[m]))
    assert 0 < iters < w.size


def test_apply_equals_dense_assembly_and_dense_solve():
    P = W.sphere_exp(8, radius=0.6)
    cls, s, spec = _setup(P)
    n = cls.gm_idx.size + cls.gp_idx.size
    A = np.stack([D.apply(cls, e, s, spec) for e in np.eye(n)], axis=1)
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n)
    assert np.allclose(A @ x, D.apply(cls, x, s, spec), rtol=0, atol=1e-12 * np.max(np.abs(A)) * n)
    # the gamma- rows are the closure: two entries, t and 1 - t
    nm = cls.gm_idx.size
    assert np.array_equal(np.count_nonzero(A[:nm], axis=1), np.where(cls.t < 1.0, 2, 1))
    g = P.g_at(cls.xstar)
    up = D.particular(cls, P.f(), P.grid.h, spec)
    w = np.linalg.solve(A, D.rhs(cls, g, up))
    u = D.reconstruct(cls, w, s, up, spec)
    ufd = fd.solve_fd(cls, P.f(), g, P.grid.h, s)
    m = cls.nplus
    assert np.max(np.abs(u[m] - ufd[m])) < 1e-11 * np.max(np.abs(ufd[m]))
