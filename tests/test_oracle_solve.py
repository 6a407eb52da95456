"""Pins of the oracle's whole solve (Algorithm 1): route A (LGF + GMRES)
against route B (sparse FD), second-order convergence, and the paper's
error tables."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import solve as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tables():
    out = {}
    with open(os.path.join(GOLDEN, "paper_tables.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                t, N, e, _ = line.split()
                out[(t, int(N))] = float(e)
    return out


def _run(P, layer="double", tol=1e-12, potential="direct"):
    g = P.grid
    return S.solve(P.phi, g.h, g.origin, P.f(), P.g_at, P.kappa2, layer=layer, tol=tol, potential=potential)


@pytest.mark.parametrize("make,layer", [
    (lambda: W.sphere_exp(16), "double"),
    (lambda: W.sphere_exp(16), "single"),
    (lambda: W.torus_helmholtz(24, kappa2=10.0), "double"),
    (lambda: W.star(20), "double"),
])
def test_route_a_equals_route_b(make, layer):
    P = make()
    r = _run(P, layer=layer)
    ufd, cls = S.solve_fd(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2)
    m = cls.nplus
    assert np.max(np.abs(r.u[m] - ufd[m])) < 1e-9 * np.max(np.abs(ufd[m]))
    # the closure rows hold for the reconstructed u
    uf = r.u.reshape(-1)
    row = cls.t * uf[cls.gm_idx] + (1 - cls.t) * uf[cls.partner]
    assert np.max(np.abs(row - P.g_at(cls.xstar))) < 1e-9 * np.max(np.abs(uf))


def test_fft_route_equals_direct_route():
    P = W.torus_helmholtz(16, kappa2=10.0)
    a = _run(P)
    b = _run(P, potential="fft")
    assert a.iterations == b.iterations
    assert np.max(np.abs(a.q - b.q)) < 1e-10 * np.max(np.abs(a.q))


def test_second_order_convergence():
    errs = []
    for N in (16, 32, 64):
        P = W.sphere_exp(N)
        u, cls = S.solve_fd(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2)
        errs.append(np.max(np.abs(u[cls.inside] - P.u_exact()[cls.inside])))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 1.7) & (rates < 2.4)), rates


@pytest.mark.parametrize("table,make", [("table1", W.paper_ellipsoid), ("table2", W.paper_torus)])
def test_paper_error_tables(table, make):
    # The closure is a reading (oracle/grid.py): it reproduces the printed
    # max errors of Tables 1 and 2 to within 14% (ellipsoid 1.50e-3 / 3.66e-4,
    # torus 7.94e-5 / 2.22e-5); 20% is the bar here.
    ref = _tables()
    errs = []
    for N in (31, 63):
        P = make(N)
        u, cls = S.solve_fd(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2)
        e = np.max(np.abs(u[cls.inside] - P.u_exact()[cls.inside]))
        errs.append(e)
        assert e == pytest.approx(ref[(table, N)], rel=0.2)
    assert 1.7 < np.log2(errs[0] / errs[1]) < 2.3
