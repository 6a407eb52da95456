"""The finite-box particular solution of Algorithm 1 (eq. [aux] with eq.
[ps]) on the GPU against the oracle:
- bae_box_particular equals oracle.potentials.box_particular (the sine-basis
  solve of the box problem) in float64 and double-float;
- a solve with the box particular solution gives the same u on N+ as the
  free-lattice route (float64, tight tolerance) and as the sparse FD
  solution (mixed precision), with a different density;
- the direct formulation rejects it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fd as OF
from oracle import grid as OG
from oracle import potentials as OP

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context
    c = Context(0)
    yield c
    c.close()


def _problem(ctx, P, layer="double"):
    import torch
    from paper_2502_05507_gb300 import Problem
    return Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer)


@pytest.mark.parametrize("make", [lambda: W.sphere_exp(32), lambda: W.torus_helmholtz(64, kappa2=10.0),
                                  lambda: W.star(64, kappa2=1.0)])
@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_box_particular_matches_oracle(ctx, make, precision):
    import torch
    P = make()
    prob = _problem(ctx, P)
    got = prob.box_particular(torch.from_numpy(P.f()).cuda(), precision).cpu().numpy()
    ref = OP.box_particular(P.f(), P.grid.h, P.kappa2 * P.grid.h ** 2, P.phi < 0)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    prob.close()


def test_box_route_solution_equals_lattice_route(ctx):
    import torch
    P = W.torus_helmholtz(64, kappa2=10.0)
    prob = _problem(ctx, P)
    g = torch.from_numpy(P.g_at(np.asarray(prob.boundary_points()))).cuda()
    f = torch.from_numpy(P.f()).cuda()
    qb, ub, stb = prob.solve(f, g, tol=1e-13, precision="fp64", particular="box", max_iter=1000)
    ql, ul, stl = prob.solve(f, g, tol=1e-13, precision="fp64", max_iter=1000)
    m = P.phi < 0
    ub, ul = ub.cpu().numpy(), ul.cpu().numpy()
    assert np.max(np.abs(ub[m] - ul[m])) <= 1e-12 * np.max(np.abs(ul[m]))
    qb, ql = qb.cpu().numpy(), ql.cpu().numpy()
    assert np.max(np.abs(qb - ql)) > 1e-6 * np.max(np.abs(ql))       # the densities differ
    # mixed precision with the box particular solution: the FD solution
    q, u, st = prob.solve(f, g, tol=1e-10, precision="mixed", particular="box")
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    ref = OF.solve_fd(cls, P.f(), P.g_at(cls.xstar), P.grid.h, P.kappa2 * P.grid.h ** 2)
    n = cls.nplus
    u = u.cpu().numpy()
    assert np.max(np.abs(u[n] - ref[n])) <= 1e-8 * np.max(np.abs(ref[n]))
    assert st["rel_residual"] <= 1e-10
    prob.close()


def test_box_particular_rejected_for_direct_formulation(ctx):
    import torch
    from paper_2502_05507_gb300 import BAEError
    P = W.sphere_exp(16, radius=0.55)
    prob = _problem(ctx, P, "direct")
    g = torch.from_numpy(P.g_at(np.asarray(prob.boundary_points()))).cuda()
    with pytest.raises(BAEError):
        prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision="mixed", particular="box")
    prob.close()
