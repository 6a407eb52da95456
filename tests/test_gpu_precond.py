"""Restricted additive Schwarz right preconditioning of the inner float32
GMRES (a local form of the right preconditioning remarked in Section 4; the
numerical section asks for preconditioning). It changes the iteration, not
the discrete solution: with and without it the mixed solve reaches the same
u on M+ to the tolerance and matches the oracle's solve, in far fewer
iterations."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as OG
from oracle import solve as OS

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


CASES = [
    ("sphere32", lambda: W.sphere_exp(32), "double"),
    ("sphere32", lambda: W.sphere_exp(32), "single"),
    ("torus64", lambda: W.torus_helmholtz(64, kappa2=10.0), "double"),
    ("star64", lambda: W.star(64, kappa2=1.0), "single"),
]


@pytest.mark.parametrize("name,make,layer", CASES, ids=[f"{c[0]}-{c[2]}" for c in CASES])
def test_precond_same_solution(ctx, name, make, layer):
    import torch
    from paper_2502_05507_gb300 import Problem
    P = make()
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer)
    try:
        g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
        f = torch.from_numpy(P.f()).cuda()
        out = {}
        for pre in (0, 1, 2):   # never, every refinement step, after the first step
            q, u, st = prob.solve(f, g, tol=1e-10, precision="mixed", precond=pre, max_iter=1000)
            assert st["rel_residual"] <= 1e-10, (pre, st)
            out[pre] = (u.cpu().numpy(), st)
        mp = OG.classify(P.phi, P.grid.h, P.grid.origin).inside
        u0 = out[0][0][mp]
        for pre in (1, 2):
            assert np.max(np.abs(out[pre][0][mp] - u0)) <= 1e-8 * np.max(np.abs(u0)), pre
        print(name, layer, "iterations", [out[k][1]["iterations"] for k in (0, 1, 2)])
        # the neighbourhood blocks cut the iterations several times over
        assert out[1][1]["iterations"] < 0.6 * out[0][1]["iterations"], [out[k][1] for k in (0, 1)]
        if name == "sphere32":
            ref = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, layer=layer, tol=1e-12)
            assert np.max(np.abs(out[1][0][mp] - ref.u[mp])) <= 1e-8 * np.max(np.abs(ref.u[mp]))
    finally:
        prob.close()


def test_precond_batched_equals_alone(ctx):
    # the preconditioned inner solves keep batch items independent
    import torch
    from paper_2502_05507_gb300 import Problem
    P = W.torus_helmholtz(32, kappa2=10.0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
    try:
        xyz = np.asarray(prob.boundary_points())
        G = np.stack([P.g_at(xyz), np.cos(xyz[:, 0] + 2 * xyz[:, 2])])
        F = np.stack([P.f(), np.zeros_like(P.f())])
        qb, ub, stb = prob.solve_batched(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), tol=1e-10,
                                         precision="mixed", precond=1)
        for b in range(2):
            q1, u1, st1 = prob.solve(torch.from_numpy(F[b]).cuda(), torch.from_numpy(G[b]).cuda(), tol=1e-10,
                                     precision="mixed", precond=1)
            assert np.array_equal(ub[b].cpu().numpy(), u1.cpu().numpy()), b
            assert stb[b]["iterations"] == st1["iterations"]
    finally:
        prob.close()


def test_problems_destroyed_while_their_rows_build(ctx):
    # the Schwarz rows start on a side stream at problem creation: problems
    # closed at once, or solved without them (float64), must leave the
    # context usable and the next preconditioned solve unchanged
    import torch
    from paper_2502_05507_gb300 import Problem
    P = W.torus_helmholtz(64, kappa2=10.0)
    phi = torch.from_numpy(P.phi).cuda()
    f = torch.from_numpy(P.f()).cuda()
    for _ in range(8):
        Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double").close()
    prob = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    _, u64, st64 = prob.solve(f, g, tol=1e-10, precision="fp64")
    prob.close()
    outs = []
    for _ in range(2):
        prob = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
        _, u, st = prob.solve(f, g, tol=1e-10, precision="mixed", precond=1)
        outs.append((u.cpu().numpy(), st))
        prob.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1]["iterations"] == outs[1][1]["iterations"]
    assert np.max(np.abs(outs[0][0] - u64.cpu().numpy())) <= 1e-8 * np.max(np.abs(u64.cpu().numpy()))
