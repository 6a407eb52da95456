"""Direct formulation on the GPU (eq. [direct_sys] with eq. [inhom]; the
difference potentials of eq. [dp]; eq. [discrete_green]) against the oracle
(oracle/direct.py) and the sparse finite-difference solve (oracle/fd.py)."""
import numpy as np
import pytest

import workloads as W
from oracle import direct as D
from oracle import fd, grid, lgf, potentials as pot

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


def _problem(ctx, P):
    import torch
    from paper_2502_05507_gb300 import Problem
    return Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "direct")


CASES = [lambda: W.sphere_exp(16, radius=0.55, kappa2=10.0), lambda: W.torus_helmholtz(32, kappa2=10.0),
         lambda: W.star(32, kappa2=1.0)]


@pytest.mark.parametrize("make", CASES)
def test_gamma_plus_and_unknowns(ctx, make):
    P = make()
    prob = _problem(ctx, P)
    try:
        cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
        assert np.array_equal(prob.gamma_plus(), cls.gp_idx)
        assert np.array_equal(prob.interior_mask(), cls.inside)
        assert prob.n_unknowns == cls.gm_idx.size + cls.gp_idx.size
    finally:
        prob.close()


@pytest.mark.parametrize("make", CASES)
def test_direct_apply_matches_oracle(ctx, make):
    P = make()
    g = P.grid
    s = P.kappa2 * g.h * g.h
    cls = grid.classify(P.phi, g.h, g.origin)
    spec = pot.lgf_spectrum(lgf.LGFTable(g.N, s))
    prob = _problem(ctx, P)
    try:
        rng = np.random.default_rng(11)
        w = rng.standard_normal(prob.n_unknowns)
        ref = D.apply(cls, w, s, spec)
        got = prob.boundary_apply(w, precision="fp64")
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
        got32 = prob.boundary_apply(w, precision="fp32")
        assert np.max(np.abs(got32 - ref)) <= 2e-5 * np.max(np.abs(ref))
        # the difference potential itself, on the whole grid
        pw = D.difference_potential(cls, w, s, spec).reshape((g.N,) * 3)
        v = prob.potential_apply(w, precision="fp64")
        assert np.max(np.abs(v - pw)) <= 1e-12 * np.max(np.abs(pw))
    finally:
        prob.close()


@pytest.mark.parametrize("make", [lambda: W.sphere_exp(32), lambda: W.torus_helmholtz(64, kappa2=10.0)])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_direct_solve_matches_fd(ctx, make, precision):
    import torch
    P = make()
    g = P.grid
    prob = _problem(ctx, P)
    try:
        cls = grid.classify(P.phi, g.h, g.origin)
        gv = P.g_at(np.asarray(prob.boundary_points()))
        q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), torch.from_numpy(gv).cuda(), tol=1e-10,
                              precision=precision, max_iter=2000)
        assert st["rel_residual"] <= 1e-10, st
        ufd = fd.solve_fd(cls, P.f(), gv, g.h, P.kappa2 * g.h * g.h)
        m = cls.nplus
        u = u.cpu().numpy()
        assert np.max(np.abs(u[m] - ufd[m])) <= 1e-8 * np.max(np.abs(ufd[m])), st
        assert np.all(u[~m] == 0.0)
        # the unknown is u on gamma
        qn = q.cpu().numpy()
        assert np.max(np.abs(qn - ufd.reshape(-1)[D.unknown_nodes(cls)])) <= 1e-8 * np.max(np.abs(ufd[m]))
        print(g.N, precision, st)
    finally:
        prob.close()


def test_direct_full_size_equals_double_layer(ctx):
    # the torus N=128 workload: both formulations solve the same discrete
    # problem (eq. [discrete] with the closure), so u agrees on N+
    import torch
    from paper_2502_05507_gb300 import Problem
    P = W.torus_helmholtz(128, kappa2=10.0)
    phi = torch.from_numpy(P.phi).cuda()
    f = torch.from_numpy(P.f()).cuda()
    pd = _problem(ctx, P)
    pl = Problem(ctx, phi, P.grid.h, P.grid.origin, P.kappa2, "double")
    try:
        gv = torch.from_numpy(P.g_at(np.asarray(pd.boundary_points()))).cuda()
        # residual 1e-12: each solution is then within cond(A) 1e-12 of the
        # discrete solution (at 1e-10 the direct one differed by 1.6e-8)
        _, ud, std = pd.solve(f, gv, tol=1e-12, precision="mixed", max_iter=4000)
        _, ul, stl = pl.solve(f, gv, tol=1e-12, precision="mixed")
        ud, ul = ud.cpu().numpy(), ul.cpu().numpy()
        assert std["rel_residual"] <= 1e-12 and stl["rel_residual"] <= 1e-12
        assert np.max(np.abs(ud - ul)) <= 1e-8 * np.max(np.abs(ul)), (std, stl)
        print("direct", std, "double", stl)
    finally:
        pd.close()
        pl.close()


def test_direct_batched_equals_alone(ctx):
    import torch
    P = W.torus_helmholtz(32, kappa2=10.0)
    prob = _problem(ctx, P)
    try:
        xyz = np.asarray(prob.boundary_points())
        G = np.stack([P.g_at(xyz), np.cos(xyz[:, 0] + 2 * xyz[:, 2])])
        F = np.stack([P.f(), np.zeros_like(P.f())])
        qb, ub, stb = prob.solve_batched(torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda(), tol=1e-10,
                                         precision="mixed")
        for b in range(2):
            q1, u1, st1 = prob.solve(torch.from_numpy(F[b]).cuda(), torch.from_numpy(G[b]).cuda(), tol=1e-10,
                                     precision="mixed")
            assert np.array_equal(ub[b].cpu().numpy(), u1.cpu().numpy()), b
            assert stb[b]["iterations"] == st1["iterations"]
    finally:
        prob.close()


def test_direct_precond_same_solution_fewer_iterations(ctx):
    # Schwarz blocks of the direct system (closure rows t, 1 - t; gamma+ rows
    # delta - P): the same solution in far fewer inner iterations
    import torch
    P = W.torus_helmholtz(64, kappa2=10.0)
    prob = _problem(ctx, P)
    try:
        gv = torch.from_numpy(P.g_at(np.asarray(prob.boundary_points()))).cuda()
        f = torch.from_numpy(P.f()).cuda()
        _, u0, s0 = prob.solve(f, gv, tol=1e-10, precision="mixed", precond=0, max_iter=2000)
        _, u1, s1 = prob.solve(f, gv, tol=1e-10, precision="mixed", precond=1, max_iter=2000)
        assert s1["rel_residual"] <= 1e-10
        u0, u1 = u0.cpu().numpy(), u1.cpu().numpy()
        assert np.max(np.abs(u1 - u0)) <= 1e-8 * np.max(np.abs(u0))
        assert s1["iterations"] < 0.5 * s0["iterations"], (s0, s1)
        print("direct precond", s0["iterations"], "->", s1["iterations"])
    finally:
        prob.close()
