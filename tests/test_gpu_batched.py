"""Batched solves (64 right-hand sides on one problem, one batched
convolution per GMRES step): every result equals the same right-hand side
solved alone, two of them are checked against the oracle, all reach the
tolerance. Workload: Poisson on the N = 128 torus, u_k = exp(a_k . x) with
seeded unit directions a_k."""
import numpy as np
import pytest

import workloads as W
from oracle import lgf as OL
from oracle import potentials as OP
from oracle import solve as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def batch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context, Problem
    dirs = W.torus_batch_dirs(64, seed=3)
    probs = [W.torus_poisson_dir(128, a) for a in dirs]
    ctx = Context(0)
    P0 = probs[0]
    prob = Problem(ctx, torch.from_numpy(P0.phi).cuda(), P0.grid.h, P0.grid.origin, 0.0, "double")
    xs = prob.boundary_points()
    f = torch.from_numpy(np.stack([P.f() for P in probs])).cuda()
    g = torch.from_numpy(np.stack([P.g_at(xs) for P in probs])).cuda()
    yield dict(ctx=ctx, prob=prob, probs=probs, f=f, g=g, xs=xs)
    prob.close()
    ctx.close()


@pytest.mark.parametrize("precision", ["mixed"])
def test_batched_equals_alone(batch, precision):
    prob, f, g = batch["prob"], batch["f"], batch["g"]
    qb, ub, stb = prob.solve_batched(f, g, tol=1e-10, precision=precision)
    assert all(s["rel_residual"] <= 1e-10 for s in stb)
    for k in (0, 17, 63):
        q1, u1, st1 = prob.solve(f[k], g[k], tol=1e-10, precision=precision)
        assert np.array_equal(q1.cpu().numpy(), qb[k].cpu().numpy()), k
        assert np.array_equal(u1.cpu().numpy(), ub[k].cpu().numpy()), k
        assert st1["iterations"] == stb[k]["iterations"]
    batch["ub"] = ub


def test_batched_against_oracle(batch):
    if "ub" not in batch:
        pytest.skip("batched solve did not run")
    probs, ub = batch["probs"], batch["ub"]
    P0 = probs[0]
    spec = OP.lgf_spectrum(OL.LGFTable(128, 0.0))
    for k in (5, 40):
        P = probs[k]
        ref = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, 0.0, layer="double", tol=1e-12,
                       potential="fft", spectrum=spec, workers=-1)
        u = ub[k].cpu().numpy()
        mp = ref.cls.inside
        e = np.max(np.abs(u[mp] - ref.u[mp])) / np.max(np.abs(ref.u[mp]))
        assert e <= 1e-8, (k, e)
