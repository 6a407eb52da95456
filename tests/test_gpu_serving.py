"""The solve server: a mix of requests (different N, kappa^2, geometry)
submitted at once to a few slots. Requests are admitted as slots free up,
their device work overlaps, and each result equals the same request solved
alone on a fresh context (bit for bit: the kernels and reductions do not
depend on what else is in flight)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _alone(P, precision):
    import torch
    from paper_2502_05507_gb300 import Context, Problem
    ctx = Context(0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, P.layer)
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision=precision)
    out = (q.cpu().numpy(), u.cpu().numpy(), st)
    prob.close()
    ctx.close()
    return out


@pytest.mark.parametrize("slots,budget", [(3, 64 << 30), (4, 1 << 20)])
def test_server_mix_equals_alone(slots, budget):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Server
    reqs = W.serving_trace(8, seed=5, sizes=(32, 64))
    probs = [W.trace_problem(r) for r in reqs]
    srv = Server(0, slots=slots, hbm_budget_bytes=budget)
    tickets = [srv.submit(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, kappa2=P.kappa2, precision="mixed")
               for P in probs]
    res = [srv.poll(t) for t in tickets]
    dens = [srv.density(t) for t in tickets]
    for P, r, d in zip(probs, res, dens):
        assert r["status"] == 0, r
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        q1, u1, st1 = _alone(P, "mixed")
        assert np.array_equal(r["u"], u1)
        assert np.array_equal(d, q1)
        assert r["stats"]["iterations"] == st1["iterations"]
        assert r["stats"]["rel_residual"] <= 1e-10
    spans = sorted((r["t_admit"], r["t_done"]) for r in res)
    overlaps = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    if budget >= (1 << 30):
        assert overlaps >= 1          # work of different requests overlapped
        assert max(r["t_admit"] - r["t_submit"] for r in res) > 0   # some waited for a slot
    else:
        assert overlaps == 0          # a tiny budget admits one request at a time
    for t in tickets:
        srv.release(t)
    srv.close()


def test_server_direct_formulation_equals_alone():
    # a direct-formulation request: its density is u on gamma- then gamma+
    # (n_gm + n_gp values) and the result matches the same solve alone
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context, Problem, Server
    P = W.torus_helmholtz(32, kappa2=10.0)
    srv = Server(0, slots=2, hbm_budget_bytes=64 << 30)
    t = srv.submit(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, kappa2=P.kappa2, layer="direct",
                   precision="mixed")
    r = srv.poll(t)
    d = srv.density(t)
    assert r["status"] == 0, r
    ctx = Context(0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "direct")
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    q1, u1, st1 = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision="mixed")
    assert d.size == prob.n_unknowns == prob.n_gm + prob.n_gp
    assert np.array_equal(d, q1.cpu().numpy())
    assert np.array_equal(r["u"], u1.cpu().numpy())
    prob.close()
    ctx.close()
    srv.release(t)
    srv.close()
