"""GPU parity at the benchmark's full size (N = 128 torus, kappa^2 = 10,
double layer), in the configuration bench.py times: the potential apply
against the oracle's FFT convolution with the oracle's own LGF table,
sampled outputs against direct sums, and the full solve (float64 and
mixed precision) against the oracle's solve."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as OG
from oracle import lgf as OL
from oracle import potentials as OP
from oracle import solve as OS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context, Problem
    P = W.torus_helmholtz(128, kappa2=10.0)
    s = P.kappa2 * P.grid.h ** 2
    table = OL.LGFTable(128, s)
    spec = OP.lgf_spectrum(table)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    ctx = Context(0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
    yield dict(P=P, table=table, spec=spec, cls=cls, ctx=ctx, prob=prob)
    prob.close()
    ctx.close()


def test_apply_full_size(setup):
    import torch
    P, cls, spec, prob = setup["P"], setup["cls"], setup["spec"], setup["prob"]
    q = W.random_density(cls.gm_idx.size, seed=21)
    ref = OP.fft_convolve(OP.source_density(cls, q, "double"), spectrum=spec, workers=-1)
    scale = np.max(np.abs(ref))
    v = prob.potential_apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert np.max(np.abs(v - ref)) <= 1e-12 * scale
    v32 = prob.potential_apply(torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    assert np.max(np.abs(v32 - ref)) <= 2e-6 * scale
    vds = prob.potential_apply(torch.from_numpy(q).cuda(), "df64").cpu().numpy()
    assert np.max(np.abs(vds - ref)) <= 1e-12 * scale


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-6), ("fp64", 1e-12), ("df64", 1e-12)])
def test_apply_full_size_each_schedule(setup, precision, tol):
    # the five-pass schedule, its second launch geometry (float32: half-width
    # column blocks) and the plane-fused one (one CTA per plane for float32,
    # a two-CTA cluster sharing the plane for the 16-byte types)
    import torch
    from paper_2502_05507_gb300 import set_conv_schedule
    P, cls, spec, prob = setup["P"], setup["cls"], setup["spec"], setup["prob"]
    q = W.random_density(cls.gm_idx.size, seed=23)
    ref = OP.fft_convolve(OP.source_density(cls, q, "double"), spectrum=spec, workers=-1)
    scale = np.max(np.abs(ref))
    try:
        for name in ("passes", "passes_alt", "persist", "plane"):
            set_conv_schedule(name)
            v = prob.potential_apply(torch.from_numpy(q).cuda(), precision).cpu().numpy()
            assert np.max(np.abs(v - ref)) <= tol * scale, name
    finally:
        set_conv_schedule("auto")


def test_apply_full_size_sampled_direct_sum(setup):
    # a sparse density: the oracle sums G(m - x) rho(x) term by term at
    # sampled targets, with G from the oracle's table
    import torch
    P, cls, table, prob = setup["P"], setup["cls"], setup["table"], setup["prob"]
    rng = np.random.default_rng(22)
    q = np.zeros(cls.gm_idx.size)
    q[rng.choice(q.size, 6, replace=False)] = rng.standard_normal(6)
    tg = np.concatenate([rng.choice(np.flatnonzero(cls.nplus), 30, replace=False), cls.gm_idx[:5]])
    ref = OP.direct_potential(table, cls, q, tg, "double")
    v = prob.potential_apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy().reshape(-1)[tg]
    assert np.max(np.abs(v - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("precision", ["mixed", "fp64", "df64"])
def test_solve_full_size(setup, precision):
    import torch
    P, spec, prob = setup["P"], setup["spec"], setup["prob"]
    if "ref" not in setup:
        setup["ref"] = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, layer="double",
                                tol=1e-12, potential="fft", spectrum=spec, workers=-1)
    ref = setup["ref"]
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision=precision)
    u = u.cpu().numpy()
    mp = ref.cls.inside
    e_mp = np.max(np.abs(u[mp] - ref.u[mp])) / np.max(np.abs(ref.u[mp]))
    info = dict(e_mp=e_mp, **st, oracle_iters=ref.iterations)
    print(info)
    assert e_mp <= 1e-8, info
    assert st["rel_residual"] <= 1e-10, info
    # second-order discretisation error against the exact solution
    err = np.max(np.abs(u[mp] - P.u_exact()[mp]))
    assert err < 1e-3, err
