"""GPU parity of every hot-path step against the CPU oracle, through the C
ABI, at sizes the oracle finishes in seconds (several FFT tiles, ragged
column tails). Tolerances: bit-exact for classification and closure; LGF
table 1e-13 relative (+1e-17 absolute); float64 potential apply 1e-12
relative to max|v|; float32 apply 2e-6; solutions 1e-8 relative at GMRES
tolerance 1e-10."""
import numpy as np
import pytest

import workloads as W
from oracle import grid as OG
from oracle import lgf as OL
from oracle import potentials as OP
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


def _problem(ctx, P, layer=None):
    import torch
    from paper_2502_05507_gb300 import Problem
    return Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer or P.layer)


# --------------------------------------------------------------- a2: LGF
@pytest.mark.parametrize("N,s", [(16, 0.0), (32, 0.0), (32, 10.0 / 4096.0), (24, 1.0), (20, 100.0 / 16384.0),
                                 (12, 30.0)])
def test_lgf_table_matches_oracle(ctx, N, s):
    got = ctx.lgf_table(N, s)
    ref = OL.lgf_triples(OL.sorted_triples(N), s)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-17)


def test_lgf_table_full_size_sampled(ctx):
    # N = 256 (the largest grid), sampled entries against per-entry quadrature
    for s in (0.0, 1.0 / 16384.0):
        got = ctx.lgf_table(256, s)
        tri = OL.sorted_triples(256)
        rng = np.random.default_rng(11)
        idx = np.concatenate([[0, 1, len(tri) - 1], rng.choice(len(tri), 40, replace=False)])
        for i in idx:
            ref = OL.lgf_entry(tuple(tri[i]), s)
            assert abs(got[i] - ref) <= 1e-13 * abs(ref) + 1e-17, (tri[i], got[i], ref)


@pytest.mark.parametrize("N,s", [(8, 0.0), (16, 10.0 / 256.0), (32, 0.0), (16, 25.0), (32, 9.0)])
def test_lgf_spectrum_matches_oracle(ctx, N, s):
    # (16, 25) and (32, 9): the closed-form periodic spectrum on the GPU
    # against the spectrum of the oracle's Bessel table
    got = ctx.lgf_spectrum(N, s)
    ref = OP.lgf_spectrum(OL.LGFTable(N, s))[: N + 1, : N + 1, :]
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


# --------------------------------------------------------- a1: classify
@pytest.mark.parametrize("make", [lambda: W.sphere_exp(32), lambda: W.torus_helmholtz(64), lambda: W.star(64),
                                  lambda: W.paper_ellipsoid(32), lambda: W.torus_helmholtz(128),
                                  lambda: W.star(256)])
def test_classification_bit_exact(ctx, make):
    P = make()
    prob = _problem(ctx, P)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    c = prob.classification()
    fl = c["flags"]
    assert np.array_equal(fl & 1 != 0, cls.inside)
    assert np.array_equal(fl & 2 != 0, cls.gm)
    assert np.array_equal(fl & 4 != 0, cls.gp)
    assert np.array_equal(fl & 8 != 0, cls.dnode)
    assert np.array_equal((fl >> 4).astype(np.int64) * cls.gm, cls.count * cls.gm)
    assert np.array_equal(c["gm"], cls.gm_idx)
    assert np.array_equal(c["partner"], cls.partner)
    assert np.array_equal(c["t"], cls.t)
    xs = prob.boundary_points()
    assert np.array_equal(xs, cls.xstar)
    assert (prob.n_gm, prob.n_gp, prob.n_mp) == (cls.gm_idx.size, cls.gp_idx.size, cls.mp_idx.size)
    prob.close()


def test_geometry_errors(ctx):
    import torch
    from paper_2502_05507_gb300 import GeometryError, BAEError, Problem
    N = 16
    phi = np.ones((N, N, N))
    with pytest.raises(GeometryError):
        Problem(ctx, torch.from_numpy(phi).cuda(), 0.1, 0.0)
    phi[1:5, 5:9, 5:9] = -1.0
    with pytest.raises(GeometryError):
        Problem(ctx, torch.from_numpy(phi).cuda(), 0.1, 0.0)
    phi = np.ones((N, N, N))
    phi[6:9, 6:9, 6:9] = -1.0
    phi[3, 3, 3] = np.nan
    with pytest.raises(BAEError):
        Problem(ctx, torch.from_numpy(phi).cuda(), 0.1, 0.0)
    with pytest.raises(BAEError):
        Problem(ctx, torch.from_numpy(np.ones((12, 12, 12))).cuda(), 0.1, 0.0)   # N not a power of two


# -------------------------------------------- a3-a7: the potential apply
@pytest.mark.parametrize("layer", ["double", "single"])
@pytest.mark.parametrize("make", [lambda: W.sphere_exp(16, radius=0.55, kappa2=10.0), lambda: W.star(32),
                                  lambda: W.torus_helmholtz(32, kappa2=10.0)])
def test_potential_apply_matches_direct_sum(ctx, make, layer):
    import torch
    P = make()
    prob = _problem(ctx, P, layer)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    T = OL.LGFTable(P.grid.N, P.kappa2 * P.grid.h ** 2)
    q = W.random_density(cls.gm_idx.size, seed=5)
    ref = OP.fft_convolve(OP.source_density(cls, q, layer), table=T)
    nplus = np.flatnonzero(cls.nplus)
    ref_dir = OP.direct_potential(T, cls, q, nplus, layer)
    assert np.max(np.abs(ref.reshape(-1)[nplus] - ref_dir)) < 1e-12 * np.max(np.abs(ref_dir))
    v = prob.potential_apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    scale = np.max(np.abs(ref))
    assert np.max(np.abs(v - ref)) <= 1e-12 * scale
    v32 = prob.potential_apply(torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    assert np.max(np.abs(v32 - ref)) <= 2e-6 * scale
    vds = prob.potential_apply(torch.from_numpy(q).cuda(), "df64").cpu().numpy()
    assert np.max(np.abs(vds - ref)) <= 1e-12 * scale
    # boundary operator: closure rows of K q
    Aq = prob.boundary_apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    ref_A = OS.closure_apply(cls, ref.reshape(-1))
    assert np.max(np.abs(Aq - ref_A)) <= 1e-12 * scale
    prob.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("df64", 1e-12)])
@pytest.mark.parametrize("layer", ["double", "single"])
def test_boundary_apply_after_full_apply(ctx, precision, tol, layer):
    # the boundary operator transforms only the x-planes that hold sources
    # and gathered nodes; a full-grid apply of another density first leaves
    # every plane filled with other values, so a needed plane left out of the
    # range would show up here
    import torch
    P = W.sphere_exp(32, radius=0.6)
    prob = _problem(ctx, P, layer)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    T = OL.LGFTable(32, 0.0)
    q1 = W.random_density(cls.gm_idx.size, seed=31)
    q2 = W.random_density(cls.gm_idx.size, seed=32)
    prob.potential_apply(torch.from_numpy(q1).cuda(), precision)
    Aq = prob.boundary_apply(torch.from_numpy(q2).cuda(), precision).cpu().numpy()
    ref = OP.fft_convolve(OP.source_density(cls, q2, layer), table=T)
    ref_A = OS.closure_apply(cls, ref.reshape(-1))
    assert np.max(np.abs(Aq - ref_A)) <= tol * np.max(np.abs(ref))
    prob.close()


def test_particular_solution(ctx):
    import torch
    P = W.torus_helmholtz(32, kappa2=10.0)
    prob = _problem(ctx, P)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    T = OL.LGFTable(32, P.kappa2 * P.grid.h ** 2)
    f = P.f()
    ref = OP.fft_convolve((P.grid.h ** 2) * np.where(cls.inside, f, 0.0), table=T)
    tg = cls.gm_idx
    assert np.max(np.abs(ref.reshape(-1)[tg] - OP.direct_particular(T, cls, f, P.grid.h, tg))) < 1e-12 * np.max(np.abs(ref))
    up = prob.particular(torch.from_numpy(f).cuda(), "fp64").cpu().numpy()
    assert np.max(np.abs(up - ref)) <= 1e-12 * np.max(np.abs(ref))
    up32 = prob.particular(torch.from_numpy(f).cuda(), "fp32").cpu().numpy()
    assert np.max(np.abs(up32 - ref)) <= 2e-6 * np.max(np.abs(ref))
    upds = prob.particular(torch.from_numpy(f).cuda(), "df64").cpu().numpy()
    assert np.max(np.abs(upds - ref)) <= 1e-12 * np.max(np.abs(ref))
    prob.close()


def test_apply_accepts_host_arrays(ctx):
    P = W.sphere_exp(16)
    prob = _problem(ctx, P)
    q = W.random_density(prob.n_gm, seed=9)
    import torch
    a = prob.potential_apply(q, "fp64")                      # numpy in, numpy out
    b = prob.potential_apply(torch.from_numpy(q).cuda(), "fp64").cpu().numpy()
    assert np.array_equal(a, b)
    prob.close()


# ------------------------------------------------------ a8: GMRES solve
@pytest.mark.parametrize("make,layer", [
    (lambda: W.sphere_exp(32), "double"),
    (lambda: W.sphere_exp(16), "single"),
    (lambda: W.torus_helmholtz(32, kappa2=10.0), "double"),
    (lambda: W.star(32), "double"),
])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "df64", "mixed/fp64res"])
def test_solve_matches_oracle(ctx, make, layer, precision):
    import torch
    P = make()
    prob = _problem(ctx, P, layer)
    ref = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, layer=layer, tol=1e-12)
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    prec, _, res = precision.partition("/")
    q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision=prec,
                          residual_precision="fp64" if res == "fp64res" else None)
    u = u.cpu().numpy()
    q = q.cpu().numpy()
    # Algorithm 1's output is u on M+; u on gamma- (the rest of N+) is the
    # extension that the closure rows tie to g, amplified by 1/t(m) there.
    mp, m = ref.cls.inside, ref.cls.nplus
    e_mp = np.max(np.abs(u[mp] - ref.u[mp])) / np.max(np.abs(ref.u[mp]))
    e_np = np.max(np.abs(u[m] - ref.u[m])) / np.max(np.abs(ref.u[m]))
    e_q = np.max(np.abs(q - ref.q)) / np.max(np.abs(ref.q))
    info = dict(e_mp=e_mp, e_np=e_np, e_q=e_q, **st, oracle_iters=ref.iterations)
    print(info)
    assert e_mp <= 1e-8, info
    assert e_np <= 1e-6 and e_q <= 1e-6, info
    assert np.all(u[~m] == 0)
    assert st["rel_residual"] <= 1e-10
    if prec in ("fp64", "df64"):
        assert st["iterations"] <= ref.iterations + 2, info   # oracle ran to 1e-12
    else:
        assert st["applies_fp32"] > 0 and st["refinements"] >= 1
    prob.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fresh_context_graph_vs_plain_launches(precision):
    # a context whose very first call is a solve (buffers sized before the
    # Arnoldi step is captured), and the graph-replayed solve equals the
    # kernel-by-kernel one bit for bit (same kernels, fixed-order reductions)
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2502_05507_gb300 import Context, Problem
    P = W.torus_helmholtz(32, kappa2=10.0)
    outs = []
    for use_graphs in (True, False):
        ctx = Context(0)
        prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
        g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
        q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision=precision,
                              use_graphs=use_graphs)
        outs.append((q.cpu().numpy(), u.cpu().numpy(), st))
        prob.close()
        ctx.close()
    assert np.array_equal(outs[0][0], outs[1][0])
    assert np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2]["iterations"] == outs[1][2]["iterations"]


def test_solve_errors_and_not_converged(ctx):
    # non-finite data is rejected; an iteration cap below what the problem
    # needs returns BAE_ERR_NOT_CONVERGED with the outputs and stats written
    import torch
    from paper_2502_05507_gb300 import BAEError, NotConverged
    P = W.sphere_exp(16)
    prob = _problem(ctx, P)
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    f = torch.from_numpy(P.f()).cuda()
    fb = f.clone()
    fb.view(-1)[int(np.flatnonzero(P.phi.reshape(-1) < 0)[3])] = float("nan")
    with pytest.raises(BAEError):
        prob.solve(fb, g, tol=1e-10)
    gb = g.clone()
    gb[5] = float("inf")
    with pytest.raises(BAEError):
        prob.solve(f, gb, tol=1e-10)
    fo = f.clone()
    fo.view(-1)[int(np.flatnonzero(P.phi.reshape(-1) > 0)[0])] = float("nan")   # outside M+: unused
    prob.solve(fo, g, tol=1e-10)
    with pytest.raises(NotConverged):
        prob.solve(f, g, tol=1e-10, max_iter=3)
    q, u, st = prob.solve(f, g, tol=1e-10, max_iter=3, allow_not_converged=True)
    assert st["iterations"] == 3 and st["rel_residual"] > 1e-10
    assert torch.isfinite(u).all()
    prob.close()


def test_large_kappa_solve_matches_fd(ctx):
    # kappa^2 = 2304 at N = 32 (s = 9): the spectrum comes from the closed form
    import torch
    from oracle import fd
    from paper_2502_05507_gb300 import Problem
    P = W.sphere_exp(32, kappa2=2304.0)
    prob = Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, "double")
    try:
        cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
        gv = P.g_at(np.asarray(prob.boundary_points()))
        for prec in ("fp64", "mixed"):
            q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), torch.from_numpy(gv).cuda(), tol=1e-10,
                                  precision=prec)
            ufd = fd.solve_fd(cls, P.f(), gv, P.grid.h, P.kappa2 * P.grid.h ** 2)
            m = cls.nplus
            assert np.max(np.abs(u.cpu().numpy()[m] - ufd[m])) <= 1e-8 * np.max(np.abs(ufd[m])), (prec, st)
    finally:
        prob.close()
