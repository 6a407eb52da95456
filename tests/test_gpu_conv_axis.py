"""The convolutions inside a solve and in bae_boundary_apply transform only
the planes that hold sources or read-back nodes, along the first axis of
the grid they run on; the library runs them on the grid with x swapped for
the axis of fewest such planes (bae_problem_conv_planes). The lattice
Green's function is symmetric under permutations of the axes, so the
results must equal the oracle's as before:
- the axis and plane range equal what the oracle's classification gives
  (sources gamma- and D-nodes, or gamma- for the single layer, one plane of
  margin), including the no-swap cases (sphere, direct formulation,
  BAE_CONV_AXIS=x);
- bae_boundary_apply on a z-flat torus (x <-> z) and a y-flat ellipsoid
  (x <-> y), both layers, float64/double-float 1e-12 and float32 2e-6
  against the oracle's FFT convolution, after a full-grid apply of another
  density has filled every plane; at N = 64 the float32 and double-float
  i passes run their narrow (shifted, few-slot) transform, on a thin disk
  the one-slot one;
- mixed-precision solves of both geometries equal the oracle's u on M+ to
  1e-8, and the torus solve equals the unswapped one (BAE_CONV_AXIS=x) to
  1e-9."""
import os

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


def flat_ellipsoid(N=32, kappa2=0.0):
    """Ellipsoid with semi-axes (0.7, 0.3, 0.6) in [-1,1]^3: thinnest in y."""
    return W._make(f"yflat_N{N}", W.cell_centred(N), lambda x, y, z: W.phi_ellipsoid(x, y, z, 0.7, 0.3, 0.6),
                   kappa2, "double", lambda x, y, z: W.sol_exp_sum(x, y, z, kappa2))


def _problem(ctx, P, layer=None):
    import torch
    from paper_2502_05507_gb300 import Problem
    return Problem(ctx, torch.from_numpy(P.phi).cuda(), P.grid.h, P.grid.origin, P.kappa2, layer or P.layer)


def _expected_axis(cls, layer):
    """(axis, lo, hi) from the oracle's point sets: per axis the planes
    holding a source, one plane of margin each side; the axis of fewest
    planes when it has a tenth fewer than x."""
    N = cls.N
    src = cls.gm | (cls.dnode if layer != "single" else False)
    rng = []
    for ax in range(3):
        other = tuple(a for a in range(3) if a != ax)
        idx = np.flatnonzero(np.any(src, axis=other))
        rng.append((max(0, idx.min() - 1), min(N, idx.max() + 2)))
    best = 0
    for ax in (1, 2):
        if 10 * (rng[ax][1] - rng[ax][0]) < 9 * (rng[best][1] - rng[best][0]):
            best = ax
    return best, rng[best][0], rng[best][1], rng[0]


@pytest.mark.parametrize("name,make,layer,axis", [
    ("torus", lambda: W.torus_helmholtz(32, kappa2=10.0), "double", 2),
    ("torus_single", lambda: W.torus_helmholtz(32, kappa2=10.0), "single", 2),
    ("yflat", lambda: flat_ellipsoid(32), "double", 1),
    ("sphere", lambda: W.sphere_exp(32), "double", 0),
    ("torus_direct", lambda: W.torus_helmholtz(32, kappa2=10.0), "direct", 0),
])
def test_conv_planes_follow_the_geometry(ctx, name, make, layer, axis):
    P = make()
    prob = _problem(ctx, P, layer)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    ax, lo, hi = prob.conv_planes()
    assert prob.plane_range() == _expected_axis(cls, layer)[3]
    if layer == "direct":
        assert (ax, lo, hi) == (0,) + prob.plane_range()
    else:
        assert (ax, lo, hi) == _expected_axis(cls, layer)[:3]
    assert ax == axis
    prob.close()


def test_conv_axis_environment_keeps_x(ctx, monkeypatch):
    monkeypatch.setenv("BAE_CONV_AXIS", "x")
    P = W.torus_helmholtz(32, kappa2=10.0)
    prob = _problem(ctx, P)
    assert prob.conv_planes() == (0,) + prob.plane_range()
    prob.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("df64", 1e-12)])
@pytest.mark.parametrize("layer", ["double", "single"])
@pytest.mark.parametrize("make", [lambda: W.torus_helmholtz(32, kappa2=10.0), lambda: flat_ellipsoid(32),
                                  lambda: W.torus_helmholtz(64, kappa2=10.0), lambda: flat_ellipsoid(64)])
def test_swapped_boundary_apply_matches_oracle(ctx, make, layer, precision, tol):
    # at N = 64 the float32 and double-float i passes also take the narrow
    # (shifted) transform: the planes span at most four blocks of its rows
    import torch
    P = make()
    prob = _problem(ctx, P, layer)
    assert prob.conv_planes()[0] != 0
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    T = OL.LGFTable(P.grid.N, P.kappa2 * P.grid.h ** 2)
    q1 = W.random_density(cls.gm_idx.size, seed=41)
    q2 = W.random_density(cls.gm_idx.size, seed=42)
    prob.potential_apply(torch.from_numpy(q1).cuda(), precision)   # every plane of the work buffers filled
    Aq = prob.boundary_apply(torch.from_numpy(q2).cuda(), precision).cpu().numpy()
    ref = OP.fft_convolve(OP.source_density(cls, q2, layer), table=T)
    ref_A = OS.closure_apply(cls, ref.reshape(-1))
    assert np.max(np.abs(Aq - ref_A)) <= tol * np.max(np.abs(ref))
    prob.close()


def thin_disk(N=64, kappa2=0.0):
    """Ellipsoid (0.7, 0.6, 0.04) centred at z = 0.37: at N = 64 its source
    planes [40, 48) fill one block of eight rows, so the float32 and
    double-float i passes (eight threads per line) run their one-slot
    transform."""
    return W._make(f"disk_N{N}", W.cell_centred(N),
                   lambda x, y, z: (x / 0.7) ** 2 + (y / 0.6) ** 2 + ((z - 0.37) / 0.04) ** 2 - 1.0,
                   kappa2, "double", lambda x, y, z: W.sol_exp_sum(x, y, z, kappa2))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6), ("df64", 1e-12)])
@pytest.mark.parametrize("layer", ["double", "single"])
def test_one_slot_i_pass_matches_oracle(ctx, layer, precision, tol):
    import torch
    P = thin_disk(64, 1.0)
    prob = _problem(ctx, P, layer)
    ax, lo, hi = prob.conv_planes()
    assert ax == 2 and lo >= 40 and hi <= 48, (ax, lo, hi)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    T = OL.LGFTable(P.grid.N, P.kappa2 * P.grid.h ** 2)
    q = W.random_density(cls.gm_idx.size, seed=43)
    Aq = prob.boundary_apply(torch.from_numpy(q).cuda(), precision).cpu().numpy()
    ref = OP.fft_convolve(OP.source_density(cls, q, layer), table=T)
    ref_A = OS.closure_apply(cls, ref.reshape(-1))
    assert np.max(np.abs(Aq - ref_A)) <= tol * np.max(np.abs(ref))
    prob.close()


@pytest.mark.parametrize("make", [lambda: W.torus_helmholtz(32, kappa2=10.0), lambda: flat_ellipsoid(32, 1.0),
                                  lambda: thin_disk(64, 1.0)])
def test_swapped_solve_matches_oracle(ctx, make):
    import torch
    P = make()
    prob = _problem(ctx, P)
    assert prob.conv_planes()[0] != 0
    ref = OS.solve(P.phi, P.grid.h, P.grid.origin, P.f(), P.g_at, P.kappa2, tol=1e-12)
    g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
    q, u, st = prob.solve(torch.from_numpy(P.f()).cuda(), g, tol=1e-10, precision="mixed")
    u = u.cpu().numpy()
    mp, m = ref.cls.inside, ref.cls.nplus
    e_mp = np.max(np.abs(u[mp] - ref.u[mp])) / np.max(np.abs(ref.u[mp]))
    assert e_mp <= 1e-8, (e_mp, st)
    assert np.all(u[~m] == 0)
    prob.close()


def test_swapped_solve_equals_unswapped(ctx, monkeypatch):
    import torch
    P = W.torus_helmholtz(64, kappa2=10.0)
    f = torch.from_numpy(P.f()).cuda()
    out = {}
    for mode in ("auto", "x"):
        if mode == "x":
            monkeypatch.setenv("BAE_CONV_AXIS", "x")
        prob = _problem(ctx, P)
        assert (prob.conv_planes()[0] != 0) == (mode == "auto")
        g = torch.from_numpy(P.g_at(prob.boundary_points())).cuda()
        for prec in ("mixed", "fp64"):
            q, u, st = prob.solve(f, g, tol=1e-10, precision=prec)
            assert st["rel_residual"] <= 1e-10
            out[(mode, prec)] = u.cpu().numpy()
        prob.close()
    for prec in ("mixed", "fp64"):
        a, b = out[("auto", prec)], out[("x", prec)]
        assert np.max(np.abs(a - b)) <= 1e-9 * np.max(np.abs(b)), prec
    os.environ.pop("BAE_CONV_AXIS", None)


@pytest.mark.parametrize("precision", ["fp32", "df64"])
@pytest.mark.parametrize("N", [64, 128])
def test_narrow_i_pass_same_in_every_schedule(ctx, N, precision):
    # every schedule the autotuner can pick runs the same i-pass transform
    # for a given plane range, so a batch item and the same right-hand side
    # alone stay bit-identical whichever schedule each size picked
    import torch
    from paper_2502_05507_gb300 import set_conv_schedule
    P = W.torus_helmholtz(N, kappa2=10.0)
    prob = _problem(ctx, P)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    q = torch.from_numpy(W.random_density(cls.gm_idx.size, seed=44)).cuda()
    out = {}
    try:
        for name in ("passes", "passes_alt", "persist", "plane"):
            set_conv_schedule(name)
            out[name] = prob.boundary_apply(q, precision).cpu().numpy()
    finally:
        set_conv_schedule("auto")
    # the double-float cluster plane kernels (N >= 128) transform their k
    # and j lines with the two-level plan, the passes with the three-level
    # one: the same convolution in another rounding order
    same_plan = precision == "fp32" or N < 128
    for name, a in out.items():
        if name == "plane" and not same_plan:
            assert np.max(np.abs(a - out["passes"])) <= 1e-12 * np.max(np.abs(out["passes"])), name
        else:
            assert np.array_equal(a, out["passes"]), name
    if N == 64:
        T = OL.LGFTable(N, P.kappa2 * P.grid.h ** 2)
        ref = OP.fft_convolve(OP.source_density(cls, q.cpu().numpy(), "double"), table=T)
        ref_A = OS.closure_apply(cls, ref.reshape(-1))
        tol = 2e-6 if precision == "fp32" else 1e-12
        assert np.max(np.abs(out["passes"] - ref_A)) <= tol * np.max(np.abs(ref))
    prob.close()


def _source_box(cls):
    """Per axis the planes holding a source (gamma-, D-nodes), one plane of
    margin each side: the box that holds M+."""
    N = cls.N
    src = cls.gm | cls.dnode
    box = []
    for ax in range(3):
        other = tuple(a for a in range(3) if a != ax)
        idx = np.flatnonzero(np.any(src, axis=other))
        box.append((max(0, idx.min() - 1), min(N, idx.max() + 2)))
    return box


@pytest.mark.parametrize("make,nrhs", [(lambda: W.torus_helmholtz(64, kappa2=10.0), 1), (lambda: flat_ellipsoid(32), 2)])
def test_host_f_copies_the_box_of_m_plus(ctx, make, nrhs):
    # a solve reads f only on M+: from host memory the library copies the
    # box of planes that holds M+ (and reports the bytes); u is 0 outside
    # N+, so into host memory it copies the same box and writes the zeros
    # around it on the host (the host u starts uninitialised). Same results
    # as with device memory.
    import torch
    P = make()
    prob = _problem(ctx, P)
    cls = OG.classify(P.phi, P.grid.h, P.grid.origin)
    box = _source_box(cls)
    inside = np.zeros_like(cls.inside)
    inside[box[0][0]:box[0][1], box[1][0]:box[1][1], box[2][0]:box[2][1]] = True
    assert not np.any(cls.inside & ~inside)
    xs = prob.boundary_points()
    f = np.stack([P.f() * (1.0 + 0.1 * k) for k in range(nrhs)])
    g = np.stack([P.g_at(xs) * (1.0 + 0.1 * k) for k in range(nrhs)])
    qd, ud, sd = prob.solve_batched(torch.from_numpy(f).cuda(), torch.from_numpy(g).cuda(), tol=1e-10,
                                    precision="mixed")
    qh, uh, sh = prob.solve_batched(f, g, tol=1e-10, precision="mixed")
    assert np.array_equal(qh, qd.cpu().numpy()) and np.array_equal(uh, ud.cpu().numpy())
    vol = int(np.prod([hi - lo for lo, hi in box]))
    N = P.grid.N
    for k in range(nrhs):
        assert sd[k]["h2d_bytes"] == 0 and sd[k]["d2h_bytes"] == 0
        assert sh[k]["h2d_bytes"] == 8 * (vol + xs.shape[0]), (sh[k], vol)
        assert sh[k]["d2h_bytes"] == 8 * (vol + qh.shape[1])
    prob.close()
