"""Pins of the oracle's point sets and closure (Section 2.1, eq. [bc])."""
import numpy as np
import pytest

import workloads as W
from oracle import grid


def _sets(cls):
    shape = (cls.N,) * 3
    tolist = lambda idx: sorted(tuple(int(v) for v in t) for t in zip(*np.unravel_index(idx, shape)))
    return dict(Mp=tolist(cls.mp_idx), gm=tolist(cls.gm_idx), gp=tolist(cls.gp_idx),
                Np=tolist(np.flatnonzero(cls.nplus)), dnodes=tolist(np.flatnonzero(cls.dnode)))


@pytest.mark.parametrize("seed", range(4))
def test_classify_equals_set_definitions_random(seed):
    # random blobs on tiny grids, interior kept two nodes off the faces
    rng = np.random.default_rng(seed)
    N = 9
    phi = rng.standard_normal((N, N, N))
    phi[:2] = phi[-2:] = 1.0
    phi[:, :2] = phi[:, -2:] = 1.0
    phi[:, :, :2] = phi[:, :, -2:] = 1.0
    cls = grid.classify(phi, 1.0, 0.0)
    bf = grid.classify_bruteforce(phi)
    got = _sets(cls)
    for key in ("Mp", "gm", "gp", "dnodes"):
        assert got[key] == bf[key], key
    # N+ of the paper (stencils of M+) restricted to the grid
    assert got["Np"] == [x for x in bf["Np"] if all(0 <= v < N for v in x)]
    # |D_n| per gamma- node
    for m in bf["gm"]:
        assert cls.count[m] == len(bf["D"][m])


def test_classify_sphere_matches_set_definitions():
    P = W.sphere_exp(12, radius=0.6)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    bf = grid.classify_bruteforce(P.phi)
    got = _sets(cls)
    for key in ("Mp", "gm", "gp", "dnodes"):
        assert got[key] == bf[key]


def test_zero_phi_is_exterior():
    N = 8
    phi = np.ones((N, N, N))
    phi[3:5, 3:5, 3:5] = -1.0
    phi[3, 3, 5] = 0.0
    cls = grid.classify(phi, 1.0, 0.0)
    assert not cls.inside[3, 3, 5]
    assert cls.gm[3, 3, 5]


def test_closure_properties():
    P = W.torus_helmholtz(32)
    cls = grid.classify(P.phi, P.grid.h, P.grid.origin)
    phi = P.phi.reshape(-1)
    pm, pp = phi[cls.gm_idx], phi[cls.partner]
    assert np.all(pp < 0) and np.all(pm >= 0)
    assert np.all((cls.t > 0) & (cls.t <= 1))
    # partner is a 6-neighbour
    a = np.stack(np.unravel_index(cls.gm_idx, P.phi.shape), 1)
    b = np.stack(np.unravel_index(cls.partner, P.phi.shape), 1)
    assert np.all(np.abs(a - b).sum(1) == 1)
    # linear interpolation of phi vanishes at x*: phi_p + t (phi_m - phi_p) = 0
    assert np.max(np.abs(pp + cls.t * (pm - pp))) < 1e-15
    # x* lies on the edge at fraction t from p towards m
    xs = P.grid.origin + b * P.grid.h + cls.t[:, None] * (a - b) * P.grid.h
    assert np.max(np.abs(xs - cls.xstar)) < 1e-14
    # largest t among the M+ neighbours
    for col in range(0, cls.gm_idx.size, 37):
        m = tuple(a[col])
        best = -1.0
        for d in grid.DIRS:
            p = tuple(np.array(m) + d)
            if P.phi[p] < 0:
                best = max(best, P.phi[p] / (P.phi[p] - P.phi[m]))
        assert cls.t[col] == best


def test_geometry_touching_faces_rejected():
    N = 8
    phi = np.ones((N, N, N))
    phi[1:4, 3:5, 3:5] = -1.0   # an interior node at i=1 puts gamma- on the face
    with pytest.raises(grid.GeometryError):
        grid.classify(phi, 1.0, 0.0)
    with pytest.raises(grid.GeometryError):
        grid.classify(np.ones((N, N, N)), 1.0, 0.0)
