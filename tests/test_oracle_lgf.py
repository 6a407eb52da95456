"""Pins of the oracle's lattice Green's function (Section 2.2)."""
import math
import os

import numpy as np
import pytest

from oracle import lgf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


@pytest.fixture(scope="module")
def table16_0():
    return lgf.LGFTable(16, 0.0)


@pytest.fixture(scope="module")
def table16_s():
    return lgf.LGFTable(16, 10.0 / 4096.0)


def test_watson_closed_forms_agree():
    # the two Gamma-function forms printed in Section 2.2 are the same number
    assert lgf.watson_g0() == pytest.approx(lgf.watson_g0_alt(), rel=1e-14)


def test_g0_origin_matches_watson(table16_0):
    ref = _golden("watson.txt")["G0_0"]
    assert lgf.watson_g0() == pytest.approx(ref, abs=1e-13)
    assert lgf.lgf_entry((0, 0, 0), 0.0) == pytest.approx(lgf.watson_g0(), rel=1e-13)
    assert table16_0((0, 0, 0)) == pytest.approx(lgf.watson_g0(), rel=1e-13)


@pytest.mark.parametrize("s", [0.0, 10.0 / 4096.0, 1.0 / 16384.0, 100.0 / 16384.0, 1.0])
def test_lattice_identity_at_origin(s):
    # (6+s) G(0) - 6 G(e1) = 1  (eq. [lgf_delta] at n = 0)
    g0 = lgf.lgf_entry((0, 0, 0), s)
    g1 = lgf.lgf_entry((1, 0, 0), s)
    assert (6.0 + s) * g0 - 6.0 * g1 == pytest.approx(1.0, abs=1e-13)


@pytest.mark.parametrize("which", ["table16_0", "table16_s"])
def test_lattice_identity_everywhere(which, request):
    # (6+s) G(n) - sum_{+-e_i} G(n +- e_i) = delta_{n,0} at every n of the table
    # whose neighbours are in the table
    T = request.getfixturevalue(which)
    N = T.N
    r = np.arange(-(N - 2), N - 1)
    n = np.stack(np.meshgrid(r, r, r, indexing="ij"), axis=-1).reshape(-1, 3)
    lhs = (6.0 + T.s) * T(n)
    for d in np.eye(3, dtype=np.int64):
        lhs -= T(n + d) + T(n - d)
    delta = np.all(n == 0, axis=1).astype(float)
    assert np.max(np.abs(lhs - delta)) < 2e-14


def test_table_matches_entries_and_symmetry(table16_s):
    rng = np.random.default_rng(7)
    for _ in range(6):
        n = tuple(int(v) for v in rng.integers(-15, 16, size=3))
        ref = lgf.lgf_entry(n, table16_s.s)
        # every permutation and sign flip gives the same value (1/48 symmetry)
        for perm in ((0, 1, 2), (2, 0, 1), (1, 2, 0)):
            m = np.array([n[perm[0]], -n[perm[1]], n[perm[2]]])
            assert table16_s(m) == pytest.approx(ref, rel=1e-13)


def test_far_field_expansion():
    # G_0 - A_G^3 = O(|n|^-7) in every direction (Section 2.2, overall sign
    # and the -228 coefficient as read in oracle/lgf.py). A dropped term, a
    # wrong sign or a wrong coefficient leaves an O(|n|^-5) remainder, more
    # than 10x this bound at these |n|.
    for n in [(60, 20, 0), (45, 30, 10), (40, 40, 40), (80, 5, 3), (25, 25, 25), (50, 40, 30)]:
        g = lgf.lgf_entry(n, 0.0)
        r = math.sqrt(sum(v * v for v in n))
        assert abs(g - lgf.far_field(n)) < 0.5 * r ** -7
    # the remainder along the diagonal is a fixed multiple of |n|^-7
    c = [(lgf.lgf_entry((a, a, a), 0.0) - lgf.far_field((a, a, a))) * (3 * a * a) ** 3.5 for a in (20, 40)]
    assert c[0] == pytest.approx(c[1], rel=0.02)


def test_periodic_trapezoid_for_positive_sigma():
    # For s = 1 the periodic M-point trapezoid sum (Section 2.2, sigma > 0) has
    # aliasing error about exp(-0.96 M/2); M = 64 reaches round-off.
    s = 1.0
    P = lgf.periodic_trapezoid(64, s)
    for n in [(0, 0, 0), (1, 0, 0), (3, 2, 1), (6, 0, 5), (10, 4, 2)]:
        assert P[n] == pytest.approx(lgf.lgf_entry(n, s), rel=1e-11)


def test_positive_and_decreasing(table16_s):
    v = table16_s.cube
    assert np.all(v > 0)
    assert np.all(np.diff(v[:, 0, 0]) < 0)


@pytest.mark.parametrize("N,s", [(16, 25.0), (32, 9.0), (8, 200.0)])
def test_periodic_spectrum_equals_table_spectrum(N, s):
    # large s: the (2N)-periodic Green's function (closed-form spectrum, the
    # 2N-point trapezoid rule of Section 2.2) is the embedded free-lattice
    # G_s up to exp(-mu N) images, far below round-off
    from oracle import potentials as pot
    assert lgf.periodic_spectrum_applies(N, s)
    ref = pot.lgf_spectrum(lgf.LGFTable(N, s))
    got = lgf.periodic_spectrum(N, s)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("N,s", [(16, 0.04), (32, 0.5)])
def test_periodic_spectrum_rejected_for_slow_decay(N, s):
    # small s: G_s has not decayed within the box, the images show above
    # round-off, and the rule keeps the table route
    from oracle import potentials as pot
    assert not lgf.periodic_spectrum_applies(N, s)
    ref = pot.lgf_spectrum(lgf.LGFTable(N, s))
    got = lgf.periodic_spectrum(N, s)
    assert np.max(np.abs(got - ref)) > 1e-12 * np.max(np.abs(ref))
