"""Pins of the oracle's velocity sets (Section 2 names D2Q9 and D3Q19).

The sets are rebuilt here from their definition (all integer vectors with
|c|^2 <= 1 in 2-D / |c|^2 <= 2 without corners in 3-D, weights by |c|^2)
and the isotropy the model relies on is checked: the CD stencils and the
moments of Gamma_i are exact only if sum w c c = T I and the fourth moment
is T^2 (delta delta + delta delta + delta delta).
"""
import itertools

import numpy as np
import pytest

from oracle import lattice as L

T = 1.0 / 3.0


def reference_set(name):
    if name == "D2Q9":
        vs = [v + (0,) for v in itertools.product((-1, 0, 1), repeat=2)]
        wt = {0: 4 / 9, 1: 1 / 9, 2: 1 / 36}
    else:
        vs = [v for v in itertools.product((-1, 0, 1), repeat=3) if sum(a * a for a in v) <= 2]
        wt = {0: 1 / 3, 1: 1 / 18, 2: 1 / 36}
    return {v: wt[sum(a * a for a in v)] for v in vs}


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
def test_velocity_set_matches_definition(lat):
    ref = reference_set(lat.name)
    got = {tuple(int(a) for a in c): w for c, w in zip(lat.c, lat.w)}
    assert len(got) == lat.Q == len(ref)
    assert set(got) == set(ref), sorted(set(got) ^ set(ref))
    for v, w in ref.items():
        assert got[v] == pytest.approx(w, abs=1e-16)


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
def test_isotropy(lat):
    c = lat.c.astype(float)
    w = lat.w
    d = lat.dim
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.abs(np.einsum("i,ia->a", w, c)).max() < 1e-16
    second = np.einsum("i,ia,ib->ab", w, c, c)
    np.testing.assert_allclose(second[:d, :d], T * np.eye(d), atol=1e-15)
    third = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.abs(third).max() < 1e-16
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    I = np.eye(3)
    iso = T * T * (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I)
                   + np.einsum("ad,bc->abcd", I, I))
    np.testing.assert_allclose(fourth[:d, :d, :d, :d], iso[:d, :d, :d, :d], atol=1e-15)


@pytest.mark.parametrize("lat", [L.D2Q9, L.D3Q19], ids=lambda l: l.name)
def test_opposites(lat):
    for i in range(lat.Q):
        assert np.all(lat.c[lat.opp[i]] == -lat.c[i])
        assert lat.w[lat.opp[i]] == lat.w[i]
