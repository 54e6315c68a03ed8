"""Pins of the velocity sets: isotropy up to fourth order fixes the weights."""
import itertools

import numpy as np
import pytest

from oracle import lattice


@pytest.mark.parametrize("name", ["D3Q19", "D3Q15"])
def test_isotropy(name):
    lat = lattice.get(name)
    c = lat.c.astype(np.float64)
    w = lat.w
    assert abs(w.sum() - 1.0) < 1e-15
    np.testing.assert_allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3.0, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    fourth = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    d = np.eye(3)
    ref = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9.0
    np.testing.assert_allclose(fourth, ref, atol=1e-15)


@pytest.mark.parametrize("name", ["D3Q19", "D3Q15"])
def test_opposites(name):
    lat = lattice.get(name)
    for i in range(lat.Q):
        np.testing.assert_array_equal(lat.c[lat.opp[i]], -lat.c[i])
    assert len({tuple(v) for v in lat.c}) == lat.Q
