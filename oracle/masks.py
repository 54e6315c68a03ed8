"""Masks combined on separate length scales, App. D (test infrastructure only).

An inner mask on a 2^k grid per axis repeated where an outer mask on a 2^l grid
per axis is one: the combined mask on 2^(l+k) cells per axis is
m(x) = m_outer(x >> k) m_inner(x mod 2^k), axis by axis.  In the scale order of
Sec. 2.4 the l most significant bits of every axis come first, so the combined
MPS is the outer MPS followed by the inner MPS (bond 1 at the junction) and its
largest bond is the larger of the two.

Pinned by tests/test_oracle_masks.py: against the definition written out on
dense grids, and the bond bound.
"""

import numpy as np


def combined_dense(outer, inner):
    """The definition on dense (N_o)^3 and (N_i)^3 arrays -> (N_o N_i)^3."""
    No, Ni = outer.shape[0], inner.shape[0]
    N = No * Ni
    x = np.arange(N)
    o = outer[np.ix_(x // Ni, x // Ni, x // Ni)]
    i = inner[np.ix_(x % Ni, x % Ni, x % Ni)]
    return o * i


def mask_product(outer_cores, inner_cores):
    """Combined mask MPS: the outer cores (coarse bits) then the inner cores."""
    assert outer_cores[-1].shape[2] == 1 and inner_cores[0].shape[0] == 1
    return [c.copy() for c in outer_cores] + [c.copy() for c in inner_cores]
