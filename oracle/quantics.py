"""Scale-ordered (quantics) index encoding, Sec. 2.4, Eq. (scale_ordering).

A 3-D field on (2^n)^3 cells, indexed [x][y][z], is reshaped to an order-3n
tensor of binary sites.  The paper regroups the bits of x, y, z by significance,
most significant first; with one binary site per bit, site k holds bit
(n-1 - k//3) of axis k % 3 (axis 0 = x).  Site 0 is the MSB of x, site 1 the MSB
of y, site 2 the MSB of z, site 3 the next bit of x, and so on.

Pinned by: bijection and explicit bit-position tests (tests/test_oracle_quantics.py).
"""

import numpy as np


def n_sites(n_bits, dim=3):
    return dim * n_bits


def site_of(axis, level, dim=3):
    """Site index of bit `level` (0 = most significant) of `axis`."""
    return dim * level + axis


def site_bits(n_bits, cell):
    """Binary index of every site for one cell (x, y, z): site k holds bit
    (n-1 - k//dim) of axis k % dim (Eq. scale_ordering)."""
    dim = len(cell)
    return [(int(cell[k % dim]) >> (n_bits - 1 - k // dim)) & 1 for k in range(dim * n_bits)]


def _perm(n_bits, dim):
    # axis of the reshaped dense array that holds site k
    return [(k % dim) * n_bits + k // dim for k in range(dim * n_bits)]


def encode(dense):
    """Dense (N,)*dim array -> tensor of shape (2,)*(dim*n) in site order."""
    dim = dense.ndim
    N = dense.shape[0]
    n = N.bit_length() - 1
    assert all(s == N for s in dense.shape) and (1 << n) == N
    t = np.asarray(dense).reshape((2,) * (dim * n))
    return np.transpose(t, _perm(n, dim))


def decode(tensor, dim=3):
    """Inverse of encode."""
    L = tensor.ndim
    n = L // dim
    p = _perm(n, dim)
    inv = np.argsort(p)
    t = np.transpose(tensor, inv)
    N = 1 << n
    return t.reshape((N,) * dim)
