"""Shift MPOs, Sec. 2.5.

1-D: the n-bit cyclic shift S^(n) and non-cyclic shift S^^(n) with
(S f)_x = f_{x+1} are rank-core products (Eq. recursive and the core
definitions that follow it):
    S^(n)  = A  |x| B |x| ... |x| B |x| C
    S^^(n) = A^ |x| B |x| ... |x| B |x| C
with A = [I P], A^ = [I J], B = [[I, J], [0, J']], C = [J; J'], most
significant bit first.  The opposite direction swaps J and J' in every core.
For n = 1 the whole operator is a single 2x2 block: P (cyclic) or J.

3-D: the cores act on the sites of one axis; the sites of the other axes carry
identity cores that pass the MPO bond through ("padding with identities").

Conventions used here: an MPO core has shape (w_k, 2_out, 2_in, w_{k+1}).
shift_mpo(n, axis, offset, cyclic) builds the operator (S f)(x) = f(x + offset
e_axis) with offset = +1 (paper's S) or -1 (J <-> J' swapped); the non-cyclic
version leaves zeros where x + offset falls outside the domain.

Pinned by tests/test_oracle_mpo.py: the printed S^(2), S^^(2) matrices and a
brute-force comparison against explicit shift permutations.
"""

import numpy as np

I2 = np.array([[1.0, 0.0], [0.0, 1.0]])
J = np.array([[0.0, 1.0], [0.0, 0.0]])
Jp = np.array([[0.0, 0.0], [1.0, 0.0]])
P = np.array([[0.0, 1.0], [1.0, 0.0]])
Z2 = np.zeros((2, 2))


def _core(blocks):
    """blocks[w][v] is a 2x2 (out, in) matrix -> array (w, 2, 2, v)."""
    b = np.array(blocks, dtype=np.float64)          # (w, v, 2, 2)
    return np.transpose(b, (0, 2, 3, 1))


def shift_mpo_1d(n, offset=+1, cyclic=True):
    """List of n MPO cores for the 1-D shift by `offset` on 2^n points."""
    j, jp = (J, Jp) if offset == +1 else (Jp, J)
    if n == 1:
        return [_core([[P if cyclic else j]])]
    first = _core([[I2, P if cyclic else j]])
    mid = _core([[I2, j], [Z2, jp]])
    last = _core([[j], [jp]])
    return [first] + [mid.copy() for _ in range(n - 2)] + [last]


def shift_mpo(n_bits, axis, offset, cyclic, dim=3):
    """3-D shift along `axis` in the scale-ordered site order (site k holds
    bit k // dim of axis k % dim)."""
    oned = shift_mpo_1d(n_bits, offset, cyclic)
    L = dim * n_bits
    cores = []
    w = 1                                             # current bond dimension
    for k in range(L):
        if k % dim == axis:
            c = oned[k // dim]
            cores.append(c)
            w = c.shape[3]
        else:
            c = np.zeros((w, 2, 2, w))
            for a in range(w):
                c[a, :, :, a] = I2
            cores.append(c)
    return cores


def mpo_to_matrix(cores):
    """Contract an MPO into a (2^L x 2^L) matrix over site-ordered indices."""
    M = cores[0]
    for c in cores[1:]:
        # M: (1, out..., in..., w) ; combine
        M = np.einsum("...w,wtsv->...tsv", M, c)
    L = len(cores)
    # axes now: 1, t0, s0, t1, s1, ..., t_{L-1}, s_{L-1}, 1
    M = M.reshape(M.shape[1:-1])
    outs = list(range(0, 2 * L, 2))
    ins = list(range(1, 2 * L, 2))
    M = np.transpose(M, outs + ins)
    return M.reshape(2 ** L, 2 ** L)
