"""Pins of the shift MPOs (Sec. 2.5): printed n=2 matrices and brute force
against explicit shift permutations built by index arithmetic."""
import numpy as np
import pytest

from oracle import mpo, quantics as q
from conftest import read_golden


def test_printed_n2_matrices():
    rows = np.array(read_golden("shift_n2.txt"))
    S2, S2hat = rows[:4], rows[4:]
    np.testing.assert_array_equal(mpo.mpo_to_matrix(mpo.shift_mpo_1d(2, +1, True)), S2)
    np.testing.assert_array_equal(mpo.mpo_to_matrix(mpo.shift_mpo_1d(2, +1, False)), S2hat)


def _perm_1d(N, offset, cyclic):
    M = np.zeros((N, N))
    for x in range(N):
        src = x + offset
        if cyclic:
            M[x, src % N] = 1.0
        elif 0 <= src < N:
            M[x, src] = 1.0
    return M


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("offset", [+1, -1])
@pytest.mark.parametrize("cyclic", [True, False])
def test_1d_bruteforce(n, offset, cyclic):
    got = mpo.mpo_to_matrix(mpo.shift_mpo_1d(n, offset, cyclic))
    np.testing.assert_array_equal(got, _perm_1d(1 << n, offset, cyclic))


def test_bond_dimension_two():
    for n in (2, 3, 6):
        for c in mpo.shift_mpo_1d(n, +1, True):
            assert max(c.shape[0], c.shape[3]) <= 2


@pytest.mark.parametrize("n", [1, 2])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("offset", [+1, -1])
@pytest.mark.parametrize("cyclic", [True, False])
def test_3d_bruteforce(n, axis, offset, cyclic):
    """The padded MPO, contracted and mapped back to [x][y][z] order, equals the
    explicit permutation (S g)(x) = g(x + offset e_axis)."""
    N = 1 << n
    L = 3 * n
    Mq = mpo.mpo_to_matrix(mpo.shift_mpo(n, axis, offset, cyclic))
    # map site-ordered row/col indices to dense [x][y][z] indices
    site_idx = q.encode(np.arange(N ** 3).reshape(N, N, N)).reshape(-1)
    dense = np.zeros((N ** 3, N ** 3))
    dense[np.ix_(site_idx, site_idx)] = Mq
    ref = np.zeros((N ** 3, N ** 3))
    for x in range(N):
        for y in range(N):
            for z in range(N):
                p = [x, y, z]
                s = list(p)
                s[axis] += offset
                if not cyclic and not (0 <= s[axis] < N):
                    continue
                s[axis] %= N
                ref[(p[0] * N + p[1]) * N + p[2], (s[0] * N + s[1]) * N + s[2]] = 1.0
    assert L == len(mpo.shift_mpo(n, axis, offset, cyclic))
    np.testing.assert_array_equal(dense, ref)
