"""Pins of the MPS algebra (Sec. 2.1-2.3) against dense elementwise identities,
Eckart-Young, the rounding error bound and orthogonality (Eq. lorg)."""
import numpy as np
import pytest

import synth
from oracle import mps as M
from oracle import mpo, quantics as q


def _rand(L, chi, seed):
    return synth.random_mps(L, synth.feasible_ranks(L, chi), seed)


def test_add_product_mpo_inner():
    L = 9
    A, B = _rand(L, 4, 1), _rand(L, 3, 2)
    ta, tb = M.to_tensor(A), M.to_tensor(B)
    np.testing.assert_allclose(M.to_tensor(M.add(A, B)), ta + tb, atol=1e-14)
    np.testing.assert_allclose(M.to_tensor(M.lincomb([(2.0, A), (-0.5, B), (3.0, A)])),
                               5.0 * ta - 0.5 * tb, atol=1e-13)
    np.testing.assert_allclose(M.to_tensor(M.hadamard_exact(A, B)), ta * tb, atol=1e-14)
    assert abs(M.inner_ones(A) - ta.sum()) < 1e-12
    vecs = [np.random.default_rng(k).standard_normal(2) for k in range(L)]
    r1 = M.to_tensor(M.rank1(vecs))
    np.testing.assert_allclose(M.to_tensor(M.mask_rank1(A, vecs)), ta * r1, atol=1e-14)
    # MPO application equals the dense shift
    g = q.decode(ta)
    S = M.apply_mpo(mpo.shift_mpo(3, 1, +1, True), A)
    np.testing.assert_allclose(q.decode(M.to_tensor(S)), np.roll(g, -1, axis=1), atol=1e-14)


def test_ttsvd_exact_and_left_orthogonal():
    rng = np.random.default_rng(3)
    T = rng.standard_normal((2,) * 8)
    A = M.tt_svd(T, 10 ** 6, 0.0)
    np.testing.assert_allclose(M.to_tensor(A), T, atol=1e-12)
    for c in A[:-1]:
        G = np.einsum("asb,asc->bc", c, c)          # Eq. (lorg)
        np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-13)


def test_round_eckart_young():
    """L = 6 binary sites: only the middle bond (8) exceeds chi = 5, so the
    rounding is the best rank-5 approximation of that unfolding."""
    rng = np.random.default_rng(4)
    Mat = rng.standard_normal((8, 8))
    A = M.tt_svd(Mat.reshape((2,) * 6), 10 ** 6, 0.0)
    assert M.ranks(A) == [1, 2, 4, 8, 4, 2, 1]
    R = M.round_mps(A, 5, 0.0)
    assert M.ranks(R) == [1, 2, 4, 5, 4, 2, 1]
    s = np.linalg.svd(Mat, compute_uv=False)
    err2 = np.sum((M.to_tensor(R).reshape(8, 8) - Mat) ** 2)
    assert abs(err2 - np.sum(s[5:] ** 2)) < 1e-12 * np.sum(s ** 2)


def test_round_eps_bound_and_orthogonality():
    L = 10
    A = M.add(_rand(L, 6, 5), M.scale(_rand(L, 6, 6), 1e-3))
    tA = M.to_tensor(A)
    for eps in (1e-2, 1e-4, 1e-8):
        R = M.round_mps(A, 10 ** 6, eps)
        err = np.sqrt(np.sum((M.to_tensor(R) - tA) ** 2))
        assert err <= eps * np.sqrt(np.sum(tA ** 2)) * (1 + 1e-10)
        for c in R[1:]:
            G = np.einsum("asb,csb->ac", c, c)      # right-orthogonal after the sweep
            np.testing.assert_allclose(G, np.eye(G.shape[0]), atol=1e-12)


def test_round_zero_and_rank_one():
    L = 6
    Z = M.scale(M.ones(L), 0.0)
    R = M.round_mps(M.add(Z, Z), 4, 1e-12)
    assert max(M.ranks(R)) == 1 and np.abs(M.to_tensor(R)).max() == 0.0
    O = M.round_mps(M.add(M.ones(L), M.ones(L)), 4, 1e-12)
    assert max(M.ranks(O)) == 1
    np.testing.assert_allclose(M.to_tensor(O), 2.0, atol=1e-14)


def test_fit_exact_when_bond_suffices():
    """B (bond 4) times a rank-1 C has rank <= 4 = the candidate's bond."""
    L = 9
    B = _rand(L, 4, 7)
    C = M.rank1([np.random.default_rng(10 + k).uniform(0.5, 1.5, 2) for k in range(L)])
    A = M.hadamard_fit(B, C, sweeps=2)
    np.testing.assert_allclose(M.to_tensor(A), M.to_tensor(B) * M.to_tensor(C), atol=1e-13)


def test_fit_error_decreases_monotonically():
    L = 8
    B = _rand(L, 3, 8)
    C = _rand(L, 3, 9)
    rec = []
    M.hadamard_fit(B, C, sweeps=2, record=rec)
    assert len(rec) == 4 * L
    for a, b in zip(rec, rec[1:]):
        assert b <= a * (1 + 1e-10) + 1e-28


def test_fit_close_to_svd_truncation():
    """At equal maximal bond the fit lands near the rounding of the exact product."""
    L = 9
    B = M.round_mps(_rand(L, 6, 11), 6, 0.0)
    x = np.linspace(0, 1, 2 ** L)
    C = M.tt_svd(np.cos(3 * x).reshape((2,) * L), 6, 1e-14)
    exact = M.to_tensor(B) * M.to_tensor(C)
    fit = M.to_tensor(M.hadamard_fit(B, C))
    rnd = M.to_tensor(M.round_mps(M.hadamard_exact(B, C), 6, 0.0))
    e_fit = np.linalg.norm(fit - exact)
    e_rnd = np.linalg.norm(rnd - exact)
    assert e_fit <= 3.0 * e_rnd + 1e-14 * np.linalg.norm(exact)


def test_entry_equals_contracted_tensor():
    A = _rand(7, 5, 11)
    T = M.to_tensor(A)
    rng = np.random.default_rng(4)
    for _ in range(40):
        bits = rng.integers(0, 2, 7)
        assert abs(M.entry(A, bits) - T[tuple(bits)]) <= 1e-13 * np.abs(T).max()
