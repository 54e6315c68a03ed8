"""GPU parity of the MPS primitives (through the C ABI) against the oracle.

Every comparison is on contracted tensors (MPS cores are fixed only up to a
gauge).  FP64: round-off tolerances; FP32: 1e-5 relative for linear algebra.
"""
import numpy as np
import pytest

import synth
from oracle import mpo, mps as M, quantics as q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_07615_gb300 as pkg
    from paper_2512_07615_gb300 import tnlbm as T
    return T


TOL = {0: 1e-12, 1: 2e-5}


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def rnd(L, chi, seed):
    return synth.random_mps(L, synth.feasible_ranks(L, chi), seed)


def smooth_field(n, seed, n_modes=6, amp=0.1, kmax=3):
    N = 1 << n
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.random.default_rng(seed)
    f = np.ones((N, N, N))
    for _ in range(n_modes):
        k = r.integers(-kmax, kmax + 1, 3)
        f += amp * r.standard_normal() * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / N + r.uniform(0, 6))
    return f


@pytest.mark.parametrize("prec", [0, 1])
def test_materialize_terms(tl, prec):
    L = 9
    A, B = rnd(L, 4, 1), rnd(L, 3, 2)
    dA = tl.DeviceMps.from_cores(A, 8, prec)
    dB = tl.DeviceMps.from_cores(B, 8, prec)
    vecs = np.random.default_rng(5).uniform(0.5, 1.5, (L, 2))
    cases = [(tl.plain(dA, -2.5), M.scale(A, -2.5)),
             (tl.kron(dA, dB, 0.5), M.scale(M.hadamard_exact(A, B), 0.5)),
             (tl.mask1(dA, vecs), M.mask_rank1(A, vecs))]
    for axis in range(3):
        for off in (1, -1):
            for cyc in (True, False):
                cases.append((tl.shift(dA, axis, off, cyc), M.apply_mpo(mpo.shift_mpo(3, axis, off, cyc), A)))
    for spec, ref in cases:
        D = tl.DeviceMps(L, 64, prec)
        tl.materialize([spec], [D])
        assert D.bonds() == M.ranks(ref)
        assert rel(M.to_tensor(D.cores()), M.to_tensor(ref)) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_lincomb_round_untruncated_ragged_batch(tl, prec):
    """A batch of jobs with different bonds, all ranks kept."""
    L = 12
    batch, refs = [], []
    dsts = []
    keep = []
    for b in range(5):
        A, B = rnd(L, 2 + b, 10 + b), rnd(L, 5 - b // 2, 20 + b)
        dA, dB = tl.DeviceMps.from_cores(A, 16, prec), tl.DeviceMps.from_cores(B, 16, prec)
        keep += [dA, dB]
        batch.append([tl.plain(dA, 1.0), tl.plain(dB, -0.7), tl.ones(0.25)])
        refs.append(M.lincomb_round([(1.0, A), (-0.7, B), (0.25, M.ones(L))], 32, 0.0))
        dsts.append(tl.DeviceMps(L, 32, prec))
    tl.lincomb_round(batch, dsts, 32, 0.0)
    for D, R in zip(dsts, refs):
        assert rel(M.to_tensor(D.cores()), M.to_tensor(R)) < TOL[prec]
        assert D.bonds() == M.ranks(R)


@pytest.mark.parametrize("prec", [0, 1])
def test_round_truncation_gapped(tl, prec):
    """chi cut inside a clear spectral gap: same bonds and values as the oracle,
    and the Eckart-Young optimum at a single truncated bond."""
    Mat = np.random.default_rng(4).standard_normal((8, 8))
    u, s, vt = np.linalg.svd(Mat)
    s = np.array([4, 3, 2, 1.5, 1.0, 1e-3, 5e-4, 1e-4])
    Mat = (u * s) @ vt
    A = M.tt_svd(Mat.reshape((2,) * 6), 10 ** 6, 0.0)
    dA = tl.DeviceMps.from_cores(A, 8, prec)
    D = tl.DeviceMps(6, 8, prec)
    tl.lincomb_round([[tl.plain(dA)]], [D], 5, 0.0)
    assert D.bonds() == [1, 2, 4, 5, 4, 2, 1]
    got = M.to_tensor(D.cores()).reshape(8, 8)
    err2 = np.sum((got - Mat) ** 2)
    assert abs(err2 - np.sum(s[5:] ** 2)) < (1e-10 if prec == 0 else 1e-5) * np.sum(s ** 2)


@pytest.mark.parametrize("prec", [0, 1])
def test_round_eps_truncation_matches_oracle(tl, prec):
    n = 4
    L = 12
    X = M.tt_svd(q.encode(smooth_field(n, 3)), 64, 0.0)
    Y = M.tt_svd(q.encode(smooth_field(n, 4)), 64, 0.0)
    dX, dY = tl.DeviceMps.from_cores(X, 64, prec), tl.DeviceMps.from_cores(Y, 64, prec)
    for eps in (1e-3, 1e-8):
        ref = M.lincomb_round([(1.0, X), (2.0, Y)], 64, eps)
        D = tl.DeviceMps(L, 64, prec)
        tl.lincomb_round([[tl.plain(dX), tl.plain(dY, 2.0)]], [D], 64, eps)
        exact = M.to_tensor(X) + 2 * M.to_tensor(Y)
        if prec == 0:
            assert D.bonds() == M.ranks(ref)
            assert rel(M.to_tensor(D.cores()), M.to_tensor(ref)) < max(1e-12, 1e-3 * eps)
        assert rel(M.to_tensor(D.cores()), exact) <= eps * (1 + 1e-6) + TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_round_large_bonds_global_memory_path(tl, prec):
    """Wide sums whose QR panels exceed shared memory (several tiles, ragged)."""
    L = 15
    terms, ref_terms, keep = [], [], []
    for t in range(4):
        A = rnd(L, 40 + 7 * t, 30 + t)
        d = tl.DeviceMps.from_cores(A, 64, prec)
        keep.append(d)
        terms.append(tl.plain(d, 1.0 / (t + 1)))
        ref_terms.append((1.0 / (t + 1), A))
    D = tl.DeviceMps(L, 128, prec)
    tl.lincomb_round([terms], [D], 128, 0.0)
    ref = M.lincomb_round(ref_terms, 128, 0.0)
    assert rel(M.to_tensor(D.cores()), M.to_tensor(ref)) < (1e-11 if prec == 0 else 2e-4)


@pytest.mark.parametrize("prec", [0, 1])
def test_round_edge_cases(tl, prec):
    L = 6
    one = tl.DeviceMps.from_cores(M.ones(L), 2, prec)
    # exact cancellation, chi = 1, rank-one inputs, a single term
    for terms, chi, ref in [([tl.plain(one), tl.plain(one, -1.0)], 4, 0.0 * M.to_tensor(M.ones(L))),
                            ([tl.plain(one), tl.ones(2.0)], 1, 3.0 * M.to_tensor(M.ones(L))),
                            ([tl.ones(-1.5)], 3, -1.5 * M.to_tensor(M.ones(L)))]:
        D = tl.DeviceMps(L, 4, prec)
        tl.lincomb_round([terms], [D], chi, 0.0)
        got = M.to_tensor(D.cores())
        assert np.abs(got - ref).max() < (1e-14 if prec == 0 else 1e-6)
        assert max(D.bonds()) <= max(chi, 2)
    with pytest.raises(Exception):
        tl.lincomb_round([[tl.plain(one)]], [tl.DeviceMps(L, 4, prec)], 8, 0.0)   # chi > capacity


@pytest.mark.parametrize("prec", [0, 1])
def test_inner_ones_and_dense(tl, prec):
    L = 12
    X = rnd(L, 9, 7)
    dX = tl.DeviceMps.from_cores(X, 16, prec)
    v = tl.inner_ones([dX, dX]).cpu().numpy()
    ref = M.inner_ones(X)
    assert abs(v[0] - ref) <= TOL[prec] * np.abs(M.to_tensor(X)).sum()
    d = tl.to_dense(dX).double().cpu().numpy()
    assert rel(d, q.decode(M.to_tensor(X))) < TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_from_dense_mask_builder(tl, prec):
    import torch
    box = synth.box_obstacle(4, (3, 5, 2), (11, 9, 13)).astype(np.float64)
    ref = M.tt_svd(q.encode(box), 16, 1e-12)
    X = tl.from_dense(torch.tensor(box, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda"),
                      16, 16, 1e-12)
    assert X.bonds() == M.ranks(ref)
    assert rel(M.to_tensor(X.cores()), q.encode(box)) < (1e-12 if prec == 0 else 1e-6)
    # a truncated sphere pack: same bonds, error close to the oracle's own
    sp = synth.sphere_pack(4, 3.0, 0.3, 1).astype(np.float64)
    ref = M.tt_svd(q.encode(sp), 8, 0.0)
    X = tl.from_dense(torch.tensor(sp, dtype=torch.float64, device="cuda"), 8, 8, 0.0)
    assert X.bonds() == M.ranks(ref)
    e_ref = rel(M.to_tensor(ref), q.encode(sp))
    assert abs(rel(M.to_tensor(X.cores()), q.encode(sp)) - e_ref) < 1e-6 * max(e_ref, 1)


@pytest.mark.parametrize("prec", [0, 1])
def test_fit_exact_when_candidate_bond_suffices(tl, prec):
    L = 12
    B = rnd(L, 24, 11)            # several 64-wide GEMM tiles after contraction
    C = M.rank1([np.random.default_rng(k).uniform(0.5, 1.5, 2) for k in range(L)])
    C = M.round_mps(M.add(C, M.scale(C, 0.5)), 4, 0.0)
    dB, dC = tl.DeviceMps.from_cores(B, 24, prec), tl.DeviceMps.from_cores(C, 4, prec)
    A = tl.DeviceMps(L, 24, prec)
    tl.hadamard_fit([dB], [dC], [A], sweeps=2)
    exact = M.to_tensor(B) * M.to_tensor(C)
    assert rel(M.to_tensor(A.cores()), exact) < (1e-11 if prec == 0 else 5e-5)


def test_fit_well_conditioned_truncation_matches_oracle(tl):
    """Truncating fit (candidate bond 4 < product rank) on a case whose ALS is
    well conditioned: the GPU reproduces the oracle's fit, not just its error."""
    n = 4
    B = M.tt_svd(q.encode(smooth_field(n, 1)), 4, 0.0)
    C = M.tt_svd(q.encode(smooth_field(n, 2)), 4, 0.0)
    ref = M.hadamard_fit(B, C, 2)
    dB, dC = tl.DeviceMps.from_cores(B, 4, 0), tl.DeviceMps.from_cores(C, 4, 0)
    A = tl.DeviceMps(3 * n, 4, 0)
    tl.hadamard_fit([dB, dB], [dC, dC], [A, tl.DeviceMps(3 * n, 4, 0)], sweeps=2)
    assert rel(M.to_tensor(A.cores()), M.to_tensor(ref)) < 1e-8
    exact = M.to_tensor(B) * M.to_tensor(C)
    assert abs(rel(M.to_tensor(A.cores()), exact) - rel(M.to_tensor(ref), exact)) < 1e-8


@pytest.mark.parametrize("prec", [0, 1])
def test_fit_quality_in_ill_conditioned_regime(tl, prec):
    """Where the ALS result is not a well-conditioned function of its inputs
    (saturated bonds, near-degenerate cut), compare approximation quality."""
    n = 4
    B = M.tt_svd(q.encode(smooth_field(n, 1)), 8, 0.0)
    C = M.tt_svd(q.encode(smooth_field(n, 2)), 8, 0.0)
    exact = M.to_tensor(B) * M.to_tensor(C)
    e_ref = rel(M.to_tensor(M.hadamard_fit(B, C, 2)), exact)
    dB, dC = tl.DeviceMps.from_cores(B, 8, prec), tl.DeviceMps.from_cores(C, 8, prec)
    A = tl.DeviceMps(3 * n, 8, prec)
    tl.hadamard_fit([dB], [dC], [A], sweeps=2)
    e_gpu = rel(M.to_tensor(A.cores()), exact)
    assert e_gpu <= 1.5 * e_ref + 1e-6
