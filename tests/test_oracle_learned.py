"""Pins of the learned-rank pieces of the oracle: MLP gradients against
finite differences; the randomized truncation against the full SVD where the
sample covers the spectrum, and its certificate rejecting samples that miss."""
import numpy as np

import synth
from oracle import learned as LR
from oracle import mps as M


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(0)
    P = LR.mlp_init(3)
    X = rng.standard_normal((7, LR.N_FEAT))
    y = rng.uniform(0, 1, 7)
    loss, g = LR.mlp_loss_grad(P, X, y)
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = LR.mlp_loss_grad(P, X, y)
            flat[idx] = old - h
            lm, _ = LR.mlp_loss_grad(P, X, y)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd))


def _mat(m, n, s, seed):
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((m, len(s))))
    V, _ = np.linalg.qr(rng.standard_normal((n, len(s))))
    return (U * s) @ V.T


def test_rsvd_full_sample_equals_svd():
    C = _mat(20, 12, np.linspace(3, 0.1, 12), 1)
    omega = synth.gaussian_matrix(64, 64, 5)
    ok, r, US, Vt, err2, res2 = LR.rsvd_truncate(C, 12, omega, 6, 0.0)
    U, S, Wt = np.linalg.svd(C, full_matrices=False)
    ref = (U[:, :6] * S[:6]) @ Wt[:6]
    assert ok and r == 6 and res2 < 1e-20
    np.testing.assert_allclose(US @ Vt, ref, atol=1e-12)
    assert abs(err2 - np.sum(S[6:] ** 2)) < 1e-12


def test_rsvd_gap_accepted_and_certificate_rejects_misses():
    s = np.concatenate([np.linspace(2, 1, 5), 1e-6 * 0.5 ** np.arange(25)])
    C = _mat(40, 40, s, 2)
    omega = synth.gaussian_matrix(64, 64, 6)
    ok, r, US, Vt, err2, res2 = LR.rsvd_truncate(C, 5, omega, 5, 0.0)
    assert ok and r == 5
    U, S, Wt = np.linalg.svd(C)
    np.testing.assert_allclose(US @ Vt, (U[:, :5] * S[:5]) @ Wt[:5], atol=1e-9)
    flat = _mat(40, 40, np.ones(40), 3)                  # no decay: a small sample misses mass
    ok, r, *_ = LR.rsvd_truncate(flat, 5, omega, 30, 0.0, p=2)
    assert not ok


def test_round_learned_without_targets_is_round():
    L = 9
    A = M.add(synth.random_mps(L, synth.feasible_ranks(L, 5), 1), synth.random_mps(L, synth.feasible_ranks(L, 4), 2))
    omega = synth.gaussian_matrix(128, 128, 7)
    a, na, nf = LR.round_mps_learned(A, 6, 1e-12, None, omega)
    b = M.round_mps(A, 6, 1e-12)
    np.testing.assert_allclose(M.to_tensor(a), M.to_tensor(b), atol=1e-12)
    assert na == 0 and nf == 0


def test_round_learned_redundant_sum_is_exact():
    """A + 0.5 A has twice the bond of its rank: the sample at target = rank
    covers the range, every randomized step is accepted, result 1.5 A."""
    L = 12
    A = synth.random_mps(L, synth.feasible_ranks(L, 16), 4)
    S = M.add(A, M.scale(A, 0.5))
    omega = synth.gaussian_matrix(128, 128, 8)
    c, na, nf = LR.round_mps_learned(S, 64, 1e-12, [0] + [16] * (L - 1) + [0], omega)
    assert na >= 3 and nf == 0
    np.testing.assert_allclose(M.to_tensor(c), 1.5 * M.to_tensor(A), atol=1e-11)


def test_certificate_lower_bound_and_near_optimality():
    """The inequality the certificate rests on: opt(r)^2 >= err(r)^2 - ||E||^2
    (Ky Fan on C^T C = B^T B + E^T E), checked against the exact SVD; and every
    accepted chi-capped truncation is within 1 / (1 - eta) of the optimum."""
    omega = synth.gaussian_matrix(128, 128, 9)
    rng = np.random.default_rng(10)
    n_acc = 0
    for trial in range(12):
        m, n = 70 + trial, 64
        s = np.exp(-rng.uniform(0.02, 0.3) * np.arange(n))
        C = _mat(m, n, s, 100 + trial)
        for k, q in ((20, 0), (20, 1), (32, 1)):
            ok, r, US, Vt, err2, res2 = LR.rsvd_truncate(C, k, omega, k, 0.0, q=q)
            sv = np.linalg.svd(C, compute_uv=False)
            opt2 = np.sum(sv[r:] ** 2)
            true2 = np.sum((C - US @ Vt) ** 2)
            assert abs(true2 - err2) <= 1e-10 * np.sum(sv ** 2)
            assert opt2 >= err2 - res2 - 1e-12 * np.sum(sv ** 2)
            if ok:
                n_acc += 1
                assert err2 <= opt2 / (1 - 0.2) * (1 + 1e-10)
    assert n_acc > 0


def test_spectrum_features():
    f = LR.spectrum_features(np.array([4.0, 2.0, 0.4]), 3, 12, 500)
    assert f.shape == (18,)
    np.testing.assert_allclose(f[:3], [0.0, np.log10(0.5), np.log10(0.1)])
    assert f[3] == -20.0 and f[16] == 0.25 and f[17] == 0.5


def _gauge(cores, seed):
    """Same tensor, random orthogonal change of basis on every interior bond."""
    rng = np.random.default_rng(seed)
    out = [c.copy() for c in cores]
    for k in range(1, len(cores)):
        r = out[k].shape[0]
        G, _ = np.linalg.qr(rng.standard_normal((r, r)))
        out[k - 1] = np.tensordot(out[k - 1], G, axes=(2, 0))
        out[k] = np.tensordot(G.T, out[k], axes=(1, 0))
    return out


def test_learned_rounding_is_gauge_independent():
    """With the sign gauge fixed at every step, the randomized result depends
    only on the tensor, not on the gauge of the input cores.  Input: a smooth
    16^3 field (decaying spectra) capped at chi = 8, so that the randomized
    steps are chi-limited and certified."""
    from oracle import quantics as qq
    N = 16
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    rng = np.random.default_rng(11)
    f = np.ones((N, N, N))
    for j in range(24):
        kv = rng.integers(-7, 8, 3)
        f += 0.7 ** j * np.cos(2 * np.pi * (kv[0] * X + kv[1] * Y + kv[2] * Z) / N + rng.uniform(0, 6))
    A = M.tt_svd(qq.encode(f), 64, 1e-14)
    B = _gauge(A, 12)
    L = len(A)
    omega = synth.gaussian_matrix(64, 64, 13)
    tg = [0] + [16] * (L - 1) + [0]
    a, na, nf = LR.round_mps_learned(A, 16, 1e-12, tg, omega)
    b, nb, nfb = LR.round_mps_learned(B, 16, 1e-12, tg, omega)
    assert na > 0 and (na, nf) == (nb, nfb)
    np.testing.assert_allclose(M.to_tensor(a), M.to_tensor(b), atol=1e-11 * np.abs(M.to_tensor(a)).max())


def test_sign_gauge_on_tied_entries():
    """Rows with entries of equal magnitude (where a largest-entry rule is
    ambiguous) get the sign that makes their probe product positive."""
    r2 = 1 / np.sqrt(2)
    Vt = np.array([[r2, -r2], [-r2, r2], [-r2, -r2]])
    US = np.eye(3)[:, :3] * np.array([1.0, 2.0, 3.0])
    w = LR.sign_probe(2)
    assert w[0] != w[1] and (w > 0).all()
    U2, V2 = LR.canonical_signs(US, Vt)
    assert (V2 @ w > 0).all()
    np.testing.assert_array_equal(V2[0], Vt[0])
    np.testing.assert_array_equal(V2[1], -Vt[1])
    np.testing.assert_array_equal(V2[2], -Vt[2])
    np.testing.assert_array_equal(U2 @ V2, US @ Vt)
