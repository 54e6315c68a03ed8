"""Pins of the zip-up product (oracle.mps.zipup_pass / hadamard_zipup, the
alternative to the fit that Sec. 2.3 names): exact when nothing is
truncated; with the all-ones MPS as second factor the pass is the
left-to-right truncated SVD sweep of the first, i.e. the mirror image of the
rounding's right-to-left sweep (Eq. svd-move), ranks included; and on smooth
fields (factors given left-canonical, as the TT-SVD leaves them) the
truncated product stays within 1.5x of the error of rounding the exact
product at the same bond, where the pass alone on those factors is not."""
import numpy as np

import synth
from oracle import mps as M


def _rand(L, chi, seed):
    return synth.random_mps(L, synth.feasible_ranks(L, chi), seed)


def _rel(X, Y):
    return np.linalg.norm(X - Y) / np.linalg.norm(Y)


def _reverse(A):
    return [c.transpose(2, 1, 0).copy() for c in A[::-1]]


def test_exact_without_truncation():
    B, C = _rand(7, 3, 1), _rand(7, 4, 2)
    exact = M.to_tensor(B) * M.to_tensor(C)
    assert _rel(M.to_tensor(M.zipup_pass(B, C, 64, 0.0)), exact) < 1e-12
    Z = M.hadamard_zipup(B, C, 64, 0.0)
    assert _rel(M.to_tensor(Z), exact) < 1e-12
    # the pass is left-orthogonal up to its last core
    for c in M.zipup_pass(B, C, 64, 0.0)[:-1]:
        Q = c.reshape(-1, c.shape[2])
        np.testing.assert_allclose(Q.T @ Q, np.eye(Q.shape[1]), atol=1e-12)


def test_ones_factor_is_the_mirrored_rounding_sweep():
    B = M.right_orthogonalize(_rand(8, 9, 3))
    one = M.ones(8)
    for chi, eps in [(4, 0.0), (16, 1e-2), (6, 1e-3)]:
        Z = M.zipup_pass(B, one, chi, eps)
        R = _reverse(M.round_mps(_reverse(B), chi, eps))
        assert M.ranks(Z) == M.ranks(R)
        assert _rel(M.to_tensor(Z), M.to_tensor(R)) < 1e-12


def test_smooth_product_close_to_best_at_equal_bond():
    rng = np.random.default_rng(5)
    n = 4
    N = 1 << n
    x = np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = 1 + 0.3 * np.sin(2 * np.pi * (X + 2 * Y)) * np.cos(2 * np.pi * Z) + 0.1 * rng.standard_normal() * X * Y
    g = 1 + 0.2 * np.cos(2 * np.pi * (3 * X - Y + Z))
    from oracle import quantics as q
    B = M.tt_svd(q.encode(f), 64, 1e-12)
    C = M.tt_svd(q.encode(g), 64, 1e-12)
    exact = M.to_tensor(B) * M.to_tensor(C)
    for chi in (4, 6, 8):
        best = _rel(M.to_tensor(M.round_mps(M.hadamard_exact(B, C), chi, 0.0)), exact)
        got = _rel(M.to_tensor(M.hadamard_zipup(B, C, chi, 0.0)), exact)
        assert max(M.ranks(M.hadamard_zipup(B, C, chi, 0.0))) <= chi
        assert got <= 1.5 * best + 1e-14, (chi, got, best)
    # the right-canonical form matters: the pass on the left-canonical factors
    raw = _rel(M.to_tensor(M.round_mps(M.zipup_pass(B, C, 4, 0.0), 4, 0.0)), exact)
    assert raw > 0.5


def test_untruncated_zipup_step_equals_dense_taylor():
    """The oracle step with zip-up products, nothing truncated, reproduces the
    dense Taylor step (as the exact-product step does)."""
    from oracle import lattice, lbm_dense as ld, mps_lbm as ml, quantics as q
    from oracle.metrics import rel_l2
    lat = lattice.D3Q19
    n = 3
    box = synth.box_obstacle(n, (2, 3, 1), (5, 6, 4)).astype(float)
    mask = M.tt_svd(q.encode(box), 10 ** 6, 1e-14)
    cfg = ml.Config(n, lat, 0.8, force=(1e-4, 2e-5, 0.0), periodic=(1, 1, 0),
                    chi_max=10 ** 6, eps=0.0, hadamard="zipup", mask=mask)
    modes = synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    f = ml.initial_perturbed(cfg, modes)
    fd = ml.to_dense_populations(f)
    f = ml.step(cfg, f)
    fd = ld.step(fd, lat, 0.8, cfg.force, box, cfg.periodic, "taylor")
    assert np.abs(ml.to_dense_populations(f) - fd).max() <= 1e-12 * np.abs(fd).max()
    _, u_dense = ld.velocity_out(lat, fd, cfg.force, box)
    _, u_mps = ml.macroscopic(cfg, f, box)
    assert rel_l2(u_mps, u_dense) <= 1e-10
