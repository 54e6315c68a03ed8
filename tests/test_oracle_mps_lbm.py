"""Pins of the MPS-LBM step: with nothing truncated it reproduces the dense
Taylor-mode step to round-off; its rank-1 wall masks and mode MPS equal their
dense definitions."""
import numpy as np
import pytest

import synth
from oracle import lattice, lbm_dense as ld, mps as M, mps_lbm as ml, quantics as q
from oracle.metrics import rel_l2


def test_wall_terms_equal_boundary_mask():
    n = 3
    for c in [(1, 0, 1), (0, -1, 1), (1, 1, -1), (-1, 0, 0)]:
        for periodic in [(1, 1, 0), (0, 1, 0), (0, 0, 0)]:
            tot = np.zeros((8, 8, 8))
            for coef, vecs in ml.wall_terms(n, c, periodic):
                tot += coef * q.decode(M.to_tensor(M.rank1(vecs)))
            np.testing.assert_array_equal(tot, ld.boundary_mask((8, 8, 8), c, periodic))


def test_fourier_mode_mps():
    n = 3
    N = 8
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    for k, ph in [((1, 0, 0), 0.3), ((2, -3, 1), 1.7), ((0, 0, 4), 0.0)]:
        ref = np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / N + ph)
        got = q.decode(M.to_tensor(ml.fourier_mode_mps(n, k, ph)))
        np.testing.assert_allclose(got, ref, atol=1e-14)


def test_tree_sum():
    cfg = ml.Config(2, lattice.D3Q19, 0.8, chi_max=64, eps=0.0)
    items = [(float(i + 1), synth.random_mps(6, synth.feasible_ranks(6, 2), i)) for i in range(7)]
    ref = sum(c * M.to_tensor(X) for c, X in items)
    np.testing.assert_allclose(M.to_tensor(ml.tree_sum(cfg, items)), ref, atol=1e-13)


@pytest.mark.parametrize("name", ["D3Q19", "D3Q15"])
def test_untruncated_step_equals_dense_taylor(name):
    lat = lattice.get(name)
    n = 3
    box = synth.box_obstacle(n, (2, 3, 1), (5, 6, 4)).astype(float)
    mask = M.tt_svd(q.encode(box), 10 ** 6, 1e-14)
    cfg = ml.Config(n, lat, 0.8, force=(1e-4, 2e-5, 0.0), periodic=(1, 1, 0),
                    chi_max=10 ** 6, eps=0.0, hadamard="exact", mask=mask)
    modes = synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    f = ml.initial_perturbed(cfg, modes)
    fd = ml.to_dense_populations(f)
    for _ in range(2):
        f = ml.step(cfg, f)
        fd = ld.step(fd, lat, 0.8, cfg.force, box, cfg.periodic, "taylor")
    fm = ml.to_dense_populations(f)
    assert np.abs(fm - fd).max() <= 1e-12 * np.abs(fd).max()
    _, u_dense = ld.velocity_out(lat, fd, cfg.force, box)
    _, u_mps = ml.macroscopic(cfg, f, box)
    assert rel_l2(u_mps, u_dense) <= 1e-10


def test_channel_fit_mode_close_to_exact_mode():
    """The 32^3-style channel (z walls, force along x) on 8^3: the variational
    products stay within 1e-6 of the exact products after a few steps."""
    lat = lattice.D3Q19
    base = dict(n_bits=3, lattice=lat, tau=0.8, force=(1e-6, 0, 0), periodic=(1, 1, 0),
                chi_max=16, eps=1e-10)
    cf = ml.Config(hadamard="fit", **base)
    ce = ml.Config(hadamard="exact", **base)
    f1 = ml.initial_rest(cf)
    f2 = ml.initial_rest(ce)
    for _ in range(3):
        f1 = ml.step(cf, f1)
        f2 = ml.step(ce, f2)
    _, u1 = ml.macroscopic(cf, f1)
    _, u2 = ml.macroscopic(ce, f2)
    assert rel_l2(u1, u2) <= 1e-6
