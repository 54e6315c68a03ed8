"""Pins of the per-face boundary functions (velocity inlet, pressure outlet,
bounce-back walls; Eq. boundaries2 and the conditions of Sec. 3.2):
a uniform stream at the inlet velocity and outlet density is a fixed point of
the whole step; a velocity face with u_b = 0 is the no-slip wall; and the MPS
oracle with faces reproduces the dense oracle to round-off when nothing is
truncated (mixed faces with shared edges, where the lowest axis decides)."""
import numpy as np

import synth
from oracle import lattice, lbm_dense as ld, mps_lbm as ml

W, V, P = ld.FACE_WALL, ld.FACE_VELOCITY, ld.FACE_PRESSURE


def faces_of(spec):
    base = [(W, (0.0, 0.0, 0.0), 1.0)] * 6
    for k, v in spec.items():
        base[k] = v
    return base


def test_uniform_stream_is_a_fixed_point():
    lat = lattice.D3Q19
    N, U = 8, 0.05
    u = np.zeros((3, N, N, N))
    u[0] = U
    f = ld.equilibrium(lat, np.ones((N, N, N)), u)
    faces = faces_of({0: (V, (U, 0.0, 0.0), 1.0), 1: (P, (0.0, 0.0, 0.0), 1.0)})
    for mode in ("exact", "taylor"):
        g = ld.step(f, lat, 0.8, (0.0, 0.0, 0.0), None, (0, 1, 1), mode, faces=faces)
        assert np.abs(g - f).max() <= 1e-15


def test_resting_velocity_face_is_the_wall():
    lat = lattice.D3Q19
    cfg = ml.Config(3, lat, 0.8, periodic=(1, 1, 0), chi_max=64, eps=0.0)
    f = ml.to_dense_populations(ml.initial_perturbed(cfg, synth.fourier_modes(4, 2, kmax=2, amp_rho=1e-2,
                                                                               amp_u=1e-2)))
    faces = faces_of({4: (V, (0.0, 0.0, 0.0), 1.0), 5: (V, (0.0, 0.0, 0.0), 1.0)})
    a = ld.step(f, lat, 0.8, (1e-4, 0, 0), None, (1, 1, 0), "taylor")
    b = ld.step(f, lat, 0.8, (1e-4, 0, 0), None, (1, 1, 0), "taylor", faces=faces)
    np.testing.assert_allclose(b, a, atol=1e-15)


def test_mps_faces_equal_dense_untruncated():
    """8^3: inlet (0.03, 0.01, 0) at x-, outlet density 1.002 at x+, walls at
    z (periodic y); two steps, exact products, nothing truncated."""
    lat = lattice.D3Q19
    faces = faces_of({0: (V, (0.03, 0.01, 0.0), 1.0), 1: (P, (0.0, 0.0, 0.0), 1.002)})
    cfg = ml.Config(3, lat, 0.8, periodic=(0, 1, 0), chi_max=4096, eps=0.0, hadamard="exact", faces=faces)
    modes = synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    f = ml.initial_perturbed(cfg, modes)
    fd = ml.to_dense_populations(f)
    for _ in range(2):
        f = ml.step(cfg, f)
        fd = ld.step(fd, lat, 0.8, (0.0, 0.0, 0.0), None, (0, 1, 0), "taylor", faces=faces)
    got = ml.to_dense_populations(f)
    assert np.abs(got - fd).max() <= 1e-12 * np.abs(fd).max()
    # the boundary terms were active: the result differs from all-wall faces
    fw = ld.step(ml.to_dense_populations(ml.initial_perturbed(cfg, modes)), lat, 0.8, (0, 0, 0), None, (0, 1, 0),
                 "taylor")
    assert np.abs(fw - ld.step(ml.to_dense_populations(ml.initial_perturbed(cfg, modes)), lat, 0.8, (0, 0, 0),
                               None, (0, 1, 0), "taylor", faces=faces)).max() > 1e-4



def test_mps_options_combined_equal_dense_untruncated():
    """The step options together -- zip-up products, block-sum moments, an
    inlet and an outlet with walls, an object mask and a body force -- still
    reproduce the dense step when nothing is truncated (8^3, one step)."""
    from oracle import mps as M, quantics as q
    lat = lattice.D3Q19
    box = synth.box_obstacle(3, (3, 2, 2), (5, 5, 4)).astype(float)
    mask = M.tt_svd(q.encode(box), 10 ** 6, 1e-14)
    faces = faces_of({0: (V, (0.02, 0.0, 0.01), 1.0), 1: (P, (0.0, 0.0, 0.0), 0.999)})
    cfg = ml.Config(3, lat, 0.8, force=(1e-4, 0.0, 0.0), periodic=(0, 1, 0), chi_max=10 ** 6, eps=0.0,
                    hadamard="zipup", block_sums=True, mask=mask, faces=faces)
    f = ml.initial_perturbed(cfg, synth.fourier_modes(3, 9, kmax=2, amp_rho=1e-2, amp_u=1e-2))
    fd = ml.to_dense_populations(f)
    f = ml.step(cfg, f)
    fd = ld.step(fd, lat, 0.8, (1e-4, 0.0, 0.0), box, (0, 1, 0), "taylor", faces=faces)
    assert np.abs(ml.to_dense_populations(f) - fd).max() <= 1e-12 * np.abs(fd).max()
