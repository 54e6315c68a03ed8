"""Pins of the dense BGK oracle: conservation laws, the Poiseuille closed form,
shear-wave decay, and taylor == exact at uniform density."""
import numpy as np
import pytest

import synth
from oracle import lattice, lbm_dense as ld


def _noisy(lat, shape, seed, amp=0.01):
    rng = np.random.default_rng(seed)
    return lat.w[:, None, None, None] * (1 + amp * rng.standard_normal((lat.Q,) + shape))


@pytest.mark.parametrize("name", ["D3Q19", "D3Q15"])
@pytest.mark.parametrize("mode", ["exact", "taylor"])
def test_mass_conservation(name, mode):
    lat = lattice.get(name)
    box = synth.box_obstacle(3, (2, 2, 2), (5, 6, 4)).astype(float)
    f = _noisy(lat, (8, 8, 8), 0) * (1 - box)[None]
    m0 = f.sum()
    for periodic in ((1, 1, 1), (1, 1, 0), (0, 1, 0)):
        g = ld.step(f, lat, 0.7, (1e-3, 2e-3, -1e-3), box, periodic, mode)
        assert abs(g.sum() - m0) <= 1e-14 * m0
        assert np.abs(g * box[None]).max() == 0.0


@pytest.mark.parametrize("name", ["D3Q19", "D3Q15"])
def test_momentum_gain_per_step(name):
    """Exact mode, periodic: sum_x j grows by exactly F per fluid cell (tau F
    enters u_eq, and relaxation by 1/tau passes F on)."""
    lat = lattice.get(name)
    f = _noisy(lat, (8, 8, 8), 1)
    F = np.array([1e-3, 2e-3, -1e-3])
    c = lat.c.astype(float)
    j0 = np.einsum("id,ixyz->d", c, f)
    g = ld.step(f, lat, 0.7, F, None, (1, 1, 1), "exact")
    j1 = np.einsum("id,ixyz->d", c, g)
    np.testing.assert_allclose((j1 - j0) / 8 ** 3, F, atol=1e-16)


def test_poiseuille_closed_form():
    """Body force along x between halfway bounce-back walls at z = -1/2 and
    Nz - 1/2: u_x(z) = F/(2 nu) (z + 1/2)(Nz - z - 1/2).  At tau = 1/2 + sqrt(3/16)
    BGK with halfway bounce-back has no wall slip, so the match is to round-off."""
    lat = lattice.D3Q19
    tau = 0.5 + np.sqrt(3.0 / 16.0)
    nu = (tau - 0.5) / 3.0
    Nz, F = 8, 1e-6
    f = np.broadcast_to(lat.w[:, None, None, None], (lat.Q, 2, 2, Nz)).copy()
    for _ in range(int(7 * Nz * Nz / nu)):
        f = ld.step(f, lat, tau, (F, 0, 0), None, (1, 1, 0), "exact")
    _, u = ld.velocity_out(lat, f, (F, 0, 0))
    z = np.arange(Nz) + 0.5
    ua = F / (2 * nu) * z * (Nz - z)
    assert np.abs(u[0, 0, 0] - ua).max() <= 1e-9 * ua.max()
    assert np.abs(u[1:]).max() <= 1e-14


def test_shear_wave_decay():
    """u_x = A sin(2 pi y / N) decays as exp(-nu k^2 t); the BGK lattice
    viscosity matches nu to O(k^2), i.e. within 0.5 % at N = 32."""
    lat = lattice.D3Q19
    tau, N, A, T = 0.8, 32, 1e-5, 400
    nu = (tau - 0.5) / 3.0
    y = np.arange(N)
    u = np.zeros((3, 2, N, 2))
    u[0] = A * np.sin(2 * np.pi * y / N)[None, :, None]
    f = ld.equilibrium(lat, np.ones((2, N, 2)), u)
    for _ in range(T):
        f = ld.step(f, lat, tau, (0, 0, 0), None, (1, 1, 1), "exact")
    _, u = ld.velocity_out(lat, f)
    amp = np.sum(u[0, 0, :, 0] * np.sin(2 * np.pi * y / N)) * 2 / N
    rate = -np.log(amp / A) / T
    assert abs(rate / (nu * (2 * np.pi / N) ** 2) - 1.0) < 5e-3


def test_taylor_equals_exact_at_uniform_density():
    lat = lattice.D3Q19
    rng = np.random.default_rng(2)
    u = 1e-3 * rng.standard_normal((3, 4, 4, 4))
    f = ld.equilibrium(lat, np.ones((4, 4, 4)), u)
    f = f / f.sum(0, keepdims=True)               # rho = 1 exactly everywhere
    a = ld.step(f, lat, 0.8, (0, 0, 0), None, (1, 1, 1), "taylor")
    b = ld.step(f, lat, 0.8, (0, 0, 0), None, (1, 1, 1), "exact")
    np.testing.assert_allclose(a, b, atol=1e-16)


def test_equilibrium_moments():
    lat = lattice.D3Q15
    rng = np.random.default_rng(3)
    rho = 1 + 0.01 * rng.standard_normal((3, 3, 3))
    u = 0.01 * rng.standard_normal((3, 3, 3, 3))
    feq = ld.equilibrium(lat, rho, u)
    r, j = ld.moments(lat, feq)
    np.testing.assert_allclose(r, rho, atol=1e-15)
    np.testing.assert_allclose(j, rho[None] * u, atol=1e-15)
