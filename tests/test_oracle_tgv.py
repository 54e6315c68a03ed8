"""Pins of the Taylor-Green vortex workload: the plane-wave parameters in
synth reproduce the closed-form field, and the dense BGK oracle damps it at
the lattice viscosity nu = (tau - 1/2) / 3 with second-order convergence in
the grid spacing (the decay rate of the energy of the |k|^2 = 3 (2 pi / N)^2
mode is 2 nu |k|^2 in the Stokes limit)."""
import numpy as np

import synth
from oracle import lattice, lbm_dense as ld, mps_lbm as ml


def test_tgv_modes_reproduce_the_closed_form_field():
    n, u0 = 4, 0.05
    N = 1 << n
    cfg = ml.Config(n, lattice.D3Q19, 0.8, chi_max=64, eps=0.0)
    f = ml.to_dense_populations(ml.initial_perturbed(cfg, synth.taylor_green_modes(u0)))
    rho, j = ld.moments(lattice.D3Q19, f)
    x = 2 * np.pi * np.arange(N) / N
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    ux = u0 * np.sin(X) * np.cos(Y) * np.cos(Z)
    uy = -u0 * np.cos(X) * np.sin(Y) * np.cos(Z)
    drho = 3 * u0 ** 2 / 16 * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2)
    np.testing.assert_allclose(rho, 1 + drho, atol=1e-13)
    np.testing.assert_allclose(j[0], ux, atol=1e-13)
    np.testing.assert_allclose(j[1], uy, atol=1e-13)
    np.testing.assert_allclose(j[2], 0.0, atol=1e-13)


def _decay_rate_error(N, tau=0.8, u0=0.01, skip=20, steps=20):
    lat = lattice.D3Q19
    cfg = ml.Config(int(np.log2(N)), lat, tau, chi_max=64, eps=0.0)
    f = ml.to_dense_populations(ml.initial_perturbed(cfg, synth.taylor_green_modes(u0)))
    energies = []
    for t in range(skip + steps + 1):
        if t in (skip, skip + steps):
            _, u = ld.velocity_out(lat, f)
            energies.append(np.sum(u ** 2))
        f = ld.step(f, lat, tau, (0.0, 0.0, 0.0), None, (1, 1, 1), "exact")
    rate = -np.log(energies[1] / energies[0]) / (2 * steps)
    nu = (tau - 0.5) / 3
    return rate / (nu * 3 * (2 * np.pi / N) ** 2) - 1


def test_dense_oracle_damps_tgv_at_the_lattice_viscosity():
    """After the initial layer (20 steps), the energy decay rate is within
    1 % of 2 nu |k|^2 at N = 32 and the error falls by ~4x from N = 16."""
    e16 = _decay_rate_error(16)
    e32 = _decay_rate_error(32)
    assert abs(e32) < 0.01
    assert 3.5 < e16 / e32 < 4.5
