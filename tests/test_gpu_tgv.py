"""GPU Taylor-Green vortex: with products formed exactly (FP64) the library's
MPS step equals the oracle's on the same truncation; the production path
(FP32, variational products, chi = 64 above every bond the vortex reaches in
10 steps at 32^3) keeps the velocity field and its kinetic energy within 1e-3
of the dense BGK oracle."""
import numpy as np
import pytest

import synth
from oracle import lattice, lbm_dense as ld, mps_lbm as ml
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_07615_gb300 as pkg
    return pkg


def dense_run(n, tau, u0, steps, inv_mode):
    lat = lattice.D3Q19
    cfg = ml.Config(n, lat, tau, chi_max=64, eps=0.0)
    f = ml.to_dense_populations(ml.initial_perturbed(cfg, synth.taylor_green_modes(u0)))
    for _ in range(steps):
        f = ld.step(f, lat, tau, (0.0, 0.0, 0.0), None, (1, 1, 1), inv_mode)
    return ld.velocity_out(lat, f)


def test_tgv_exact_products_match_oracle_mps(tl):
    """16^3, FP64, products formed exactly, chi = 32 (population bonds grow 14 ->
    24 -> 32 in the first steps): the same algorithm and truncation as the
    oracle's MPS step, 3 steps."""
    n, tau, u0, steps = 4, 0.8, 0.05, 3
    modes = synth.taylor_green_modes(u0)
    sim = tl.Sim(n, tau=tau, periodic=(1, 1, 1), chi_max=32, eps=1e-13, precision=0, hadamard=1, modes=modes)
    sim.step(steps)
    rho, u = sim.macroscopic()
    cfg = ml.Config(n, lattice.D3Q19, tau, chi_max=32, eps=1e-13, hadamard="exact")
    f = ml.initial_perturbed(cfg, modes)
    for _ in range(steps):
        f = ml.step(cfg, f)
    rho_o, u_o = ml.macroscopic(cfg, f)
    assert rel_l2(u, u_o) <= 1e-9
    assert np.abs(rho - rho_o).max() <= 1e-11
    assert sim.stats()["max_bond"] <= 32
    sim.close()


def test_tgv_production_path_fp32(tl):
    n, tau, u0, steps = 5, 0.8, 0.05, 10
    sim = tl.Sim(n, tau=tau, periodic=(1, 1, 1), chi_max=64, eps=1e-7, precision=1, hadamard=0,
                 modes=synth.taylor_green_modes(u0), conserve_mass=True)
    rho0, _ = sim.macroscopic()
    sim.step(steps)
    rho, u = sim.macroscopic()
    rho_d, u_d = dense_run(n, tau, u0, steps, "exact")
    assert rel_l2(u, u_d) <= 1e-3
    e, e_d = np.sum(u ** 2), np.sum(u_d ** 2)
    assert abs(e - e_d) / e_d <= 1e-3
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() <= 1e-6        # drift of its own mass
    sim.close()


def test_tgv_fp64_near_half_tau_tracks_dense_energy(tl):
    """Near tau = 1/2 (tau = 0.5038, omega ~ 1.985) the FP64 path keeps the
    dense oracle's kinetic-energy history (16^3, chi 32, eps 1e-10, 100
    steps): E/E0 at every 25 steps within 1e-6."""
    n, tau, u0, steps = 4, 0.5038, 0.05, 100
    sim = tl.Sim(n, tau=tau, periodic=(1, 1, 1), chi_max=32, eps=1e-10, precision=0, hadamard=0,
                 modes=synth.taylor_green_modes(u0))
    lat = lattice.D3Q19
    cfg = ml.Config(n, lat, tau, chi_max=64, eps=0.0)
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, synth.taylor_green_modes(u0)))
    e_mps, e_dense = [], []
    for t in range(0, steps + 1, 25):
        if t:
            sim.step(25)
            for _ in range(25):
                fd = ld.step(fd, lat, tau, (0.0, 0.0, 0.0), None, (1, 1, 1), "taylor")
        rho, u = sim.macroscopic()
        e_mps.append(0.5 * float(np.sum(rho * np.sum(u ** 2, axis=0))))
        rd, ud = ld.velocity_out(lat, fd)
        e_dense.append(0.5 * float(np.sum(rd * np.sum(ud ** 2, axis=0))))
    for a, b in zip(e_mps, e_dense):
        assert abs(a / e_mps[0] - b / e_dense[0]) <= 1e-6
    assert e_dense[-1] < e_dense[0]
    sim.close()
