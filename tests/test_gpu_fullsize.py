"""Full-size workloads, in the launch configuration the benchmark times,
checked on outputs the oracle computes one by one: entries of the
populations' MPS at seeded sample cells (Eq. MPS at fixed indices, with the
scale-ordered site bits of Sec. 2.4) summed into rho and rho u, against the
library's contracted macroscopic fields; one rounding of two full-size
populations against the oracle's rounding of the same pair at sampled cells;
and the properties that hold at any size (mass, finiteness, bonds within chi,
device status)."""
import numpy as np
import pytest

import synth
from oracle import lattice, mps as M, quantics as q

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


def _sample_cells(n, count, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, 1 << n, size=(count, 3))


def _mask_cores(tl, solid, chi):
    """The object mask m_O as the library compresses it (TT-SVD on the device,
    eps 1e-8), handed to the simulation as its mask so that the sampled
    check knows m_O(x) at every cell."""
    import torch
    m = tl.from_dense(torch.tensor(solid, dtype=torch.float64, device="cuda"), chi, chi, 1e-8)
    return m.cores()


def _check_macroscopic_at_samples(sim, n, mask, force, cells):
    """rho = sum_i f_i and rho u - F (1 - m_O) / 2 = sum_i c_i f_i at each
    sampled cell, from oracle entries of the library's own populations and
    mask."""
    rho, u = sim.macroscopic()
    pops = sim.get_populations()
    c = np.asarray(lattice.D3Q19.c, dtype=np.float64)
    N = 1 << n
    for x, y, z in cells:
        bits = q.site_bits(n, (x, y, z))
        f = np.array([M.entry(p, bits) for p in pops])
        flat = (x * N + y) * N + z
        r_gpu = rho.reshape(-1)[flat]
        assert abs(r_gpu - f.sum()) <= 2e-5
        fluid = 1.0 - M.entry(mask, bits)
        j_gpu = np.array([u[d].reshape(-1)[flat] for d in range(3)]) * r_gpu - 0.5 * np.asarray(force) * fluid
        if r_gpu > 0.5:
            assert np.abs(j_gpu - c.T @ f).max() <= 2e-6


def test_porous_128cubed_sampled_outputs_vs_oracle(tl):
    """128^3 sphere pack (radius 10, 35 % solid), chi 64, FP32, two steps
    (the mask compressed as the library does, passed in as cores)."""
    n, force = 7, (1e-5, 0.0, 0.0)
    sp = synth.sphere_pack(n, 10.0, 0.35, 0)
    modes = synth.fourier_modes(31, 0, kmax=4, amp_rho=1e-3, amp_u=1e-3)
    mask = _mask_cores(tl, sp, 64)
    sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), mask_cores=mask, force=force,
                 chi_max=64, eps=1e-7, precision=1, hadamard=0, modes=modes, conserve_mass=True)
    sim.step(2)
    _check_macroscopic_at_samples(sim, n, mask, force, _sample_cells(n, 200, 1))
    # one rounding of a full-size pair (the first level of the moment fold)
    pops = sim.get_populations()
    L = 3 * n
    A = tl.DeviceMps.from_cores(pops[1], 64, 1)
    B = tl.DeviceMps.from_cores(pops[2], 64, 1)
    D = tl.DeviceMps(L, 64, 1)
    tl.lincomb_round([[tl.tnlbm.plain(A), tl.tnlbm.plain(B)]], [D], 64, 1e-7)
    got = D.cores()
    ref = M.lincomb_round([(1.0, pops[1]), (1.0, pops[2])], 64, 1e-7)
    exact_err, gpu_err = [], []
    for x, y, z in _sample_cells(n, 200, 2):
        bits = q.site_bits(n, (x, y, z))
        exact = M.entry(pops[1], bits) + M.entry(pops[2], bits)
        exact_err.append(abs(M.entry(ref, bits) - exact))
        gpu_err.append(abs(M.entry(got, bits) - exact))
    scale = 2 * lattice.D3Q19.w[1]
    assert max(gpu_err) <= 2 * max(exact_err) + 1e-5 * scale
    sim.close()


def test_vessel_256cubed_sampled_outputs_and_properties(tl):
    """256^3 branching vessel (depth 4, Murray radii from 24 cells), chi 128,
    FP32, one step: mass to 1e-6, finite fields, bonds within chi, no device
    error, and the sampled macroscopic fields against oracle entries."""
    n, force = 8, (1e-5, 0.0, 0.0)
    vs = synth.vessel_tree(n, 24.0, 4, 0)
    modes = synth.fourier_modes(31, 0, kmax=4, amp_rho=1e-3, amp_u=1e-3)
    mask = _mask_cores(tl, vs, 128)
    sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), mask_cores=mask, force=force,
                 chi_max=128, eps=1e-7, precision=1, hadamard=0, modes=modes, conserve_mass=True)
    rho0, _ = sim.macroscopic()
    sim.step(1)
    rho, u = sim.macroscopic()
    assert np.isfinite(u).all() and np.isfinite(rho).all()
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() <= 1e-6
    st = sim.stats()
    assert st["max_bond"] <= 128 and st["status"] == 0
    _check_macroscopic_at_samples(sim, n, mask, force, _sample_cells(n, 100, 3))
    # one rounding of a full-size pair at chi 128 (256 x 256 centre matrices,
    # held in global memory: the block Jacobi path)
    pops = sim.get_populations()
    L = 3 * n
    A = tl.DeviceMps.from_cores(pops[7], 128, 1)
    B = tl.DeviceMps.from_cores(pops[8], 128, 1)
    D = tl.DeviceMps(L, 128, 1)
    tl.lincomb_round([[tl.tnlbm.plain(A), tl.tnlbm.plain(B)]], [D], 128, 1e-7)
    got = D.cores()
    ref = M.lincomb_round([(1.0, pops[7]), (1.0, pops[8])], 128, 1e-7)
    exact_err, gpu_err = [], []
    for x, y, z in _sample_cells(n, 100, 4):
        bits = q.site_bits(n, (x, y, z))
        exact = M.entry(pops[7], bits) + M.entry(pops[8], bits)
        exact_err.append(abs(M.entry(ref, bits) - exact))
        gpu_err.append(abs(M.entry(got, bits) - exact))
    assert max(gpu_err) <= 2 * max(exact_err) + 1e-5 * 2 * lattice.D3Q19.w[7]
    sim.close()
