"""GPU parity of the whole MPS-LBM step (tnlbm_create / step / macroscopic)
against the oracle, on contracted fields."""
import numpy as np
import pytest

import synth
from oracle import lattice, lbm_dense as ld, mps as M, mps_lbm as ml, quantics as q
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


def test_channel_32cubed_config_vs_oracle_mps(tl):
    """The 32^3 channel as configured: D3Q19, tau = 0.8, z walls with
    bounce-back, x/y periodic, force 1e-6 along x, rest start, chi = 16,
    eps = 1e-10, 20 steps, FP64, products formed exactly and rounded.
    Same algorithm and truncation as the oracle MPS step.  |u| ~ 1e-5 here, so
    FP64 round-off amplified by ||f|| / ||rho u|| over ~4000 roundings sets a
    floor of ~4e-10 on rel-L2(u) between any two FP64 implementations (the
    oracle itself differs from the dense LBM by 5e-10 at eps = 0): gate 1e-9."""
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-6, 0.0, 0.0), chi_max=16, eps=1e-10)
    sim = tl.Sim(5, precision=0, hadamard=1, **kw)
    cfg = ml.Config(5, lattice.D3Q19, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=16,
                    eps=1e-10, hadamard="exact")
    f = ml.initial_rest(cfg)
    for _ in range(20):
        f = ml.step(cfg, f)
    sim.step(20)
    rho, u = sim.macroscopic()
    rho_o, uo = ml.macroscopic(cfg, f)
    assert rel_l2(u, uo) <= 1e-9
    mass0 = 32.0 ** 3
    assert abs(rho.sum() - mass0) / mass0 <= 1e-6
    st = sim.stats()
    assert st["max_bond"] <= 16 and st["status"] == 0
    sim.close()


def test_channel_untruncated_vs_dense(tl):
    """Nothing truncated (eps = 0; the flow depends on z only, so chi = 16 is
    above every rank that carries information): the MPS step equals the
    dense Taylor-mode LBM.  The force is raised to 1e-4 so that |u| ~ 1e-3 and
    round-off amplified by 1/|u| stays below the 1e-10 gate."""
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-4, 0.0, 0.0), chi_max=16, eps=0.0)
    sim = tl.Sim(4, precision=0, hadamard=1, **kw)
    lat = lattice.D3Q19
    f = ld.initial_rest(lat, 16)
    for _ in range(10):
        f = ld.step(f, lat, 0.8, kw["force"], None, kw["periodic"], "taylor")
    sim.step(10)
    rho, u = sim.macroscopic()
    _, ud = ld.velocity_out(lat, f, kw["force"])
    assert rel_l2(u, ud) <= 1e-10
    assert abs(rho.sum() - 16.0 ** 3) / 16.0 ** 3 <= 1e-12
    sim.close()


def test_box_obstacle_walls_exact_vs_dense(tl):
    """8^3, box obstacle given as the oracle's mask MPS, z walls, force in x and
    y, smooth perturbed start: exact products == dense Taylor-mode LBM."""
    n = 3
    box = synth.box_obstacle(n, (2, 3, 1), (5, 6, 4)).astype(float)
    mask = M.tt_svd(q.encode(box), 64, 1e-14)
    modes = synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-4, 2e-5, 0.0), chi_max=64, eps=1e-13)
    for latname, Q in (("D3Q19", 19), ("D3Q15", 15)):
        sim = tl.Sim(n, lattice=Q, precision=0, hadamard=1, mask_cores=mask, modes=modes, **kw)
        lat = lattice.get(latname)
        cfg = ml.Config(n, lat, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=64, eps=1e-13,
                        hadamard="exact", mask=mask)
        fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
        for _ in range(2):
            fd = ld.step(fd, lat, 0.8, kw["force"], box, kw["periodic"], "taylor")
        sim.step(2)
        rho, u = sim.macroscopic()
        _, ud = ld.velocity_out(lat, fd, kw["force"], box)
        assert rel_l2(u, ud) <= 1e-10, latname
        sim.close()


def test_fit_mode_vs_oracle_fit_mode(tl):
    """Variational products (Sec. 2.3) on the 8^3 channel: GPU step == oracle step."""
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-6, 0.0, 0.0), chi_max=16, eps=1e-10)
    sim = tl.Sim(3, precision=0, hadamard=0, **kw)
    cfg = ml.Config(3, lattice.D3Q19, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=16,
                    eps=1e-10, hadamard="fit")
    f = ml.initial_rest(cfg)
    for _ in range(4):
        f = ml.step(cfg, f)
    sim.step(4)
    _, u = sim.macroscopic()
    _, uo = ml.macroscopic(cfg, f)
    assert rel_l2(u, uo) <= 1e-8
    sim.close()


def test_fp32_path_vs_fp64_oracle(tl):
    """FP32 storage and contractions (FP64 tails): within 1e-3 of the FP64 oracle
    for lattice velocities of order 1e-2 (FP32 storage of f ~ w_i limits the
    relative accuracy of u to ~6e-8 ||f|| / ||rho u||); with the mass
    correction on, the total mass holds to 1e-6."""
    modes = synth.fourier_modes(3, 7, kmax=2, amp_rho=1e-3, amp_u=1e-2)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0.0, 0.0), chi_max=16, eps=1e-9)
    sim = tl.Sim(3, precision=1, hadamard=1, modes=modes, conserve_mass=True, **kw)
    rho_start, _ = sim.macroscopic()
    lat = lattice.D3Q19
    cfg = ml.Config(3, lat, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=16, eps=1e-9, hadamard="exact")
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
    for _ in range(3):
        fd = ld.step(fd, lat, 0.8, kw["force"], None, kw["periodic"], "taylor")
    sim.step(3)
    rho, u = sim.macroscopic()
    _, ud = ld.velocity_out(lat, fd, kw["force"])
    assert rel_l2(u, ud) <= 1e-3
    assert abs(rho.sum() - rho_start.sum()) / rho_start.sum() <= 1e-6     # drift of its own mass
    sim.close()


def test_sphere_mask_built_on_gpu(tl):
    """Solid voxels compressed on the GPU (TT-SVD); exact at chi_mask = 16 on 8^3."""
    n = 3
    sp = synth.sphere_pack(n, 1.8, 0.25, 3)
    kw = dict(tau=0.8, periodic=(1, 1, 1), force=(1e-5, 0.0, 0.0), chi_max=16, eps=1e-12)
    sim = tl.Sim(n, precision=0, hadamard=1, solid=sp, chi_mask=16, eps_mask=1e-12, **kw)
    lat = lattice.D3Q19
    fd = ld.initial_rest(lat, 8, sp.astype(float))
    for _ in range(2):
        fd = ld.step(fd, lat, 0.8, kw["force"], sp.astype(float), kw["periodic"], "taylor")
    sim.step(2)
    rho, u = sim.macroscopic()
    _, ud = ld.velocity_out(lat, fd, kw["force"], sp.astype(float))
    assert rel_l2(u, ud) <= 1e-6
    sim.close()


def test_checkpoint_resume_bitwise(tl):
    modes = synth.fourier_modes(2, 9, kmax=2, amp_rho=1e-3, amp_u=1e-3)
    kw = dict(tau=0.7, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=8, eps=1e-10, modes=modes)
    a = tl.Sim(3, **kw)
    a.step(4)
    ra, ua = a.macroscopic()
    b = tl.Sim(3, **kw)
    b.step(2)
    pops = b.get_populations()
    c = tl.Sim(3, **kw)
    c.set_populations(pops)
    c.step(2)
    rc, uc = c.macroscopic()
    assert np.array_equal(ra, rc) and np.array_equal(ua, uc)
    for s in (a, b, c):
        s.close()


def test_porous_128cubed_bench_configuration_properties(tl):
    """The benchmark workload at full size (128^3 sphere pack at 35 % solid,
    radius 10, chi = 64, FP32, rank-saturated smooth start, mass correction on),
    in the launch configuration the benchmark times: two steps keep mass to
    1e-6, stay finite, keep every bond
    within chi, report no device error, and lower the mean population held in
    solid cells."""
    sp = synth.sphere_pack(7, 10.0, 0.35, 0)
    modes = synth.fourier_modes(31, 0, kmax=4, amp_rho=1e-3, amp_u=1e-3)
    sim = tl.Sim(7, tau=0.7, periodic=(1, 1, 1), solid=sp, chi_mask=64, eps_mask=1e-8,
                 force=(1e-5, 0, 0), chi_max=64, eps=1e-7, precision=1, hadamard=0, modes=modes,
                 conserve_mass=True)
    rho0, _ = sim.macroscopic()
    sim.step(2)
    rho, u = sim.macroscopic()
    assert np.isfinite(u).all() and np.isfinite(rho).all()
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() <= 1e-6
    st = sim.stats()
    assert st["max_bond"] <= 64 and st["status"] == 0
    solid = sp.astype(bool)
    assert rho[solid].mean() < rho0[solid].mean()
    sim.close()


def test_macroscopic_slices_equal_planes_of_the_dense_fields(tl):
    """tnlbm_macroscopic_slice contracts one plane with the axis's sites fixed:
    every plane it returns equals that plane of tnlbm_macroscopic (FP32
    storage, FP64 accumulation in both), for all three axes, with a mask."""
    n = 4
    sp = synth.sphere_pack(n, 3.0, 0.3, 5)
    modes = synth.fourier_modes(9, 2, kmax=3, amp_rho=1e-3, amp_u=1e-2)
    sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), solid=sp, chi_mask=16, eps_mask=1e-8, force=(1e-5, 0, 0),
                 chi_max=24, eps=1e-7, precision=1, hadamard=0, modes=modes)
    sim.step(2)
    rho, u = sim.macroscopic()
    for axis, index in [(0, 0), (0, 11), (1, 5), (2, 15), (2, 8)]:
        rs, us = sim.macroscopic_slice(axis, index)
        sel = [slice(None)] * 3
        sel[axis] = index
        np.testing.assert_allclose(rs, rho[tuple(sel)], rtol=0, atol=1e-12)
        for d in range(3):
            np.testing.assert_allclose(us[d], u[d][tuple(sel)], rtol=0, atol=1e-12)
    with pytest.raises(tl.TnlbmError):
        sim.macroscopic_slice(3, 0)
    with pytest.raises(tl.TnlbmError):
        sim.macroscopic_slice(0, 16)
    sim.close()


def test_stats_mass_and_discarded_weight(tl):
    """stats: `mass` is rho_0 N_fluid from the step's rho_0 node (the lattice
    sum of rho); `discarded2` accumulates the squared tails cut by every
    rounding: ~0 without truncation, positive and growing with it."""
    exact = tl.Sim(3, tau=0.8, periodic=(1, 1, 0), force=(1e-4, 0, 0), chi_max=64, eps=1e-14, precision=0,
                   hadamard=1, modes=synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2))
    exact.step(2)
    st = exact.stats()
    rho, _ = exact.macroscopic()
    assert abs(st["mass"] - rho.sum()) <= 1e-9 * rho.sum()
    assert st["discarded2"] <= 1e-20 * rho.sum() ** 2
    exact.close()
    trunc = tl.Sim(4, tau=0.7, periodic=(1, 1, 1), force=(1e-5, 0, 0), chi_max=8, eps=1e-7, precision=1,
                   hadamard=0, modes=synth.fourier_modes(15, 1, kmax=3, amp_rho=1e-3, amp_u=1e-2))
    trunc.step(1)
    d1 = trunc.stats()["discarded2"]
    trunc.step(1)
    d2 = trunc.stats()["discarded2"]
    assert 0 < d1 < d2
    trunc.close()
