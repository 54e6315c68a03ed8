"""GPU velocity inlet / pressure outlet faces against the oracle: the library
step with per-face boundary functions equals the dense step untruncated
(FP64, exact products; mixed faces with shared edges); an inlet velocity
changed between steps follows the same sequence in the dense step; a uniform
stream at the inlet velocity and outlet density stays put; and the FP32
production path of an inlet / outlet channel tracks the dense oracle."""
import numpy as np
import pytest

import synth
from oracle import lattice, lbm_dense as ld, mps_lbm as ml
from oracle.metrics import rel_l2

pytestmark = pytest.mark.gpu

W, V, P = ld.FACE_WALL, ld.FACE_VELOCITY, ld.FACE_PRESSURE


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2512_07615_gb300 as pkg
    return pkg


def dense_faces(spec):
    base = [(W, (0.0, 0.0, 0.0), 1.0)] * 6
    for k, v in spec.items():
        base[k] = v
    return base


def start(n, modes):
    cfg = ml.Config(n, lattice.D3Q19, 0.8, chi_max=64, eps=0.0)
    return ml.to_dense_populations(ml.initial_perturbed(cfg, modes))


def test_faces_equal_dense_untruncated_with_changing_inflow(tl):
    n, tau = 3, 0.8
    spec = {0: (V, (0.03, 0.01, 0.0), 1.0), 1: (P, (0.0, 0.0, 0.0), 1.002)}
    modes = synth.fourier_modes(3, 5, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    sim = tl.Sim(n, tau=tau, periodic=(0, 1, 0), chi_max=64, eps=1e-14, precision=0, hadamard=1, modes=modes,
                 faces=spec)
    fd = start(n, modes)
    inflow = [(0.03, 0.01, 0.0), (0.05, 0.0, 0.0), (0.02, -0.01, 0.0)]
    for ub in inflow:
        sim.set_face_velocity(0, ub)
        spec_t = dict(spec)
        spec_t[0] = (V, ub, 1.0)
        sim.step(1)
        fd = ld.step(fd, lattice.D3Q19, tau, (0.0, 0.0, 0.0), None, (0, 1, 0), "taylor", faces=dense_faces(spec_t))
    rho, u = sim.macroscopic()
    rho_d, u_d = ld.velocity_out(lattice.D3Q19, fd)
    assert rel_l2(u, u_d) <= 1e-10
    assert np.abs(rho - rho_d).max() <= 1e-12
    sim.close()


def test_uniform_stream_stays_put(tl):
    n, U = 4, 0.05
    lat = lattice.D3Q19
    spec = {0: (V, (U, 0.0, 0.0), 1.0), 1: (P, (0.0, 0.0, 0.0), 1.0)}
    sim = tl.Sim(n, tau=0.8, periodic=(0, 1, 1), chi_max=16, eps=1e-12, precision=0, hadamard=0, faces=spec)
    L = 3 * n
    feq = ld.equilibrium(lat, np.ones(1), np.array([[U], [0.0], [0.0]]))[:, 0]
    pops = []
    for i in range(lat.Q):
        cores = [np.ones((1, 2, 1)) for _ in range(L)]
        cores[0] = cores[0] * feq[i]
        pops.append(cores)
    sim.set_populations(pops)
    sim.step(5)
    rho, u = sim.macroscopic()
    assert np.abs(rho - 1.0).max() <= 1e-12
    assert np.abs(u[0] - U).max() <= 1e-12 and np.abs(u[1:]).max() <= 1e-12
    sim.close()


def test_inlet_outlet_fp32_tracks_dense(tl):
    """32^3 channel along x: inlet 0.04 at x = 0, outlet density 1 at x = N-1,
    walls at z (periodic y); FP32, variational products, chi 32, eps 1e-7,
    10 steps, against the dense oracle."""
    n, tau = 5, 0.8
    spec = {0: (V, (0.04, 0.0, 0.0), 1.0), 1: (P, (0.0, 0.0, 0.0), 1.0)}
    sim = tl.Sim(n, tau=tau, periodic=(0, 1, 0), chi_max=32, eps=1e-7, precision=1, hadamard=0, faces=spec)
    sim.step(10)
    rho, u = sim.macroscopic()
    f = ld.initial_rest(lattice.D3Q19, 32)
    for _ in range(10):
        f = ld.step(f, lattice.D3Q19, tau, (0.0, 0.0, 0.0), None, (0, 1, 0), "exact", faces=dense_faces(spec))
    rho_d, u_d = ld.velocity_out(lattice.D3Q19, f)
    assert np.abs(u_d[0]).max() > 0.01                    # the inflow has entered
    assert rel_l2(u, u_d) <= 1e-3
    assert np.abs(rho - rho_d).max() <= 1e-4
    assert sim.stats()["status"] == 0
    sim.close()


def test_step_options_combined_equal_dense(tl):
    """Zip-up products, block-sum moments, inlet / outlet faces with walls,
    an object mask (the oracle's TT-SVD cores) and a body force together,
    FP64, nothing truncated (8^3: chi 48 holds every bond): one step equals
    the dense step."""
    from oracle import mps as M, quantics as q
    n, tau = 3, 0.8
    box = synth.box_obstacle(n, (3, 2, 2), (5, 5, 4)).astype(float)
    mask = M.tt_svd(q.encode(box), 10 ** 6, 1e-14)
    spec = {0: (V, (0.02, 0.0, 0.01), 1.0), 1: (P, (0.0, 0.0, 0.0), 0.999)}
    modes = synth.fourier_modes(3, 9, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    sim = tl.Sim(n, tau=tau, periodic=(0, 1, 0), mask_cores=mask, force=(1e-4, 0.0, 0.0), chi_max=48, eps=1e-14,
                 precision=0, hadamard=2, block_sums=True, modes=modes, faces=spec)
    fd = start(n, modes)
    sim.step(1)
    fd = ld.step(fd, lattice.D3Q19, tau, (1e-4, 0.0, 0.0), box, (0, 1, 0), "taylor", faces=dense_faces(spec))
    rho, u = sim.macroscopic()
    rho_d, u_d = ld.velocity_out(lattice.D3Q19, fd, (1e-4, 0.0, 0.0), box)
    assert rel_l2(u, u_d) <= 1e-10
    assert np.abs(rho - rho_d).max() <= 1e-12
    assert sim.stats()["status"] == 0
    sim.close()
