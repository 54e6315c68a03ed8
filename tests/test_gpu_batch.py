"""Batched simulations (tnlbm_batch_*): several independent simulations of
the same lattice size stepped in one graph, each job of a level carrying its
own simulation's data.  The per-job arithmetic is that of the simulations
stepped alone, so the results must be bitwise equal."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tl():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_07615_gb300 import tnlbm as T
    return T


def configs():
    n = 4
    return [
        dict(n_per_axis=n, tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=16, eps=1e-7,
             precision=1, hadamard=0, modes=synth.fourier_modes(5, 1, kmax=2, amp_rho=1e-3, amp_u=1e-2),
             conserve_mass=True),
        dict(n_per_axis=n, tau=0.7, periodic=(1, 1, 1), solid=synth.sphere_pack(n, 2.0, 0.25, 2), chi_mask=16,
             eps_mask=1e-8, force=(1e-5, 0, 0), chi_max=24, eps=1e-7, precision=1, hadamard=0,
             modes=synth.fourier_modes(7, 3, kmax=2, amp_rho=1e-3, amp_u=1e-3), conserve_mass=True),
        dict(n_per_axis=n, lattice=15, tau=0.9, periodic=(1, 0, 1), force=(0, 0, 2e-5), chi_max=8, eps=1e-6,
             precision=1, hadamard=0, modes=synth.fourier_modes(3, 4, kmax=1, amp_rho=1e-3, amp_u=1e-2)),
    ]


def test_batch_equals_simulations_alone(tl):
    cfgs = configs()
    b = tl.Batch(cfgs)
    info = b.info()
    assert info["sims"] == 3 and info["launches_per_step"] > 0
    b.step(3)
    got = [s.macroscopic() for s in b.sims]
    stats = [s.stats() for s in b.sims]
    for i, kw in enumerate(cfgs):
        kw = dict(kw)
        n = kw.pop("n_per_axis")
        alone = tl.Sim(n, **kw)
        alone.step(3)
        rho, u = alone.macroscopic()
        st = alone.stats()
        alone.close()
        assert np.array_equal(rho, got[i][0]) and np.array_equal(u, got[i][1]), i
        assert st["max_bond"] == stats[i]["max_bond"]
    b.close()


def test_batch_timed_steps_and_borrowed_handles(tl):
    b = tl.Batch(configs()[:2])
    ms = b.step_timed(2)
    assert ms > 0
    st = b.sims[1].stats()
    assert st["status"] == 0 and st["steps"] == 2
    b.sims[0].step(1)                 # a borrowed simulation may also step alone
    b.close()


def test_batch_of_uneven_sizes_equals_simulations_alone(tl):
    """Simulations of 8^3, 16^3 and 32^3 with different chi in one graph: the
    rounding launches mix jobs of different chain lengths, the fits of each
    length run on their own stream."""
    cfgs = [
        dict(n_per_axis=3, tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=8, eps=1e-7,
             precision=1, hadamard=0, modes=synth.fourier_modes(2, 1, kmax=1, amp_rho=1e-3, amp_u=1e-2)),
        dict(n_per_axis=5, tau=0.7, periodic=(1, 1, 1), solid=synth.sphere_pack(5, 4.0, 0.25, 1), chi_mask=16,
             eps_mask=1e-8, force=(1e-5, 0, 0), chi_max=32, eps=1e-7, precision=1, hadamard=0, conserve_mass=True),
        configs()[0],
        dict(n_per_axis=5, tau=0.9, periodic=(1, 1, 1), solid=synth.vessel_tree(5, 3.0, 2, 3), chi_mask=16,
             eps_mask=1e-8, force=(1e-5, 0, 0), chi_max=16, eps=1e-7, precision=1, hadamard=0),
    ]
    b = tl.Batch(cfgs)
    b.step(3)
    got = [s.macroscopic() for s in b.sims]
    for i, kw in enumerate(cfgs):
        kw = dict(kw)
        n = kw.pop("n_per_axis")
        alone = tl.Sim(n, **kw)
        alone.step(3)
        rho, u = alone.macroscopic()
        alone.close()
        assert np.array_equal(rho, got[i][0]) and np.array_equal(u, got[i][1]), i
        assert b.sims[i].stats()["status"] == 0
    b.close()


def test_batch_rejects_mixed_precision(tl):
    cfgs = configs()[:2]
    cfgs[1] = dict(cfgs[1], precision=0)
    with pytest.raises(tl.nat.TnlbmError):
        tl.Batch(cfgs)


@pytest.mark.parametrize("precision,hadamard", [(1, 2), (2, 0)])
def test_batch_with_zipup_or_tensor_core_products_equals_alone(tl, precision, hadamard):
    """Batches whose products are zip-up passes (their own stream per chain
    length) or tensor-core fits (TF32): bitwise the simulations alone, for
    two lattice sizes."""
    cfgs = [
        dict(n_per_axis=3, tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=8, eps=1e-7,
             precision=precision, hadamard=hadamard,
             modes=synth.fourier_modes(2, 1, kmax=1, amp_rho=1e-3, amp_u=1e-2)),
        dict(n_per_axis=4, tau=0.7, periodic=(1, 1, 1), solid=synth.sphere_pack(4, 2.0, 0.25, 2), chi_mask=16,
             eps_mask=1e-8, force=(1e-5, 0, 0), chi_max=16, eps=1e-7, precision=precision, hadamard=hadamard,
             modes=synth.fourier_modes(7, 3, kmax=2, amp_rho=1e-3, amp_u=1e-3)),
    ]
    b = tl.Batch(cfgs)
    b.step(2)
    got = [s.macroscopic() for s in b.sims]
    for i, kw in enumerate(cfgs):
        kw = dict(kw)
        n = kw.pop("n_per_axis")
        alone = tl.Sim(n, **kw)
        alone.step(2)
        rho, u = alone.macroscopic()
        alone.close()
        assert np.array_equal(rho, got[i][0]) and np.array_equal(u, got[i][1]), i
        assert b.sims[i].stats()["status"] == 0
    b.close()
