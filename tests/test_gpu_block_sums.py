"""Block-sum moments on the GPU (tnlbm_config.block_sums: rho and rho u as
one rounding of the block sum of all Q populations, Eq. add) against the
oracle's block-sum mode: same algorithm and truncation, FP64 exact products.
Untruncated (chi 16 holds every bond of an 8^3 lattice), the block fold and
the pairwise tree give the same moments; the block fold runs fewer dependent
levels, so one step launches fewer kernels."""
import numpy as np
import pytest

import synth
from oracle import lattice, mps_lbm as ml
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


def _run(tl, n, steps, chi, eps, block):
    modes = synth.fourier_modes(3, 8, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-4, 0.0, 0.0), chi_max=chi, eps=eps)
    sim = tl.Sim(n, precision=0, hadamard=1, modes=modes, block_sums=block, **kw)
    cfg = ml.Config(n, lattice.D3Q19, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=chi, eps=eps,
                    hadamard="exact", block_sums=block)
    f = ml.initial_perturbed(cfg, modes)
    for _ in range(steps):
        f = ml.step(cfg, f)
    sim.step(steps)
    rho, u = sim.macroscopic()
    st = sim.stats()
    sim.close()
    return (rho, u), ml.macroscopic(cfg, f), st


def test_block_sum_step_matches_oracle_block_mode(tl):
    (rho, u), (rho_o, u_o), st = _run(tl, 4, 4, 16, 1e-10, True)
    assert rel_l2(u, u_o) <= 1e-9
    assert np.abs(rho - rho_o).max() <= 1e-11
    assert st["status"] == 0 and st["max_bond"] <= 16


def test_block_and_pairwise_folds_agree_untruncated(tl):
    (rb, ub), _, sb = _run(tl, 3, 3, 16, 1e-14, True)
    (rp, up), _, sp = _run(tl, 3, 3, 16, 1e-14, False)
    assert rel_l2(ub, up) <= 1e-10
    assert np.abs(rb - rp).max() <= 1e-12
    assert sb["gpu_launches_per_step"] < sp["gpu_launches_per_step"]


def test_block_sums_reject_wide_bonds(tl):
    with pytest.raises(tl.TnlbmError):
        tl.Sim(3, chi_max=64, block_sums=True)
