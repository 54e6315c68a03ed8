"""GPU builder of masks combined on separate length scales (App. D) against
the oracle's definition: a sphere cell repeated over a seeded arrangement,
128^3 cells built from a 8^3 and a 16^3 grid; the bonds stay at the larger
of the two parts; the mask drives a simulation step."""
import numpy as np
import pytest

import synth
from oracle import masks, mps as M, quantics as q

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


@pytest.mark.parametrize("prec", [0, 1])
def test_mask_product_matches_definition(tl, prec):
    import torch
    dt = torch.float64 if prec == 0 else torch.float32
    outer = synth.cell_pattern(3, 0.4, 7).astype(np.float64)
    inner = synth.sphere_cell(4, 5.5).astype(np.float64)
    X = tl.mask_product(torch.tensor(outer, dtype=dt, device="cuda"), torch.tensor(inner, dtype=dt, device="cuda"),
                        64, 64, 1e-12)
    got = tl.to_dense(X).cpu().numpy()
    ref = masks.combined_dense(outer, inner)
    assert got.shape == (128, 128, 128)
    assert np.abs(got - ref).max() <= (1e-6 if prec == 0 else 1e-4)
    r = X.bonds()
    ro = M.ranks(M.tt_svd(q.encode(outer), 64, 1e-12))
    ri = M.ranks(M.tt_svd(q.encode(inner), 64, 1e-12))
    assert max(r) <= max(max(ro), max(ri)) and r[9] == 1
    # the same as the oracle's concatenation of its own TT-SVDs, cell by cell
    oc = masks.mask_product(M.tt_svd(q.encode(outer), 64, 1e-12), M.tt_svd(q.encode(inner), 64, 1e-12))
    np.testing.assert_allclose(got, q.decode(M.to_tensor(oc)), atol=1e-6 if prec == 0 else 1e-4)


def test_mask_product_drives_a_simulation(tl):
    import torch
    outer = synth.cell_pattern(2, 0.5, 9).astype(np.float32)
    inner = synth.sphere_cell(4, 5.0).astype(np.float32)
    X = tl.mask_product(torch.tensor(outer, device="cuda"), torch.tensor(inner, device="cuda"), 32, 32, 1e-7)
    sim = tl.Sim(6, tau=0.7, periodic=(1, 1, 1), mask_cores=X.cores(), force=(1e-5, 0, 0), chi_max=32,
                 eps=1e-7, precision=1, hadamard=0, conserve_mass=True)
    rho0, _ = sim.macroscopic()
    sim.step(2)
    rho, u = sim.macroscopic()
    assert np.isfinite(u).all()
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() <= 1e-6
    assert sim.stats()["status"] == 0
    sim.close()
