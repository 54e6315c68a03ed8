"""The zip-up product on the GPU (tnlbm_hadamard_zipup, and the step with
hadamard = TNLBM_HADAMARD_ZIPUP) against the oracle's hadamard_zipup / step
with hadamard='zipup': same algorithm (right-canonical factors, one
left-to-right truncated pass, a rounding), compared on contracted tensors."""
import numpy as np
import pytest

import synth
from oracle import lattice, mps as M, mps_lbm as ml, quantics as q
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


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def smooth(n, seed, n_modes=6, amp=0.1, kmax=3):
    N = 1 << n
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.random.default_rng(seed)
    f = np.ones((N, N, N))
    for _ in range(n_modes):
        k = r.integers(-kmax, kmax + 1, 3)
        f += amp * r.standard_normal() * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / N + r.uniform(0, 6))
    return f


def _run(tl, Bs, Cs, capB, capC, chi, eps, prec, capA=None):
    T = tl.tnlbm
    L = len(Bs[0])
    dB = [tl.DeviceMps.from_cores(B, capB, prec) for B in Bs]
    dC = [tl.DeviceMps.from_cores(C, capC, prec) for C in Cs]
    A = [tl.DeviceMps(L, capA or chi, prec) for _ in Bs]
    T.hadamard_zipup(dB, dC, A, chi, eps)
    return [a.cores() for a in A]


@pytest.mark.parametrize("prec", [0, 1])
def test_zipup_exact_without_truncation(tl, prec):
    """Random factors (bonds 6 and 5, left-canonical and unnormalised as
    given), chi above every product rank: the exact product."""
    L = 9
    B, C = synth.random_mps(L, synth.feasible_ranks(L, 6), 3), synth.random_mps(L, synth.feasible_ranks(L, 5), 4)
    B2, C2 = synth.random_mps(L, synth.feasible_ranks(L, 3), 5), synth.random_mps(L, synth.feasible_ranks(L, 7), 6)
    got = _run(tl, [B, B2], [C, C2], 7, 7, 64, 0.0, prec)
    for g, (x, y) in zip(got, [(B, C), (B2, C2)]):
        assert rel(M.to_tensor(g), M.to_tensor(x) * M.to_tensor(y)) < (1e-11 if prec == 0 else 5e-5)


@pytest.mark.parametrize("chi,eps", [(6, 0.0), (10, 1e-3), (16, 1e-6)])
def test_zipup_truncated_matches_oracle_fp64(tl, chi, eps):
    n = 4
    B = M.tt_svd(q.encode(smooth(n, 1)), 12, 0.0)
    C = M.tt_svd(q.encode(smooth(n, 2)), 12, 0.0)
    ref = M.hadamard_zipup(B, C, chi, eps)
    got = _run(tl, [B], [C], 12, 12, chi, eps, 0)[0]
    assert M.ranks(got) == M.ranks(ref)
    assert rel(M.to_tensor(got), M.to_tensor(ref)) < 1e-9


def test_zipup_fp32_tracks_oracle(tl):
    n = 4
    B = M.tt_svd(q.encode(smooth(n, 7)), 16, 0.0)
    C = M.tt_svd(q.encode(smooth(n, 8)), 16, 0.0)
    exact = M.to_tensor(B) * M.to_tensor(C)
    ref = M.hadamard_zipup(B, C, 8, 0.0)
    got = _run(tl, [B], [C], 16, 16, 8, 0.0, 1)[0]
    e_ref, e_got = rel(M.to_tensor(ref), exact), rel(M.to_tensor(got), exact)
    assert abs(e_got - e_ref) <= 1e-4 + 0.05 * e_ref
    assert rel(M.to_tensor(got), M.to_tensor(ref)) <= 2 * e_ref + 1e-4


def test_zipup_edge_cases(tl):
    T = tl.tnlbm
    B = synth.random_mps(3, synth.feasible_ranks(3, 2), 1)
    C = synth.random_mps(3, synth.feasible_ranks(3, 2), 2)
    got = _run(tl, [B], [C], 2, 2, 8, 0.0, 0)[0]          # n_bits = 1
    assert rel(M.to_tensor(got), M.to_tensor(B) * M.to_tensor(C)) < 1e-12
    dB = tl.DeviceMps.from_cores(B, 2, 0)
    with pytest.raises(tl.TnlbmError):                        # capA < chi_max
        T.hadamard_zipup([dB], [dB], [tl.DeviceMps(3, 4, 0)], 8, 0.0)


def test_zipup_step_matches_oracle(tl):
    """The step with zip-up products (FP64) against the oracle step with
    hadamard='zipup', same chi and eps, three steps of a perturbed channel."""
    n, tau = 3, 0.8
    modes = synth.fourier_modes(3, 8, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    kw = dict(tau=tau, periodic=(1, 1, 0), force=(1e-4, 0.0, 0.0), chi_max=12, eps=1e-10)
    sim = tl.Sim(n, precision=0, hadamard=2, modes=modes, **kw)
    cfg = ml.Config(n, lattice.D3Q19, tau, force=kw["force"], periodic=kw["periodic"], chi_max=12, eps=1e-10,
                    hadamard="zipup")
    f = ml.initial_perturbed(cfg, modes)
    for _ in range(3):
        f = ml.step(cfg, f)
    sim.step(3)
    rho, u = sim.macroscopic()
    rho_o, u_o = ml.macroscopic(cfg, f)
    assert rel_l2(u, u_o) <= 1e-8
    assert np.abs(rho - rho_o).max() <= 1e-10
    assert sim.stats()["status"] == 0
    sim.close()
