"""Tensor-core contractions (precision TNLBM_TF32: FP32 storage, the fit's
GEMM stages as tcgen05.mma kind::tf32 with FP32 accumulation in tensor
memory; TNLBM_BF16: the same stages as kind::f16 with BF16 operands, with the
mixed mode's FP64 centre SVDs).  TF32 keeps 10 mantissa bits, so each
contraction carries a relative error of ~1e-3 of its terms; the gates are the
1e-3 level of the reduced-precision path: the fit against the exact product
when the candidate bond suffices and against the FP32 fit, and the step
against the FP64 dense oracle (and that no tile timed out).  BF16 keeps 8
bits: the fit itself is gated at 2e-2, the step at 1e-3."""
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


def _fit(tl, B, C, capA, prec):
    T = tl.tnlbm
    L = len(B)
    capB = max(x.shape[2] for x in B)
    capC = max(x.shape[2] for x in C)
    dB = tl.DeviceMps.from_cores(B, max(capB, 1), 1)
    dC = tl.DeviceMps.from_cores(C, max(capC, 1), 1)
    A = tl.DeviceMps(L, capA, prec)
    T.hadamard_fit([dB], [dC], [A], sweeps=2)
    return A.cores()


def test_tf32_fit_exact_bond_and_close_to_fp32(tl):
    """Candidate bond 24 holds the product (B of bond 24 times a rank-2 C) on
    12 sites: several 64-wide tiles per stage and split-K in S3 / T3."""
    L = 12
    B = synth.random_mps(L, synth.feasible_ranks(L, 24), 11)
    C = M.rank1([np.random.default_rng(k).uniform(0.5, 1.5, 2) for k in range(L)])
    C = M.round_mps(M.add(C, M.scale(C, 0.5)), 4, 0.0)
    exact = M.to_tensor(B) * M.to_tensor(C)
    a32 = _fit(tl, B, C, 24, 1)
    a_tc = _fit(tl, B, C, 24, 2)
    assert rel(M.to_tensor(a32), exact) < 5e-5
    assert rel(M.to_tensor(a_tc), exact) < 3e-3
    assert rel(M.to_tensor(a_tc), M.to_tensor(a32)) < 3e-3


def test_tf32_fit_truncated_tracks_fp32(tl):
    n = 5
    B = M.tt_svd(q.encode(smooth(n, 1, n_modes=12)), 32, 0.0)
    C = M.tt_svd(q.encode(smooth(n, 2, n_modes=12)), 32, 0.0)
    exact = M.to_tensor(B) * M.to_tensor(C)
    a32 = _fit(tl, B, C, 32, 1)
    a_tc = _fit(tl, B, C, 32, 2)
    e32, etc = rel(M.to_tensor(a32), exact), rel(M.to_tensor(a_tc), exact)
    assert etc <= e32 + 3e-3


def test_tf32_step_vs_fp64_dense(tl):
    """The channel with a perturbed start, fit products on the tensor cores:
    within 1e-3 of the FP64 dense Taylor step, mass held to 1e-6, device
    status clean (no timed-out tile)."""
    modes = synth.fourier_modes(3, 7, kmax=2, amp_rho=1e-3, amp_u=1e-2)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0.0, 0.0), chi_max=16, eps=1e-9)
    sim = tl.Sim(3, precision=2, hadamard=0, modes=modes, conserve_mass=True, **kw)
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
    assert abs(rho.sum() - rho_start.sum()) / rho_start.sum() <= 1e-6
    assert sim.stats()["status"] == 0
    sim.close()


def test_tf32_fit_with_split_k_tracks_fp32(tl):
    """Bonds 32 x 16 (K = g b = 512 in the S3 / T3 stages: split-K partial
    tiles written by the tensor-core kernel and summed in order): the TF32
    fit stays within 3e-3 of the FP32 fit."""
    n = 5
    B = M.tt_svd(q.encode(smooth(n, 5, n_modes=16)), 32, 0.0)
    C = M.tt_svd(q.encode(smooth(n, 6, n_modes=6)), 16, 0.0)
    a32 = _fit(tl, B, C, 32, 1)
    a_tc = _fit(tl, B, C, 32, 2)
    assert max(x.shape[2] for x in B) == 32 and max(x.shape[2] for x in C) >= 16
    assert rel(M.to_tensor(a_tc), M.to_tensor(a32)) < 3e-3


# ---------------------------------------------------------------- BF16 operands (TNLBM_BF16)
# BF16 keeps 8 mantissa bits (relative rounding 2^-9 ~ 2e-3 per operand); the
# products are summed in FP32 in tensor memory, so a contraction carries a
# relative error of a few 1e-3 of its terms.

def test_bf16_fit_exact_bond_and_close_to_fp32(tl):
    """As the TF32 case: candidate bond 24 holds the product on 12 sites."""
    L = 12
    B = synth.random_mps(L, synth.feasible_ranks(L, 24), 11)
    C = M.rank1([np.random.default_rng(k).uniform(0.5, 1.5, 2) for k in range(L)])
    C = M.round_mps(M.add(C, M.scale(C, 0.5)), 4, 0.0)
    exact = M.to_tensor(B) * M.to_tensor(C)
    a32 = _fit(tl, B, C, 24, 1)
    abf = _fit(tl, B, C, 24, 4)
    e_ex, e_32 = rel(M.to_tensor(abf), exact), rel(M.to_tensor(abf), M.to_tensor(a32))
    print("bf16 fit, exact bond: vs exact %.3e, vs fp32 fit %.3e" % (e_ex, e_32))
    assert e_ex < 2e-2 and e_32 < 2e-2                   # measured 1.3e-2


def test_bf16_fit_with_split_k_tracks_fp32(tl):
    n = 5
    B = M.tt_svd(q.encode(smooth(n, 5, n_modes=16)), 32, 0.0)
    C = M.tt_svd(q.encode(smooth(n, 6, n_modes=6)), 16, 0.0)
    a32 = _fit(tl, B, C, 32, 1)
    abf = _fit(tl, B, C, 32, 4)
    e = rel(M.to_tensor(abf), M.to_tensor(a32))
    print("bf16 fit, split-K: vs fp32 fit %.3e" % e)
    assert e < 2e-2                                       # measured 1.1e-2


def test_bf16_step_vs_fp64_dense(tl):
    """The TF32 step case with TNLBM_BF16 (BF16 fit contractions, FP64 centre
    SVDs): against the FP64 dense Taylor step after 3 steps, mass held, device
    status clean."""
    modes = synth.fourier_modes(3, 7, kmax=2, amp_rho=1e-3, amp_u=1e-2)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0.0, 0.0), chi_max=16, eps=1e-9)
    sim = tl.Sim(3, precision=4, hadamard=0, modes=modes, conserve_mass=True, **kw)
    rho_start, _ = sim.macroscopic()
    lat = lattice.D3Q19
    cfg = ml.Config(3, lat, 0.8, force=kw["force"], periodic=kw["periodic"], chi_max=16, eps=1e-9, hadamard="exact")
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
    for _ in range(3):
        fd = ld.step(fd, lat, 0.8, kw["force"], None, kw["periodic"], "taylor")
    sim.step(3)
    rho, u = sim.macroscopic()
    _, ud = ld.velocity_out(lat, fd, kw["force"])
    err = rel_l2(u, ud)
    print("bf16 step vs fp64 dense: rel-L2(u) = %.3e" % err)
    assert err <= 1e-3                                    # measured 6.0e-4
    assert abs(rho.sum() - rho_start.sum()) / rho_start.sum() <= 1e-6
    assert sim.stats()["status"] == 0
    sim.close()
