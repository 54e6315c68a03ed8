"""GPU parity of the mixed precision mode (TNLBM_MIXED: FP32 cores,
contractions and QR sweeps; FP64 one-sided Jacobi for every centre SVD of
Eq. svd-move, shared by a thread-block cluster) against the FP64 oracle, and
of the cluster Jacobi against the single-CTA one.

Tolerances.  FP32 storage rounds every core to 2^-24 relative; a step forms
~10^3 rounded sums whose cores are contracted into u, and |u| ~ 1e-2 ... 1e-3
of ||f|| here, so FP32 storage alone limits rel-L2(u) to ~1e-4 -- the gate
of the mixed path is 1e-3, as for the other reduced-precision paths.  The
FP64 path runs the same algorithm as the oracle and is gated at 1e-8 (the
equal-chi gate with truncation).  Comparisons are on contracted fields."""
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
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


# ---------------------------------------------------------------- the rounding primitive
@pytest.mark.parametrize("L,chi,eps", [(6, 8, 0.0), (9, 6, 1e-3), (12, 12, 1e-6), (15, 24, 1e-9)])
def test_mixed_rounding_vs_oracle(tl, L, chi, eps):
    """Rounded sums of three random MPS (ragged bonds, truncation by chi and
    by eps) in TNLBM_MIXED equal the oracle's FP64 rounding to FP32 storage
    accuracy (inputs and outputs are rounded to float), and keep its ranks."""
    from paper_2512_07615_gb300 import tnlbm as T
    nat = tl.native
    batches, dsts, refs = [], [], []
    for b in range(3):
        A = synth.random_mps(L, synth.feasible_ranks(L, chi // 2 + b), 40 + b)
        B = synth.random_mps(L, synth.feasible_ranks(L, chi - b), 50 + b)
        C = synth.random_mps(L, synth.feasible_ranks(L, 3), 60 + b)
        # round the inputs to float first: both sides see the same data
        A, B, C = ([c.astype(np.float32).astype(np.float64) for c in X] for X in (A, B, C))
        dA, dB, dC = (T.DeviceMps.from_cores(X, 32, nat.MIXED) for X in (A, B, C))
        batches.append([T.plain(dA, 1.0), T.plain(dB, -0.5), T.plain(dC, 2.0)])
        dsts.append(T.DeviceMps(L, 32, nat.MIXED))
        refs.append(M.lincomb_round([(1.0, A), (-0.5, B), (2.0, C)], chi, eps))
    T.lincomb_round(batches, dsts, chi, eps)
    for d, ref in zip(dsts, refs):
        assert d.bonds() == M.ranks(ref)
        assert rel(M.to_tensor(d.cores()), M.to_tensor(ref)) < 2e-6


# ---------------------------------------------------------------- cluster vs single CTA
@pytest.mark.parametrize("prec,gate", [(0, 1e-10), (3, 1e-4)])
def test_cluster_svd_equals_single_cta(tl, prec, gate):
    """The FP64 centre SVD spread over a thread-block cluster (rows of the
    Jacobi matrices split over the CTAs, inner products summed in rank order)
    and the single-CTA Jacobi differ only by the order of FP64 sums: a 16^3
    sphere-pack step with products formed exactly (Kronecker bonds up to
    24^2), chi 24, eps 1e-8, taken with clusters (max_cluster = 0) and with one
    CTA per job (max_cluster = 1), agrees to round-off in FP64 and to FP32
    storage in the mixed mode."""
    solid = synth.sphere_pack(4, 3.0, 0.3, 1)
    modes = synth.fourier_modes(7, 3, kmax=2, amp_rho=1e-3, amp_u=1e-3)
    kw = dict(tau=0.7, periodic=(1, 1, 1), solid=solid, chi_mask=16, eps_mask=1e-10, force=(1e-5, 0, 0),
              chi_max=24, eps=1e-8, precision=prec, hadamard=1, modes=modes)
    out = []
    for mc in (1, 0):
        sim = tl.Sim(4, max_cluster=mc, **kw)
        sim.step(2)
        out.append(sim.macroscopic())
        assert sim.stats()["status"] == 0
        sim.close()
    err = rel_l2(out[1][1], out[0][1])
    print("cluster vs single CTA prec %d: rel-L2(u) = %.3e" % (prec, err))
    assert err <= gate
    assert np.abs(out[1][0] - out[0][0]).max() <= 1e2 * gate


# ---------------------------------------------------------------- the benchmarked combination
def _porous_case(n, chi, chi_mask, radius, hadamard, eps):
    solid = synth.sphere_pack(n, radius, 0.35, 0).astype(np.float64)
    mask = M.tt_svd(q.encode(solid), chi_mask, 1e-10)
    modes = synth.fourier_modes(31, 0, kmax=4, amp_rho=1e-3, amp_u=1e-3)
    cfg = ml.Config(n, lattice.D3Q19, 0.7, force=(1e-5, 0.0, 0.0), periodic=(1, 1, 1), chi_max=chi, eps=eps,
                    hadamard=hadamard, mask=mask)
    return cfg, mask, modes


@pytest.mark.parametrize("prec,gate", [(0, 1e-8), (3, 1e-3)])
def test_porous_32cubed_exact_products_vs_oracle(tl, prec, gate):
    """The benchmarked combination on a 32^3 sphere pack (radius 2.5, 35 %
    solid, mask MPS of bond 16), D3Q19, tau 0.7, body force, smooth 31-mode
    start, chi 16 (bonds capped), products formed exactly and rounded, 3 steps:
    FP64 within 1e-8 of the oracle, the mixed mode within 1e-3."""
    n, chi = 5, 16
    cfg, mask, modes = _porous_case(n, chi, 16, 2.5, "exact", 1e-7)
    f = ml.initial_perturbed(cfg, modes)
    for _ in range(3):
        f = ml.step(cfg, f)
    _, uo = ml.macroscopic(cfg, f)
    sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), mask_cores=mask, force=(1e-5, 0, 0), chi_max=chi, eps=1e-7,
                 precision=prec, hadamard=1, modes=modes)
    sim.step(3)
    _, u = sim.macroscopic()
    err = rel_l2(u, uo)
    print("porous32 exact prec %d: rel-L2(u) = %.3e" % (prec, err))
    assert err <= gate
    assert sim.stats()["status"] == 0
    sim.close()


@pytest.mark.parametrize("prec,gate", [(0, 1e-8), (3, 1e-3), (1, 1e-3)])
def test_porous_16cubed_fit_products_eps_limited_vs_oracle(tl, prec, gate):
    """Variational products (Sec. 2.3) in an eps-limited regime: 16^3 sphere
    pack, chi 64 (no bond of L = 12 sites can exceed 64, so eps = 1e-6 alone
    sets the ranks), mask of full bond, 2 steps.  Here the oracle's step moves
    by 3.5e-12 under 1e-13 perturbations of its start (measured), so the fit is
    well conditioned and the FP64 gate of 1e-8 applies; FP32 and mixed 1e-3
    (measured 6.5e-5 and 9e-6; FP32 Householder column norms are summed in
    FP64, so small directions of the centre are kept, as FP64 keeps them)."""
    n, chi = 4, 64
    cfg, mask, modes = _porous_case(n, chi, 64, 3.75, "fit", 1e-6)
    f = ml.initial_perturbed(cfg, modes)
    for _ in range(2):
        f = ml.step(cfg, f)
    _, uo = ml.macroscopic(cfg, f)
    sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), mask_cores=mask, force=(1e-5, 0, 0), chi_max=chi, eps=1e-6,
                 precision=prec, hadamard=0, modes=modes)
    sim.step(2)
    _, u = sim.macroscopic()
    err = rel_l2(u, uo)
    print("porous16 fit prec %d: rel-L2(u) = %.3e" % (prec, err))
    assert err <= gate
    sim.close()


# ---------------------------------------------------------------- weakly damped flow
def test_mixed_tgv_near_half_tau_tracks_dense_energy(tl):
    """Taylor-Green vortex at tau = 0.5038 (omega ~ 1.985), 16^3, chi 32,
    eps 1e-7, fit products, 100 steps: the mixed mode keeps the dense FP64
    oracle's kinetic-energy history (E/E0 at every 25 steps within 2e-4),
    where the FP32 Jacobi of TNLBM_FP32 drifts by ~2e-3 after 30 steps."""
    n, tau, u0, steps = 4, 0.5038, 0.05, 100
    modes = synth.taylor_green_modes(u0)
    sim = tl.Sim(n, tau=tau, periodic=(1, 1, 1), chi_max=32, eps=1e-7, precision=3, hadamard=0, modes=modes)
    lat = lattice.D3Q19
    cfg = ml.Config(n, lat, tau, chi_max=64, eps=0.0)
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
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
    dev = max(abs(a / e_mps[0] - b / e_dense[0]) for a, b in zip(e_mps, e_dense))
    print("tgv16 mixed near tau 1/2: max |E/E0 - dense| = %.3e" % dev)
    assert dev <= 2e-4
    sim.close()


def test_learned_rank_from_config(tl):
    """learned_rank = 3 in the config switches on the randomized truncation at
    the previous step's rank from the first step (test matrix from `seed`):
    certified steps are taken, and in FP64 with eps = 1e-8 the flow stays
    within 1e-5 of the full-SVD run (each accepted truncation is certified to
    within 1 / (1 - eta) of the optimal error at that bond)."""
    modes = synth.fourier_modes(7, 3, kmax=2, amp_rho=1e-3, amp_u=1e-3)
    kw = dict(tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=32, eps=1e-8, precision=0, hadamard=1,
              modes=modes)
    a = tl.Sim(4, learned_rank=3, seed=11, **kw)
    b = tl.Sim(4, **kw)
    a.step(4)
    b.step(4)
    cnt = a.learn_counters()
    _, ua = a.macroscopic()
    _, ub = b.macroscopic()
    assert cnt[0] + cnt[1] > 0
    print("learned rank 3 vs full SVD: rel-L2(u) = %.3e, accepted %d, fell back %d" % (rel_l2(ua, ub), cnt[0], cnt[1]))
    assert rel_l2(ua, ub) <= 1e-5
    a.close()
    b.close()


# ---------------------------------------------------------------- chi-limited accuracy
def test_reduced_precision_keeps_the_truncation_error_of_fp64(tl):
    """In the chi-limited regime of the benchmark (64^3 sphere pack, radius 5,
    35 % solid, mask MPS of bond 64, chi 64, 31-mode start: every inner bond
    sits at chi), the truncation error against the dense FP64 oracle after
    3 steps is ~0.4 in rel-L2(u) for FP64 itself.  The singular values at the
    cut are then close, so FP32 storage picks another, equally good, rank-64
    subspace than FP64 does (the two fields differ by ~6e-2 while both keep
    the same error): the mixed and FP32 modes must stay within 1 % of FP64's
    error against the dense solution."""
    n, chi, steps = 6, 64, 3
    solid = synth.sphere_pack(n, 5.0, 0.35, 0).astype(np.float64)
    mask = M.tt_svd(q.encode(solid), 64, 1e-8)
    md = q.decode(M.to_tensor(mask))
    modes = synth.fourier_modes(31, 0, kmax=4, amp_rho=1e-3, amp_u=1e-3)
    lat = lattice.D3Q19
    cfg = ml.Config(n, lat, 0.7, force=(1e-5, 0, 0), periodic=(1, 1, 1), chi_max=128, eps=0.0, mask=mask)
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
    for _ in range(steps):
        fd = ld.step(fd, lat, 0.7, (1e-5, 0.0, 0.0), md, (1, 1, 1), "taylor")
    ud = ld.velocity_out(lat, fd, (1e-5, 0.0, 0.0), md)[1]
    err = {}
    for prec in (0, 3, 1):
        sim = tl.Sim(n, tau=0.7, periodic=(1, 1, 1), mask_cores=mask, force=(1e-5, 0, 0), chi_max=chi, eps=1e-7,
                     precision=prec, hadamard=0, modes=modes, conserve_mass=prec != 0)
        sim.step(steps)
        err[prec] = rel_l2(sim.macroscopic()[1], ud)
        assert sim.stats()["status"] == 0
        sim.close()
    print("porous64 chi 64 rel-L2(u) vs dense: fp64 %.4e mixed %.4e fp32 %.4e" % (err[0], err[3], err[1]))
    assert 0.1 < err[0] < 1.0                     # the regime: truncation dominates
    assert err[3] <= 1.01 * err[0]
    assert err[1] <= 1.01 * err[0]


def test_mixed_tgv_64cubed_tau_0_5076_tracks_dense_energy(tl):
    """Sec. 4.1 flow near tau = 1/2 at the benchmark's viscosity: Taylor-Green
    vortex at tau = 0.5076 (u0 = 0.05, 64^3, Re ~ 200), chi 64, eps 1e-7,
    fit products, 100 steps.  The mixed mode keeps the dense FP64 oracle's
    kinetic-energy history (E/E0 every 25 steps) within 1e-3 (measured
    4.9e-5 over 200 steps; FP64 1.2e-6; the FP32 mode drifts by 2.1e-2)."""
    n, tau, u0, steps, every = 6, 0.5076, 0.05, 100, 25
    modes = synth.taylor_green_modes(u0)
    lat = lattice.D3Q19
    cfg = ml.Config(n, lat, tau, chi_max=64, eps=0.0)
    fd = ml.to_dense_populations(ml.initial_perturbed(cfg, modes))
    sim = tl.Sim(n, tau=tau, periodic=(1, 1, 1), chi_max=64, eps=1e-7, precision=3, hadamard=0, modes=modes)
    e_mps, e_dense = [], []
    for t in range(0, steps + 1, every):
        if t:
            sim.step(every)
            for _ in range(every):
                fd = ld.step(fd, lat, tau, (0.0, 0.0, 0.0), None, (1, 1, 1), "taylor")
        rho, u = sim.macroscopic()
        e_mps.append(0.5 * float(np.sum(rho * np.sum(u ** 2, axis=0))))
        rd, ud = ld.velocity_out(lat, fd)
        e_dense.append(0.5 * float(np.sum(rd * np.sum(ud ** 2, axis=0))))
    dev = max(abs(a / e_mps[0] - b / e_dense[0]) for a, b in zip(e_mps, e_dense))
    print("tgv64 mixed tau 0.5076: max |E/E0 - dense| = %.3e (E/E0 dense %.6f after %d steps)"
          % (dev, e_dense[-1] / e_dense[0], steps))
    assert dev <= 1e-3
    assert sim.stats()["status"] == 0
    sim.close()


@pytest.mark.parametrize("prec,gate", [(0, 1e-12), (3, 5e-6)])
def test_rounding_at_chi_256_on_a_full_cluster(tl, prec, gate):
    """The rounding at chi 256 (the branching-vessel configuration's bond):
    the sum of two random MPS of L = 18 sites with bonds up to 128 each gives
    centre matrices of 256 x 512, whose FP64 Jacobi fills the shared memory of
    a 16-CTA cluster (row layout of 172 KB per CTA).  Untruncated (chi 256
    holds every summed bond, eps 0), so the result is the exact sum: FP64
    within 1e-12 of the oracle, the mixed mode within FP32 storage."""
    from paper_2512_07615_gb300 import tnlbm as T
    nat = tl.native
    L, cap = 18, 256
    A = synth.random_mps(L, synth.feasible_ranks(L, 128), 71)
    B = synth.random_mps(L, synth.feasible_ranks(L, 128), 72)
    if prec == 3:
        A, B = ([c.astype(np.float32).astype(np.float64) for c in X] for X in (A, B))
    dA, dB = (T.DeviceMps.from_cores(X, cap, prec) for X in (A, B))
    dst = T.DeviceMps(L, cap, prec)
    T.lincomb_round([[T.plain(dA, 1.0), T.plain(dB, -0.75)]], [dst], cap, 0.0)
    ref = M.lincomb_round([(1.0, A), (-0.75, B)], cap, 0.0)
    assert max(dst.bonds()) == 256
    err = rel(M.to_tensor(dst.cores()), M.to_tensor(ref))
    print("chi 256 rounding prec %d: rel-L2 = %.3e" % (prec, err))
    assert err <= gate
