"""GPU parity of the learned rounding against the oracle: the rank model's
forward pass, loss gradient and Adam step (own kernels) against the FP64
analytic forms; the certified randomized truncation against
oracle.learned.round_mps_learned on the same inputs and the same Gaussian
test matrix; and a simulation that logs its spectra, trains the model on the
GPU and then rounds with predicted ranks, compared with the same simulation
rounded by full SVDs."""
import numpy as np
import pytest

import synth
from oracle import learned as LR, mps as M, quantics as q
from oracle.metrics import rel_l2

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


def half_params(seed):
    """Oracle initial parameters rounded to FP16 (what both sides evaluate)."""
    P = LR.mlp_init(seed)
    return {k: v.astype(np.float16).astype(np.float64) for k, v in P.items()}


def dev(x, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype or torch.float32, device="cuda")


def features(M_, seed):
    """Rank-model inputs shaped like logged spectra: 16 decreasing log10 values
    starting at 0, bond fraction, step fraction."""
    rng = np.random.default_rng(seed)
    X = np.zeros((M_, LR.N_FEAT))
    dec = rng.uniform(0.05, 1.0, (M_, 1))
    X[:, :16] = -np.cumsum(np.concatenate([np.zeros((M_, 1)), rng.exponential(dec, (M_, 15))], axis=1), axis=1)
    X[:, 16] = rng.integers(1, 21, M_) / 21.0
    X[:, 17] = rng.uniform(0, 1, M_)
    return X.astype(np.float32)


@pytest.mark.parametrize("M_", [1, 200, 5000])
def test_mlp_forward_and_gradient_match_oracle(tl, M_):
    """M = 200: seven tiles of 32 with a ragged tail; M = 5000: more tiles than
    CTAs.  FP32 arithmetic against the FP64 analytic gradient."""
    P = half_params(1)
    X = features(M_, 2)
    y = np.random.default_rng(3).uniform(0, 1, M_).astype(np.float32)
    flat = dev(tl.mlp_flatten(P))
    out = tl.mlp_forward(flat, dev(X)).cpu().numpy()
    ref, _ = LR.mlp_forward(P, X.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-5, atol=1e-5 * np.abs(ref).max())
    loss, grad = tl.mlp_loss_grad(flat, dev(X), dev(y))
    lo, go = LR.mlp_loss_grad(P, X.astype(np.float64), y.astype(np.float64))
    assert abs(loss.item() - lo) <= 1e-5 * lo
    g = tl.mlp_unflatten(grad.cpu().numpy())
    for k in go:
        scale = max(np.abs(go[k]).max(), 1e-12)
        assert np.abs(g[k] - go[k]).max() <= 1e-4 * scale, k


def test_mlp_first_adam_step_and_fp16_copy(tl):
    """From zero moments the first Adam step moves each parameter by
    lr * g / (|g| + 1e-8) (bias corrections cancel); the FP16 copy is the
    master rounded to nearest."""
    import torch
    P = half_params(4)
    X = features(300, 5)
    y = np.random.default_rng(6).uniform(0, 1, 300).astype(np.float32)
    tr = tl.MlpTrainer(dev(tl.mlp_flatten(P)))
    lr = 1e-3
    hist = tr.train(dev(X), dev(y), iters=1, batch=300, lr=lr)
    lo, go = LR.mlp_loss_grad(P, X.astype(np.float64), y.astype(np.float64))
    assert abs(hist[0].item() - lo) <= 1e-5 * lo
    g = np.concatenate([go[k].reshape(-1) for k in ("W1", "b1", "W2", "b2", "W3", "b3")])
    w0 = tl.mlp_flatten(P).astype(np.float64)
    expect = w0 - lr * g / (np.abs(g) + 1e-8)
    got = tr.master.cpu().numpy().astype(np.float64)
    big = np.abs(g) > 1e-3 * np.abs(g).max()
    np.testing.assert_allclose(got[big], expect[big], atol=2e-6 * lr + 1e-7)
    half = tr.half.cpu().numpy()
    assert np.array_equal(half.view(np.uint16), tr.master.cpu().numpy().astype(np.float16).view(np.uint16))
    assert torch.isfinite(tr.master).all()


def test_mlp_training_learns_a_rank_rule(tl):
    """Labels = fraction of the 16 logged values above -3 (a rank rule at a
    fixed tolerance): GPU training brings the loss to under a tenth of that of
    predicting the mean, on held-out samples."""
    X = features(8192, 7)
    y = ((X[:, :16] > -3).sum(axis=1) / 16.0).astype(np.float32)
    Xt, yt = X[:6144], y[:6144]
    Xv, yv = X[6144:], y[6144:]
    P = LR.mlp_init(8)
    tr = tl.MlpTrainer(dev(tl.mlp_flatten(P)))
    hist = tr.train(dev(Xt), dev(yt), iters=3000, batch=256, lr=2e-3)
    assert np.isfinite(hist.cpu().numpy()).all()
    pred = tl.mlp_forward(tr.master, dev(Xv)).cpu().numpy()
    mse = np.mean((pred - yv) ** 2)
    assert mse < 0.1 * np.var(yv)


def smooth_field(n, seed, K=24, kmax=7, decay=0.7):
    N = 1 << n
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    r = np.random.default_rng(seed)
    f = np.ones((N, N, N))
    for j in range(K):
        k = r.integers(-kmax, kmax + 1, 3)
        f += decay ** j * np.cos(2 * np.pi * (k[0] * X + k[1] * Y + k[2] * Z) / N + r.uniform(0, 6))
    return f


@pytest.fixture(scope="module")
def smooth_pair():
    n = 5
    A = M.tt_svd(q.encode(smooth_field(n, 1)), 64, 1e-13)
    B = M.tt_svd(q.encode(smooth_field(n, 2)), 64, 1e-13)
    return n, A, B


@pytest.mark.parametrize("prec", [0, 1])
def test_rsvd_rounding_matches_oracle(tl, smooth_pair, prec):
    """Sum of two 32^3 smooth fields (bonds up to 47) rounded to chi = 32,
    eps = 1e-6, with the full rounding's ranks as targets: bonds cut by eps
    and bonds capped by chi both take the randomized path.  FP64: same
    accept / fall-back decisions and the same tensor as the oracle to
    round-off (both fix the sign gauge of every singular pair the same way);
    FP32: within 1e-4."""
    import torch
    n, A, B = smooth_pair
    L = 3 * n
    omega = synth.gaussian_matrix(128, 128, 7)
    ref_full = M.lincomb_round([(1.0, A), (0.5, B)], 32, 1e-6)
    tg = [0] + [M.ranks(ref_full)[k] for k in range(1, L)] + [0]
    S = M.add(A, M.scale(B, 0.5))
    ref, na, nf = LR.round_mps_learned(S, 32, 1e-6, tg, omega)
    assert na >= 4
    dA, dB = tl.DeviceMps.from_cores(A, 64, prec), tl.DeviceMps.from_cores(B, 64, prec)
    D = tl.DeviceMps(L, 32, prec)
    om = torch.tensor(omega, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    acc, fb, full = tl.lincomb_round_rsvd([[tl.plain(dA), tl.plain(dB, 0.5)]], [D], 32, 1e-6, [tg], om)
    got = M.to_tensor(D.cores())
    if prec == 0:
        assert (acc, fb) == (na, nf)
        assert acc + full == L - 1               # every bond: accepted, or a full SVD
        assert rel_l2(got, M.to_tensor(ref)) <= 1e-10
    else:
        # FP32 storage moves the full rounding of this input by 2.8e-5 already
        # (unit round-off over the 2e-2 relative gap at the chi cut)
        assert acc >= na - 2
        assert rel_l2(got, M.to_tensor(ref)) <= 1e-4
    # randomized and full truncation agree to the truncation error itself
    exact = M.to_tensor(A) + 0.5 * M.to_tensor(B)
    assert rel_l2(got, exact) <= 1.2 * rel_l2(M.to_tensor(ref_full), exact) + 1e-6


@pytest.mark.parametrize("prec", [0, 1])
def test_rsvd_low_targets_fall_back_and_redundant_sum_is_exact(tl, prec):
    """Targets of 1 where the rank is ~16 cannot be certified: every
    randomized step falls back and the result is the full rounding.  A + 0.5 A
    at target = rank is exact (1.5 A)."""
    import torch
    L = 12
    A = synth.random_mps(L, synth.feasible_ranks(L, 16), 4)
    omega = synth.gaussian_matrix(128, 128, 8)
    om = torch.tensor(omega, dtype=torch.float64 if prec == 0 else torch.float32, device="cuda")
    dA = tl.DeviceMps.from_cores(A, 16, prec)
    D = tl.DeviceMps(L, 64, prec)
    acc, fb, full = tl.lincomb_round_rsvd([[tl.plain(dA), tl.plain(dA, 0.5)]], [D], 64, 1e-12,
                                          [[0] + [16] * (L - 1) + [0]], om)
    ref, na, nf = LR.round_mps_learned(M.add(A, M.scale(A, 0.5)), 64, 1e-12, [0] + [16] * (L - 1) + [0], omega)
    tol = 1e-11 if prec == 0 else 2e-5
    assert rel_l2(M.to_tensor(D.cores()), 1.5 * M.to_tensor(A)) <= tol
    if prec == 0:
        assert (acc, fb) == (na, nf) and acc >= 3
    # low targets on a wide random MPS (bonds 32, no spectral decay): a sample
    # of 16 cannot meet eps = 1e-12 and chi does not cap, so nothing is certified
    W = M.add(synth.random_mps(L, synth.feasible_ranks(L, 16), 5), synth.random_mps(L, synth.feasible_ranks(L, 16), 6))
    dW1 = tl.DeviceMps.from_cores(W, 32, prec)
    D2 = tl.DeviceMps(L, 64, prec)
    D3 = tl.DeviceMps(L, 64, prec)
    acc, fb, full = tl.lincomb_round_rsvd([[tl.plain(dW1)]], [D2], 64, 1e-12, [[0] + [1] * (L - 1) + [0]], om,
                                          oversample=0, power=0)
    tl.lincomb_round([[tl.plain(dW1)]], [D3], 64, 1e-12)
    assert acc == 0 and fb > 0
    assert rel_l2(M.to_tensor(D2.cores()), M.to_tensor(D3.cores())) <= (1e-12 if prec == 0 else 1e-5)


def channel_sim(tl):
    """32^3 channel (z walls), smooth start with velocity amplitude 1e-2, FP32,
    chi = 64 above every bond it reaches, eps = 1e-5: bonds set by eps."""
    modes = synth.fourier_modes(15, 7, kmax=3, amp_rho=1e-3, amp_u=1e-2)
    return tl.Sim(5, tau=0.8, periodic=(1, 1, 0), force=(1e-5, 0, 0), chi_max=64, eps=1e-5, precision=1,
                  hadamard=0, modes=modes, conserve_mass=True)


def test_sim_learned_rank_gain_over_full_svd(tl):
    """(1) Log spectra for 2 steps; (2) train the rank model on the GPU from the
    log; (3) run 4 more steps with predicted ranks.  Against the same 6 steps
    with full SVDs: velocity within 1e-3, density within 1e-4, mass within
    1e-6.  Gain over the method without the trained model: with the untrained
    network no randomized truncation is certified; with the trained one a
    share of the full SVDs is replaced by certified randomized ones."""
    import time
    omega = synth.gaussian_matrix(128, 128, 21)
    ref = channel_sim(tl)
    ref.step(4)
    t_full = ref.step_timed(2) / 2
    rho_r, u_r = ref.macroscopic()
    ref.close()

    def run(train_iters):
        sim = channel_sim(tl)
        rho0, _ = sim.macroscopic()
        sim.learn_configure(1, omega, dataset_cap=1 << 16)
        sim.step(2)
        X, y, cnt = sim.learn_dataset(1 << 16)
        assert cnt == len(y) and cnt > 1000
        assert np.isfinite(X).all() and (y > 0).all() and (y <= 1).all()
        assert (X[:, 0] == 0).all() and (np.diff(X[:, :16], axis=1) <= 0).all()
        perm = np.random.default_rng(0).permutation(len(y))
        tr = tl.MlpTrainer(dev(tl.mlp_flatten(LR.mlp_init(3))))
        if train_iters:
            tr.train(dev(X[perm]), dev(y[perm]), iters=train_iters, batch=256, lr=2e-3)
        sim.learn_set_mlp(tr.half)
        sim.learn_configure(2, omega)
        sim.step(2)
        sim.learn_counters(reset=True)
        t = sim.step_timed(2) / 2
        acc, fb, full = sim.learn_counters()
        rho, u = sim.macroscopic()
        st = sim.stats()
        sim.close()
        return acc, fb, full, rho, u, rho0, st, t

    acc, fb, full, rho, u, rho0, st, t = run(3000)
    acc0, fb0, _, _, _, _, _, t0 = run(0)
    print("learned rank: accepted %d, fell back %d, full SVDs %d; ms/step %.1f (full SVD %.1f, "
          "untrained %.1f); untrained accepted %d of %d" % (acc, fb, full, t, t_full, t0, acc0, acc0 + fb0))
    assert st["status"] == 0 and st["max_bond"] <= 64
    assert acc > 0
    assert acc / (acc + fb) > acc0 / max(acc0 + fb0, 1)
    assert rel_l2(u, u_r) <= 1e-3 and rel_l2(rho, rho_r) <= 1e-4
    assert abs(rho.sum() - rho0.sum()) / rho0.sum() <= 1e-6
