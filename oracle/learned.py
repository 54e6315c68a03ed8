"""Learned-rank rounding: randomized truncation with an exact certificate, and
the rank-predicting MLP (test infrastructure only).

Neither part is in the paper; they replace the full SVD of the rounding sweep
(Eq. svd-move) where that is safe.

Randomized truncation of the centre matrix C (m x n) at target rank k:
  l = min(max(k + p, l_min), m, n);  Y = C Omega[:n, :l];
  q power steps (each: Q = qr(Y); Z = qr(C^T Q); Y = C Z);
  Q = qr(Y);  B = Q^T C;  B = U S V^T;  the candidate rank r follows the usual
  rule applied to the true errors:  err(r)^2 = ||C - Q B||^2 + sum_{j >= r} s_j^2.
Since C^T C = B^T B + E^T E with E = C - Q B (Q^T E = 0), Ky Fan's inequality
bounds the optimal rank-r error from below by err(r)^2 - ||E||^2, so
||E||^2 <= eta err(r)^2 proves err(r)^2 <= opt(r)^2 / (1 - eta).  The result is
accepted when the rank rule is met inside the sample and either the measured
error is within the tolerance (err(r) <= delta) or, at the chi_max cap, the
near-optimality bound above holds; otherwise the full SVD is used.  A spectrum
with a flat tail beyond the sample cannot be certified this way and falls
back.  Omega is a fixed Gaussian matrix passed in (drawn by synth).  The
sample has at least l_min = 16 columns so that the spectrum it yields carries
the 16 values the rank model reads at the next step.

MLP: input 18 features (top-16 log10 singular values of the previous step at
that bond, relative to the largest; bond index / L; min(step / 1000, 1)),
two hidden layers of 64 with ReLU, one linear output = predicted rank / chi.
Loss: mean squared error.  Pinned by tests/test_oracle_learned.py (finite
differences for the gradients; the randomized truncation equals the full SVD
when the sample covers the whole range; the certificate rejects a sample that
misses part of the spectrum).
"""

import numpy as np

from .mps import choose_rank, left_orthogonalize, qr_pos

N_FEAT = 18
HIDDEN = 64


# ---------------------------------------------------------------- features
def spectrum_features(s, bond, L, step):
    """Features of one bond from its singular values s (descending)."""
    f = np.full(N_FEAT, -20.0)
    if len(s) and s[0] > 0:
        top = np.asarray(s[:16], dtype=np.float64)
        f[: len(top)] = np.log10(np.maximum(top / s[0], 1e-20))
    f[16] = bond / float(L)
    f[17] = min(step / 1000.0, 1.0)
    return f


# ---------------------------------------------------------------- MLP
def mlp_init(seed):
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((HIDDEN, N_FEAT)) * np.sqrt(2.0 / N_FEAT)
    W2 = rng.standard_normal((HIDDEN, HIDDEN)) * np.sqrt(2.0 / HIDDEN)
    W3 = rng.standard_normal((1, HIDDEN)) * np.sqrt(1.0 / HIDDEN)
    return {"W1": W1, "b1": np.zeros(HIDDEN), "W2": W2, "b2": np.zeros(HIDDEN),
            "W3": W3, "b3": np.zeros(1)}


def mlp_forward(P, X):
    """X (M x 18) -> (prediction (M,), cache)."""
    z1 = X @ P["W1"].T + P["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ P["W2"].T + P["b2"]
    h2 = np.maximum(z2, 0.0)
    out = (h2 @ P["W3"].T + P["b3"])[:, 0]
    return out, (X, z1, h1, z2, h2)


def mlp_loss_grad(P, X, y):
    """Mean squared error and its gradients with respect to every parameter."""
    out, (X, z1, h1, z2, h2) = mlp_forward(P, X)
    M = X.shape[0]
    d = (out - y)                                   # (M,)
    loss = float(np.mean(d * d))
    g_out = (2.0 / M) * d[:, None]                  # (M, 1)
    gW3 = g_out.T @ h2
    gb3 = g_out.sum(axis=0)
    g_h2 = g_out @ P["W3"]
    g_z2 = g_h2 * (z2 > 0)
    gW2 = g_z2.T @ h1
    gb2 = g_z2.sum(axis=0)
    g_h1 = g_z2 @ P["W2"]
    g_z1 = g_h1 * (z1 > 0)
    gW1 = g_z1.T @ X
    gb1 = g_z1.sum(axis=0)
    return loss, {"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3}


# ---------------------------------------------------------------- randomized truncation
def rsvd_truncate(C, k, omega, chi_max, delta, p=8, eta=0.2, floor_rel=1e-12, l_min=16, q=1):
    """Randomized truncation of C at target rank k.  Returns
    (accepted, r, U*S (m x r), Vt (r x n), err_r^2, residual^2).  Residuals
    below (floor_rel ||C||)^2 count as round-off (a sample that spans C)."""
    m, n = C.shape
    l = min(max(k + p, l_min), m, n)
    Y = C @ omega[:n, :l]
    for _ in range(q):
        Qy, _ = qr_pos(Y)
        Z, _ = qr_pos(C.T @ Qy)
        Y = C @ Z
    Q, _ = qr_pos(Y)
    B = Q.T @ C
    U, S, Vt = np.linalg.svd(B, full_matrices=False)
    resid2 = float(np.sum((C - Q @ B) ** 2))
    tails = np.zeros(len(S) + 1)
    acc = 0.0
    for j in range(len(S) - 1, -1, -1):
        acc += S[j] * S[j]
        tails[j] = acc
    rmax = min(chi_max, len(S))
    r = rmax
    for rr in range(1, rmax + 1):
        if np.sqrt(resid2 + tails[rr]) <= delta:
            r = rr
            break
    err2 = resid2 + tails[r]
    full_cap = min(chi_max, m, n)
    rule_ok = (np.sqrt(err2) <= delta) or (r == full_cap) or (r == chi_max)
    floor2 = (floor_rel * np.sqrt(np.sum(C * C))) ** 2
    accepted = bool(rule_ok and (np.sqrt(err2) <= delta or resid2 <= max(eta * err2, floor2)))
    return accepted, r, (Q @ U[:, :r]) * S[None, :r], Vt[:r], err2, resid2


SIGN_PROBE_STEP = 0.6180339887498949      # golden-ratio step of the probe weights


def sign_probe(n):
    """Weights w_c = frac((c + 1) * 0.618...) + 0.25 of the sign gauge: a
    generic positive vector, so that no structured singular vector (entries of
    equal magnitude, mirror symmetries) is orthogonal to it."""
    c = np.arange(1, n + 1, dtype=np.float64) * SIGN_PROBE_STEP
    return c - np.floor(c) + 0.25


def canonical_signs(US, Vt):
    """Fix the sign freedom of each kept singular pair: every row of Vt gets a
    positive inner product with the probe weights, and the matching column of
    US is flipped with it.  The randomized range finder draws its sample in
    the frame of the right bond, so both implementations must leave that frame
    in the same gauge for their samples to agree."""
    US = US.copy()
    Vt = Vt.copy()
    w = sign_probe(Vt.shape[1])
    for j in range(Vt.shape[0]):
        if float(Vt[j] @ w) < 0:
            Vt[j] = -Vt[j]
            US[:, j] = -US[:, j]
    return US, Vt


def round_mps_learned(cores, chi_max, eps, targets, omega, p=8, eta=0.2, spectra=None, q=1):
    """round_mps with the randomized truncation at target ranks targets[k]
    (bond k, 1 <= k < L; None or 0 = full SVD) and the full SVD as fallback.
    Bonds whose sample would cover the whole matrix (l = min(m, n)) take the
    full SVD directly.
    Every step leaves its singular pairs in the sign gauge of canonical_signs.
    Returns (cores, n_accepted, n_fallback).  If `spectra` is a dict, the full
    or randomized singular values of each bond are stored in it."""
    L = len(cores)
    A = left_orthogonalize(cores)
    nrm = float(np.sqrt(np.sum(A[L - 1] ** 2)))
    delta = eps * nrm / np.sqrt(L - 1)
    n_acc = n_fb = 0
    for k in range(L - 1, 0, -1):
        r0, d, r1 = A[k].shape
        Cm = A[k].reshape(r0, d * r1)
        done = False
        tk = None if targets is None or targets[k] is None else min(int(targets[k]), chi_max)
        if tk and min(max(tk + p, 16), r0, d * r1) < min(r0, d * r1):
            ok, r, US, Vt, _, _ = rsvd_truncate(Cm, tk, omega, chi_max, delta, p, eta, q=q)
            if ok:
                n_acc += 1
                done = True
            else:
                n_fb += 1
        if not done:
            U, S, Vt = np.linalg.svd(Cm, full_matrices=False)
            r = choose_rank(S, chi_max, delta)
            US = U[:, :r] * S[None, :r]
            Vt = Vt[:r]
            if spectra is not None:
                spectra[k] = S.copy()
        US, Vt = canonical_signs(US, Vt)
        A[k] = Vt.reshape(r, d, r1)
        A[k - 1] = np.tensordot(A[k - 1], US, axes=(2, 0))
    return A, n_acc, n_fb
