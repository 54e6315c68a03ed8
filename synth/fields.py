"""Seeded parameters of smooth synthetic fields, and random tensor-train cores.

Random numbers that the method's inputs need are drawn here and passed to both
the oracle and the CUDA library, so neither side draws its own.
"""

import numpy as np


def fourier_modes(n_modes, seed, kmax=4, amp_rho=1e-3, amp_u=1e-3):
    """Parameters of n_modes plane waves cos(2 pi k.x / N + phase).

    Returns an (n_modes, 8) float64 array with columns
    kx, ky, kz (integers in [-kmax, kmax], not all zero), phase in [0, 2 pi),
    and the amplitudes a_rho, a_ux, a_uy, a_uz of that mode in the density and
    velocity perturbations (uniform in [-amp, amp]).
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((n_modes, 8))
    for m in range(n_modes):
        while True:
            k = rng.integers(-kmax, kmax + 1, size=3)
            if np.any(k != 0):
                break
        out[m, 0:3] = k
        out[m, 3] = rng.uniform(0.0, 2.0 * np.pi)
        out[m, 4] = rng.uniform(-amp_rho, amp_rho)
        out[m, 5:8] = rng.uniform(-amp_u, amp_u, size=3)
    return out


def random_mps(L, ranks, seed, scale=None):
    """Random cores (r_k, 2, r_{k+1}) with standard normal entries.

    ranks is the list of the L+1 bond dimensions (first and last 1).  With
    scale=None every core is divided by sqrt(2 r_k) so that contracted entries
    stay of order one.
    """
    assert len(ranks) == L + 1 and ranks[0] == 1 and ranks[-1] == 1
    rng = np.random.default_rng(seed)
    cores = []
    for k in range(L):
        c = rng.standard_normal((ranks[k], 2, ranks[k + 1]))
        s = (1.0 / np.sqrt(2.0 * ranks[k])) if scale is None else scale
        cores.append(c * s)
    return cores


def feasible_ranks(L, chi):
    """Bond dimensions min(chi, 2**k, 2**(L-k)) of a generic MPS of L binary sites."""
    return [min(chi, 2 ** k, 2 ** (L - k)) for k in range(L + 1)]


def gaussian_matrix(rows, cols, seed):
    """Fixed standard normal test matrix of the randomized range finder."""
    return np.random.default_rng(seed).standard_normal((rows, cols))


def taylor_green_modes(u0):
    """The Taylor-Green vortex in the plane-wave form of fourier_modes, with
    x = 2 pi X / N:  u = u0 (sin x cos y cos z, -cos x sin y cos z, 0) and the
    density perturbation 3 u0^2 / 16 (cos 2x + cos 2y)(cos 2z + 2) of its
    pressure.  Product-to-sum: sin x cos y cos z = 1/4 sum of sin(x +- y +- z),
    cos x sin y cos z = 1/4 [sin(x+y+z) + sin(x+y-z) - sin(x-y+z) - sin(x-y-z)],
    and sin t = cos(t - pi/2).  Returns a (10, 8) array (rows as fourier_modes)."""
    h = -0.5 * np.pi
    q = u0 / 4.0
    d = 3.0 * u0 * u0 / 16.0
    rows = [
        [1, 1, 1, h, 0.0, q, -q, 0.0],
        [1, 1, -1, h, 0.0, q, -q, 0.0],
        [1, -1, 1, h, 0.0, q, q, 0.0],
        [1, -1, -1, h, 0.0, q, q, 0.0],
        [2, 0, 2, 0.0, d / 2, 0.0, 0.0, 0.0],
        [2, 0, -2, 0.0, d / 2, 0.0, 0.0, 0.0],
        [0, 2, 2, 0.0, d / 2, 0.0, 0.0, 0.0],
        [0, 2, -2, 0.0, d / 2, 0.0, 0.0, 0.0],
        [2, 0, 0, 0.0, 2 * d, 0.0, 0.0, 0.0],
        [0, 2, 0, 0.0, 2 * d, 0.0, 0.0, 0.0],
    ]
    return np.array(rows, dtype=np.float64)
