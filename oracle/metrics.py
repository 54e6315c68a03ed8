"""Metrics of Sec. 3.2.

rel_l2            epsilon_l2 = ||u - u_ref|| / ||u_ref|| over all components and cells
nvps_fused        NVPS of the paper's fused-site MPS (2^D physical dimension per
                  site, n sites), the formula of Sec. 3.2
compression_ratio NVPS_ref / NVPS with NVPS_ref = (2^n)^D
nvps_binary       NVPS of an MPS with binary sites from its realised bonds

Pinned by tests/test_oracle_metrics.py against the compression ratios printed
in Sec. 4 (TGV, aneurysm, pin-fin) and App. A; nvps_binary against the number
of values held by TT-SVD cores and by the product state.
"""

import numpy as np


def rel_l2(u, u_ref):
    u = np.asarray(u, dtype=np.float64)
    u_ref = np.asarray(u_ref, dtype=np.float64)
    return float(np.sqrt(np.sum((u - u_ref) ** 2)) / np.sqrt(np.sum(u_ref ** 2)))


def nvps_fused(n, D, chi):
    q = 2 ** D
    total = 0
    for i in range(1, n + 1):
        left = min(q ** (i - 1), q ** (n - i + 1), chi)
        right = min(q ** i, q ** (n - i), chi)
        total += left * q * right
    return total


def compression_ratio(n, D, chi):
    return (2 ** n) ** D / nvps_fused(n, D, chi)


def nvps_binary(bonds):
    """bonds = [r_0, ..., r_L] of one MPS with binary sites."""
    return int(sum(bonds[k] * 2 * bonds[k + 1] for k in range(len(bonds) - 1)))
