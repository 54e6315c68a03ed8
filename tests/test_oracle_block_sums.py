"""Pin of the alternative linear fold: the moments as one rounded block sum of
all populations give the same step as the pairwise tree when nothing is
truncated."""
import numpy as np

import synth
from oracle import lattice, mps_lbm as ml


def test_block_sum_moments_equal_pairwise_untruncated():
    """The alternative linear fold (one block sum for the moments) gives the
    same step as the pairwise tree when nothing is truncated."""
    lat = lattice.D3Q19
    modes = synth.fourier_modes(3, 8, kmax=2, amp_rho=1e-2, amp_u=1e-2)
    a = ml.Config(3, lat, 0.8, periodic=(1, 1, 0), force=(1e-4, 0, 0), chi_max=4096, eps=0.0, hadamard="exact")
    b = ml.Config(3, lat, 0.8, periodic=(1, 1, 0), force=(1e-4, 0, 0), chi_max=4096, eps=0.0, hadamard="exact",
                  block_sums=True)
    fa = ml.step(a, ml.initial_perturbed(a, modes))
    fb = ml.step(b, ml.initial_perturbed(b, modes))
    da, db = ml.to_dense_populations(fa), ml.to_dense_populations(fb)
    assert np.abs(da - db).max() <= 1e-13 * np.abs(da).max()
