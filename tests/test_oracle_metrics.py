"""Pins of the compression-ratio formula against the paper's printed values."""
import pytest

from oracle import metrics
from conftest import read_golden


@pytest.mark.parametrize("row", read_golden("compression_ratios.txt"))
def test_printed_compression_ratios(row):
    n, D, chi, printed, tol = row
    assert abs(metrics.compression_ratio(int(n), int(D), int(chi)) - printed) <= tol


def test_full_rank_mps_has_no_compression():
    # chi large enough: NVPS >= the dense count
    assert metrics.compression_ratio(3, 3, 10 ** 6) <= 1.0


def test_rel_l2():
    assert metrics.rel_l2([3.0, 4.0], [3.0, 4.0]) == 0.0
    assert abs(metrics.rel_l2([0.0, 0.0], [3.0, 4.0]) - 1.0) < 1e-15


def test_nvps_binary_counts_the_stored_values():
    """NVPS of a binary-site MPS is the number of values its cores hold: pinned
    by the product state (2 L values), by the two-site full-rank MPS (bonds
    1, 2, 1: 8 values) and by the sizes of TT-SVD cores of a random tensor
    (ragged bonds 2, 4, ..., 4, 2)."""
    import numpy as np
    from oracle import mps as M
    L = 7
    assert metrics.nvps_binary([1] * (L + 1)) == 2 * L
    assert metrics.nvps_binary([1, 2, 1]) == 8
    x = np.random.default_rng(3).standard_normal((2,) * L)
    cores = M.tt_svd(x, 64, 0.0)
    assert M.ranks(cores) == [1, 2, 4, 8, 8, 4, 2, 1]
    assert metrics.nvps_binary(M.ranks(cores)) == sum(c.size for c in cores)
