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
