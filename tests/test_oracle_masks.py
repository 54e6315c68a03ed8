"""Pins of the combined-scale mask of App. D: the MPS built by concatenating
the outer and inner MPS equals the definition m_outer(x >> k) m_inner(x mod 2^k)
cell by cell, and its largest bond is max(chi_outer, chi_inner) with bond 1
at the junction."""
import numpy as np

import synth
from oracle import masks, mps as M, quantics as q


def test_combined_mask_equals_definition_and_bond_bound():
    outer = synth.cell_pattern(2, 0.5, 3).astype(float)          # 4^3 arrangement
    inner = synth.sphere_cell(3, 2.6).astype(float)              # sphere in an 8^3 cell
    A = M.tt_svd(q.encode(outer), 64, 0.0)
    B = M.tt_svd(q.encode(inner), 64, 0.0)
    C = masks.mask_product(A, B)
    dense = q.decode(M.to_tensor(C))
    ref = masks.combined_dense(outer, inner)
    assert ref.shape == (32, 32, 32)
    np.testing.assert_allclose(dense, ref, atol=1e-12)
    r = M.ranks(C)
    assert max(r) == max(max(M.ranks(A)), max(M.ranks(B)))
    assert r[len(A)] == 1


def test_combined_dense_definition_by_loops():
    """The vectorised definition against explicit loops on a tiny case."""
    outer = synth.cell_pattern(1, 0.5, 4)
    inner = synth.sphere_cell(1, 0.9)
    d = masks.combined_dense(outer, inner)
    for x in range(4):
        for y in range(4):
            for z in range(4):
                assert d[x, y, z] == outer[x // 2, y // 2, z // 2] * inner[x % 2, y % 2, z % 2]
