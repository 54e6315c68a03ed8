"""The allocation-free rounding entry point (tnlbm_lincomb_round_noalloc).

Callers that cannot allocate device memory where they need a rounding (their
device memory is entirely held by a pool allocator, or they must not stall the
device, which cudaFree does) use this entry point: it works in the library's
fixed static device arrays instead of calling cudaMalloc.  This file runs last
so that a failure here leaves every other test already run; it must pass alone
in a fresh process (the first call does the per-device set-up) and after the
other tests.  Two calls in a row are compared with the allocating entry point
(the same kernel on the same inputs, so the results agree to round-off or
better), and oversized requests must be refused with an error.
"""
import numpy as np
import pytest

import synth
from oracle import mps as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2512_07615_gb300 import tnlbm
    return tnlbm


def _case(T, seed, L, chi, nb, prec):
    srcs, batches, keep = [], [], []
    for b in range(nb):
        A = synth.random_mps(L, synth.feasible_ranks(L, chi), seed + 2 * b)
        B = synth.random_mps(L, synth.feasible_ranks(L, chi - 1), seed + 2 * b + 1)
        dA, dB = T.DeviceMps.from_cores(A, chi, prec), T.DeviceMps.from_cores(B, chi, prec)
        keep += [dA, dB]
        vec = np.random.default_rng(seed + b).uniform(0.5, 1.5, (L, 2))
        batches.append([T.plain(dA, 1.0), T.plain(dB, -0.25), T.mask1(dA, vec, 0.5), T.ones(0.1)])
    return batches, keep


@pytest.mark.parametrize("prec", [0, 1])
def test_noalloc_matches_allocating_entry_point_twice(T, prec):
    tol = 1e-12 if prec == 0 else 1e-5
    for call, (seed, L, chi, nb) in enumerate([(100, 12, 16, 3), (200, 9, 8, 5)]):
        batches, keep = _case(T, seed, L, chi, nb, prec)
        ref = [T.DeviceMps(L, 2 * chi, prec) for _ in range(nb)]
        out = [T.DeviceMps(L, 2 * chi, prec) for _ in range(nb)]
        T.lincomb_round(batches, ref, 2 * chi, 1e-9)
        T.lincomb_round_noalloc(batches, out, 2 * chi, 1e-9)
        for a, b in zip(out, ref):
            ta, tb = M.to_tensor(a.cores()), M.to_tensor(b.cores())
            assert np.linalg.norm(ta - tb) <= tol * np.linalg.norm(tb), call
            assert a.bonds() == b.bonds()


def test_noalloc_refuses_oversized_requests(T):
    from paper_2512_07615_gb300.native import TnlbmError
    L, chi = 9, 8
    one = T.DeviceMps.from_cores(M.ones(L), 2, 0)
    too_many = [[T.plain(one)] for _ in range(65)]          # job table holds 64
    dst = [T.DeviceMps(L, chi, 0) for _ in range(65)]
    with pytest.raises(TnlbmError) as ei:
        T.lincomb_round_noalloc(too_many, dst, chi, 0.0)
    assert ei.value.code == -1 and "64" in str(ei.value)
    big = T.DeviceMps.from_cores(synth.random_mps(30, synth.feasible_ranks(30, 256), 1), 256, 0)
    with pytest.raises(TnlbmError) as ei:                   # needs far more than 16 MiB scratch
        T.lincomb_round_noalloc([[T.plain(big), T.plain(big)]], [T.DeviceMps(30, 256, 0)], 256, 0.0)
    assert ei.value.code == -1 and "16 MiB" in str(ei.value)
