"""CPU checks of the C ABI: the library builds, loads, exports every symbol
declared in include/tnlbm.h, its layout helpers agree with the documented
formula, and argument errors are reported without touching a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tnlbm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2512_07615_gb300 import build
    build.build()
    import paper_2512_07615_gb300 as tl
    return tl.lib()


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tnlbm_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tnlbm_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_layout_helpers(lib):
    # capacity 1 at the two ends, cap inside; slot k = cap_k * 2 * cap_(k+1)
    for L, cap in [(3, 1), (9, 4), (15, 16), (21, 64)]:
        caps = [1] + [cap] * (L - 1) + [1]
        offs = [0]
        for k in range(L):
            offs.append(offs[-1] + caps[k] * 2 * caps[k + 1])
        assert lib.tnlbm_mps_size(L, cap) == offs[-1]
        for k in range(L + 1):
            assert lib.tnlbm_mps_offset(L, cap, k) == offs[k]


def test_argument_errors_without_gpu(lib):
    import paper_2512_07615_gb300.native as nat
    h = ctypes.c_void_p()
    assert lib.tnlbm_create(None, ctypes.byref(h)) == -1
    c = nat.Config()
    c.n_per_axis = 3
    c.lattice = 17           # not a supported velocity set
    c.tau = 0.8
    c.chi_max = 8
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"lattice" in lib.tnlbm_last_error()
    c.lattice = 19
    c.tau = 0.4              # unstable relaxation time
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert lib.tnlbm_step(None, 1) == -1
    assert lib.tnlbm_destroy(None) == 0
    assert lib.tnlbm_lincomb_round(0, 3, 1, 0, None, None, None, 4, 4, 0.0, None) == -1


def test_oracle_not_imported_by_package():
    """The product package must not reach the oracle."""
    pkg = os.path.join(ROOT, "paper_2512_07615_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("no oracle", ""), f


def test_argument_errors_of_the_newer_entry_points(lib):
    """Zip-up product, plane slices, batches and the config options added
    with them (precision TF32, zip-up products, block sums) reject bad
    arguments before any device call."""
    import paper_2512_07615_gb300.native as nat
    h = ctypes.c_void_p()
    # zip-up primitive: NULL operands, chi above the supported 512
    assert lib.tnlbm_hadamard_zipup(0, 3, 1, None, None, 4, None, None, 4, None, None, 8, 8, 0.0, None) == -1
    assert b"zipup" in lib.tnlbm_last_error()
    assert lib.tnlbm_hadamard_zipup(0, 3, 0, None, None, 4, None, None, 4, None, None, 600, 600, 0.0, None) == -1
    # plane slice of no simulation
    assert lib.tnlbm_macroscopic_slice(None, 0, 0, None, None) == -1
    # batches
    assert lib.tnlbm_batch_create(None, 0, ctypes.byref(h)) == -1
    assert lib.tnlbm_batch_step(None, 1) == -1
    # cluster sizes of no simulation / batch
    n = ctypes.c_int()
    ms = (ctypes.c_double * 17)()
    assert lib.tnlbm_clusters(None, None, None, 0, ctypes.byref(n)) == -1
    assert lib.tnlbm_set_clusters(None, None, 0) == -1
    assert lib.tnlbm_tune_clusters(None, 1, ms, 17) == -1
    assert lib.tnlbm_batch_clusters(None, None, None, 0, ctypes.byref(n)) == -1
    assert lib.tnlbm_batch_set_clusters(None, None, 0) == -1
    assert lib.tnlbm_batch_tune_clusters(None, 1, ms, 17) == -1
    assert b"tune_clusters" in lib.tnlbm_last_error()
    c = nat.Config()
    c.n_per_axis = 3
    c.lattice = 19
    c.tau = 0.8
    c.chi_max = 8
    c.eps = 1e-8
    c.precision = 7                     # no such precision
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"precision" in lib.tnlbm_last_error()
    c.precision = nat.TF32
    c.hadamard = 3                      # no such product
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"hadamard" in lib.tnlbm_last_error()
    c.hadamard = nat.HADAMARD_ZIPUP
    c.chi_max = 600                     # zip-up bonds are capped at 512
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    c.hadamard = nat.HADAMARD_FIT
    c.chi_max = 64
    c.block_sums = 1                    # 19 x 64 > 1024: the summed bond of one rounding
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"block_sums" in lib.tnlbm_last_error()


def test_argument_errors_of_the_precision_and_failure_options(lib):
    """Mixed precision, the learned-rank and seed members, the Jacobi sweep
    cap, the wait limit and the cluster cap reject bad values before any
    device call."""
    import paper_2512_07615_gb300.native as nat
    h = ctypes.c_void_p()
    c = nat.Config()
    c.n_per_axis = 3
    c.lattice = 19
    c.tau = 0.8
    c.chi_max = 8
    c.eps = 1e-8
    c.precision = nat.MIXED
    for field, bad in (("max_cluster", 17), ("max_cluster", 32), ("max_cluster", -1),
                       ("jacobi_max_sweeps", -1), ("wait_limit_ns", -5)):
        setattr(c, field, bad)
        assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1, field
        assert b"max_cluster" in lib.tnlbm_last_error()
        setattr(c, field, 0)
    c.learned_rank = 2                  # the rank model needs a trained network first
    assert lib.tnlbm_create(ctypes.byref(c), ctypes.byref(h)) == -1
    assert b"learned_rank" in lib.tnlbm_last_error()
    c.learned_rank = 3                  # batched steps take the full SVD
    arr = (nat.Config * 2)(c, c)
    assert lib.tnlbm_batch_create(arr, 2, ctypes.byref(h)) == -1
    assert b"learned_rank" in lib.tnlbm_last_error() and not h.value
    c.learned_rank = 0
    # primitives: precision beyond the enum
    assert lib.tnlbm_lincomb_round(9, 3, 1, 1, None, None, None, 8, 8, 0.0, None) == -1
