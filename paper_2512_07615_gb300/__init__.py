"""GB300-native MPS lattice Boltzmann (tensor-network LBM) library.

The compute path is libtnlbm.so (hand-written CUDA for sm_103a) behind the C
ABI in include/tnlbm.h; this package only marshals arguments to it.
"""
from .native import lib, Config, Stats, Term, TnlbmError  # noqa: F401
from .tnlbm import DeviceMps, Sim, Batch, lincomb_round, materialize, hadamard_fit, inner_ones, to_dense, from_dense  # noqa: F401
