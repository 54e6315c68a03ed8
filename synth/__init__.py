"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

This module holds input generation only: voxel geometries, and the factor
tensors of smooth perturbation fields written directly as tensor-train cores.
It contains none of the lattice Boltzmann or MPS arithmetic of the method
(no rounding, no products, no streaming); both the oracle and the CUDA path
consume what it returns and do their own arithmetic on it.

Every generator takes an explicit seed and uses numpy's PCG64 generator.
"""

from .geometry import channel, sphere_pack, vessel_tree, box_obstacle, sphere_cell, cell_pattern
from .fields import fourier_modes, random_mps, feasible_ranks, gaussian_matrix, taylor_green_modes

__all__ = [
    "channel", "sphere_pack", "vessel_tree", "box_obstacle", "sphere_cell", "cell_pattern",
    "fourier_modes", "random_mps", "feasible_ranks", "gaussian_matrix", "taylor_green_modes",
]
