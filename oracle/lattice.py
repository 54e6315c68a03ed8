"""Velocity sets, Sec. 3.1 (the paper uses D3Q15 in 3-D with c_s^2 = 1/3;
D3Q19 is the lattice of the synthetic channel, porous and vessel workloads).

The paper prints no weights; these are the standard weights of the two
lattices.  Ordering: the rest velocity first, then opposite pairs next to each
other, so that the opposite of i > 0 is i + 1 for odd i and i - 1 for even i.

Pinned by tests/test_oracle_lattice.py: the isotropy conditions up to fourth
order, which fix the weights of each velocity shell.
"""

import numpy as np

CS2 = 1.0 / 3.0

_D3Q19 = [
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0),
    (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1),
    (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1),
]
_D3Q15 = [
    (0, 0, 0),
    (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
    (1, 1, 1), (-1, -1, -1), (1, 1, -1), (-1, -1, 1),
    (1, -1, 1), (-1, 1, -1), (-1, 1, 1), (1, -1, -1),
]


class Lattice:
    def __init__(self, name):
        if name == "D3Q19":
            c = _D3Q19
            w = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12
        elif name == "D3Q15":
            c = _D3Q15
            w = [2.0 / 9.0] + [1.0 / 9.0] * 6 + [1.0 / 72.0] * 8
        else:
            raise ValueError(name)
        self.name = name
        self.c = np.array(c, dtype=np.int64)
        self.w = np.array(w, dtype=np.float64)
        self.Q = len(c)
        self.opp = np.array([0] + [i + 1 if i % 2 == 1 else i - 1 for i in range(1, self.Q)])


D3Q19 = Lattice("D3Q19")
D3Q15 = Lattice("D3Q15")


def get(name):
    return {"D3Q19": D3Q19, "D3Q15": D3Q15}[name]
