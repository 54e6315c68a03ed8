"""Seeded voxel geometries on an N^3 lattice, indexed [x][y][z], 1 = solid.

These stand in for the paper's geometries (Sec. 3.1: an idealised aneurysm and a
pin-fin heat sink), which are not available: a plain channel, a periodic packing
of spheres (porous medium) and a binary tree of cylinders (branching vessel).
"""

import numpy as np


def channel(n_bits):
    """Empty domain of N = 2**n_bits cells per axis (walls come from the
    boundary flags, not from voxels)."""
    N = 1 << n_bits
    return np.zeros((N, N, N), dtype=np.uint8)


def box_obstacle(n_bits, lo, hi):
    """Axis-aligned solid box lo <= x < hi (per axis).  Its mask has a small
    exact tensor-train rank, which makes it useful for exact-mask tests."""
    N = 1 << n_bits
    m = np.zeros((N, N, N), dtype=np.uint8)
    m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1
    return m


def sphere_pack(n_bits, radius, solid_fraction, seed):
    """Periodic porous medium: spheres of the given radius with centres drawn
    uniformly in [0, N)^3 (minimum-image periodic distance), added one at a
    time (overlap allowed) until the solid fraction reaches the target."""
    N = 1 << n_bits
    rng = np.random.default_rng(seed)
    ax = np.arange(N, dtype=np.float64) + 0.5
    solid = np.zeros((N, N, N), dtype=bool)
    target = solid_fraction * N ** 3
    r2 = float(radius) ** 2
    while solid.sum() < target:
        c = rng.uniform(0.0, N, size=3)
        d = []
        for k in range(3):
            t = np.abs(ax - c[k])
            d.append(np.minimum(t, N - t) ** 2)
        solid |= (d[0][:, None, None] + d[1][None, :, None] + d[2][None, None, :]) <= r2
    return solid.astype(np.uint8)


def _unit(v):
    return v / np.linalg.norm(v)


def _segment_mask(N, p0, p1, r, grid):
    """Cells whose centre lies within distance r of the segment p0-p1."""
    d = p1 - p0
    L2 = float(d @ d)
    rel = grid - p0
    t = np.clip((rel @ d) / L2, 0.0, 1.0)
    closest = p0 + t[..., None] * d
    dist2 = ((grid - closest) ** 2).sum(-1)
    return dist2 <= r * r


def vessel_tree(n_bits, root_radius, depth, seed, length_factor=3.0,
                half_angle_deg=(25.0, 45.0)):
    """Branching vessel: a symmetric binary tree of cylinders.

    The root starts left of the domain centre and points along +x.  Each
    generation halves the flow area by Murray's law (child radius r / 2**(1/3)),
    segments are length_factor * parent radius long, each bifurcation opens by a
    half-angle drawn uniformly from half_angle_deg, and the branching plane is
    rotated uniformly about the parent axis.  Fluid is the union of cylinders
    (with spherical joints); everything else is solid.
    """
    N = 1 << n_bits
    rng = np.random.default_rng(seed)
    c = np.arange(N, dtype=np.float64) + 0.5
    fluid = np.zeros((N, N, N), dtype=bool)
    start = np.array([0.25 * N, 0.5 * N, 0.5 * N])
    stack = [(start, np.array([1.0, 0.0, 0.0]), float(root_radius), 0)]
    while stack:
        p0, direction, r, gen = stack.pop()
        seg_len = length_factor * r
        p1 = p0 + seg_len * direction
        # only the cells of the segment's bounding box can lie within r of it
        lo = np.maximum(np.floor(np.minimum(p0, p1) - r - 1.0).astype(int), 0)
        hi = np.minimum(np.ceil(np.maximum(p0, p1) + r + 1.0).astype(int), N)
        if np.all(hi > lo):
            sub = np.stack(np.meshgrid(c[lo[0]:hi[0]], c[lo[1]:hi[1]], c[lo[2]:hi[2]], indexing="ij"), axis=-1)
            fluid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] |= _segment_mask(N, p0, p1, r, sub)
        if gen + 1 >= depth:
            continue
        # an orthonormal frame around the parent axis
        helper = np.array([0.0, 0.0, 1.0]) if abs(direction[2]) < 0.9 else np.array([0.0, 1.0, 0.0])
        e1 = _unit(np.cross(direction, helper))
        e2 = np.cross(direction, e1)
        rot = rng.uniform(0.0, 2.0 * np.pi)
        normal = np.cos(rot) * e1 + np.sin(rot) * e2
        r_child = r / 2.0 ** (1.0 / 3.0)
        for sign in (1.0, -1.0):
            a = np.deg2rad(rng.uniform(*half_angle_deg))
            child = _unit(np.cos(a) * direction + sign * np.sin(a) * normal)
            stack.append((p1, child, r_child, gen + 1))
    return (~fluid).astype(np.uint8)


def sphere_cell(n_bits, radius):
    """One cell of a periodic array: a solid sphere of `radius` cells centred in
    a (2^n_bits)^3 cell."""
    N = 1 << n_bits
    c = (N - 1) / 2.0
    x = np.arange(N)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    return (((X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2) <= radius * radius).astype(np.uint8)


def cell_pattern(n_bits, fill, seed):
    """Which cells of a (2^n_bits)^3 arrangement hold the inner geometry: each
    independently with probability `fill`."""
    N = 1 << n_bits
    rng = np.random.default_rng(seed)
    return (rng.uniform(size=(N, N, N)) < fill).astype(np.uint8)
