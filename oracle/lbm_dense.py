"""Full-grid BGK lattice Boltzmann step in float64, Sec. 3.1 and App. A.

One step, collide then stream (Eq. evolution):
  moments          rho = sum_i f_i, j = sum_i c_i f_i              (Eq. macro)
  inverse density  'exact': 1/rho;  'taylor': second-order expansion about
                   the mean density rho_0 (Sec. 3.2), rho_0 = sum(rho)/N_fluid
  forcing          J~ = j + tau F (1 - m_O), u = J~ * inv         (App. A)
  collision        f*_i = f_i + (f^eq_i - f_i)/tau                (Eq. collision)
                   with w_i rho u.u terms written through P_de = J~_d u_e:
                   f^eq_i = w_i [rho + 3 c_i.J~ + 4.5 sum c_d c_e P_de
                                 - 1.5 sum_d P_dd]               (Eq. equilibrium)
                   which equals Eq. (equilibrium) exactly when inv = 1/rho
  streaming        f_i(x) = f*_i(x - c_i), cyclic on periodic axes; on wall
                   axes cells whose upstream neighbour lies outside receive the
                   halfway bounce-back value f*_opp(i)(x)  (Eq. boundaries2, no_slip)
  objects          f_i <- (1 - m_O) f_i + S(c_i)(m_O f_opp(i))     (Eq. objects)
                   with the product m_O f_i formed once and used in both terms.
  faces            optional per-face boundary functions b of Eq. (boundaries2)
                   instead of bounce-back on every wall face; see face_value.

Fields are arrays f[i, x, y, z].  `mask` is m_O on the grid (binary, or the
contraction of a mask MPS), or None.

Pinned by tests/test_oracle_dense.py: mass conservation, momentum gain N_fluid F
per step (exact mode, periodic), the Poiseuille profile, shear-wave decay,
and taylor == exact at uniform density.
"""

import numpy as np

from .lattice import CS2


def equilibrium(lat, rho, u):
    """Eq. (equilibrium) with c_s^2 = 1/3: w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u)."""
    cu = np.einsum("id,d...->i...", lat.c.astype(np.float64), u)
    uu = np.sum(u * u, axis=0)
    w = lat.w.reshape((-1,) + (1,) * rho.ndim)
    return w * rho[None] * (1.0 + cu / CS2 + cu * cu / (2 * CS2 * CS2) - uu[None] / (2 * CS2))


def shift(g, c, periodic):
    """h(x) = g(x - c); on non-periodic axes the cells whose source lies
    outside the domain are set to zero (the non-cyclic shift)."""
    h = g
    for d in range(3):
        cd = int(c[d])
        if cd == 0:
            continue
        h = np.roll(h, cd, axis=d)
        if not periodic[d]:
            idx = [slice(None)] * 3
            idx[d] = 0 if cd > 0 else -1
            h = h.copy()
            h[tuple(idx)] = 0.0
    return h


def boundary_mask(shape, c, periodic):
    """m_B for velocity c: 1 where x - c lies outside along a wall axis."""
    m = np.zeros(shape)
    for d in range(3):
        cd = int(c[d])
        if cd == 0 or periodic[d]:
            continue
        idx = [slice(None)] * 3
        idx[d] = 0 if cd > 0 else shape[d] - 1
        m[tuple(idx)] = 1.0
    return m


FACE_WALL, FACE_VELOCITY, FACE_PRESSURE = 0, 1, 2


def face_index(d, cd):
    """Face through which a population with c_d = cd enters: 2d for the plane
    x_d = 0 (cd > 0), 2d + 1 for x_d = N - 1 (cd < 0)."""
    return 2 * d + (0 if cd > 0 else 1)


def face_masks(shape, c, periodic):
    """[(face, mask)]: a cell whose upstream neighbour x - c lies outside
    through several wall faces is assigned to the one of lowest axis; the
    masks partition the union of the incoming planes."""
    out = []
    taken = np.zeros(shape)
    for d in range(3):
        cd = int(c[d])
        if cd == 0 or periodic[d]:
            continue
        plane = np.zeros(shape)
        idx = [slice(None)] * 3
        idx[d] = 0 if cd > 0 else shape[d] - 1
        plane[tuple(idx)] = 1.0
        m = plane * (1.0 - taken)
        taken = np.maximum(taken, plane)
        out.append((face_index(d, cd), m))
    return out


def face_value(kind, lat, i, fstar_opp, rho0, u_b, rho_b, P):
    """Boundary function b(f*_opp(i), rho_b, u_b) of one face (Eqs. no_slip,
    boundaries2 and the velocity and pressure conditions of Sec. 3.2):
      wall      f*_opp
      velocity  f*_opp + 2 w_i rho_0 (c_i . u_b) / c_s^2, c_i pointing into the
                domain (moving-wall bounce-back, density rho_b = rho_0)
      pressure  -f*_opp + 2 w_i rho_b (1 + (c_i . u)^2 / (2 c_s^4) - u . u / (2 c_s^2))
                with u the local fluid velocity, u_d u_e taken as P_de / rho_0
                (P_de = J~_d u_e of the collision), which makes
                2 w_i rho_b (1 + sum_{d<=e} kappa_de P_de / rho_0)."""
    c = lat.c[i].astype(np.float64)
    w = lat.w[i]
    if kind == FACE_WALL:
        return fstar_opp
    if kind == FACE_VELOCITY:
        return fstar_opp + 2.0 * w * rho0 * float(c @ np.asarray(u_b, dtype=np.float64)) / CS2
    if kind == FACE_PRESSURE:
        acc = np.ones_like(fstar_opp)
        for de, kap in second_order_coeffs(lat.c[i]).items():
            if kap != 0.0:
                acc = acc + kap * P[de] / rho0
        return -fstar_opp + 2.0 * w * rho_b * acc
    raise ValueError(kind)


def moments(lat, f):
    rho = f.sum(axis=0)
    j = np.einsum("id,i...->d...", lat.c.astype(np.float64), f)
    return rho, j


def second_order_coeffs(c):
    """kappa_de for d <= e: 4.5 c_d^2 - 1.5 on the diagonal, 9 c_d c_e off it."""
    out = {}
    for d in range(3):
        for e in range(d, 3):
            out[(d, e)] = 4.5 * c[d] * c[d] - 1.5 if d == e else 9.0 * c[d] * c[e]
    return out


def step(f, lat, tau, force=(0.0, 0.0, 0.0), mask=None, periodic=(1, 1, 1), inv_mode="taylor",
         faces=None):
    """One collide-and-stream step; returns the new populations.  faces: None
    (bounce-back on every wall face) or six (kind, u_b, rho_b) for the faces
    x-, x+, y-, y+, z-, z+ (used on the non-periodic axes)."""
    omega = 1.0 / tau
    F = np.asarray(force, dtype=np.float64)
    m = np.zeros(f.shape[1:]) if mask is None else np.asarray(mask, dtype=np.float64)
    rho, j = moments(lat, f)
    if inv_mode == "taylor":
        n_fluid = np.sum(1.0 - m)
        rho0 = rho.sum() / n_fluid
        drho = rho - rho0
        inv = 1.0 / rho0 - drho / rho0 ** 2 + drho * drho / rho0 ** 3
    elif inv_mode == "exact":
        safe = np.where(rho > 0, rho, 1.0)
        inv = np.where(rho > 0, 1.0 / safe, 0.0)
    else:
        raise ValueError(inv_mode)
    Jt = j + tau * F[:, None, None, None] * (1.0 - m)[None]
    u = Jt * inv[None]
    P = {(d, e): Jt[d] * u[e] for d in range(3) for e in range(d, 3)}
    fstar = np.empty_like(f)
    for i in range(lat.Q):
        c = lat.c[i]
        E = rho.copy()
        for d in range(3):
            if c[d] != 0:
                E += 3.0 * c[d] * Jt[d]
        for de, kap in second_order_coeffs(c).items():
            if kap != 0.0:
                E += kap * P[de]
        fstar[i] = (1.0 - omega) * f[i] + omega * lat.w[i] * E
    fs = np.empty_like(f)
    rho0_b = rho.sum() / np.sum(1.0 - m)
    for i in range(lat.Q):
        c = lat.c[i]
        if faces is None:
            fs[i] = shift(fstar[i], c, periodic) + boundary_mask(f.shape[1:], c, periodic) * fstar[lat.opp[i]]
        else:
            fs[i] = shift(fstar[i], c, periodic)
            for face, fm in face_masks(f.shape[1:], c, periodic):
                kind, u_b, rho_b = faces[face]
                fs[i] = fs[i] + fm * face_value(kind, lat, i, fstar[lat.opp[i]], rho0_b, u_b, rho_b, P)
    if mask is None:
        return fs
    g = m[None] * fs
    out = np.empty_like(f)
    out[0] = fs[0]
    for i in range(1, lat.Q):
        out[i] = fs[i] - g[i] + shift(g[lat.opp[i]], lat.c[i], periodic)
    return out


def velocity_out(lat, f, force=(0.0, 0.0, 0.0), mask=None, rho_min=0.5):
    """Reported velocity u = (j + F (1 - m_O) / 2) / rho where rho > rho_min,
    zero elsewhere (solid cells hold no fluid)."""
    F = np.asarray(force, dtype=np.float64)
    m = np.zeros(f.shape[1:]) if mask is None else np.asarray(mask, dtype=np.float64)
    rho, j = moments(lat, f)
    jj = j + 0.5 * F[:, None, None, None] * (1.0 - m)[None]
    safe = np.where(rho > rho_min, rho, 1.0)
    return rho, np.where(rho[None] > rho_min, jj / safe[None], 0.0)


def initial_rest(lat, N, mask=None):
    """f_i = w_i (1 - m_O): unit density, zero velocity, empty solids."""
    m = np.zeros((N, N, N)) if mask is None else np.asarray(mask, dtype=np.float64)
    return lat.w[:, None, None, None] * (1.0 - m)[None]
