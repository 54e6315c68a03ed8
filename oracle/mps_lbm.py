"""The MPS-LBM time step, Sec. 3.2, written plainly on top of oracle.mps.

Every population f_i is an MPS on L = 3n binary sites (Sec. 2.4).  One step:

 a1 moments      rho = sum_i f_i, j_d = sum_i c_id f_i          (Eq. macro)
                 as balanced pairwise trees, each pair added (Eq. add) and
                 rounded (Sec. 3.2: sums are re-compressed after each addition)
 a2 mean density rho_0 = <rho, 1> / N_fluid, N_fluid = N^3 - <m_O, 1>
 a3 Taylor 1/rho drho = rho - rho_0 1;  s = drho * drho;
                 inv = (1/rho_0) 1 - drho / rho_0^2 + s / rho_0^3   (Sec. 3.2)
 a4 velocity     J~_d = j_d + tau F_d (1 - m_O);  u_d = J~_d * inv  (App. A)
 a5 products     P_de = J~_d * u_e, d <= e
 a6 collision    f*_i = (1 - 1/tau) f_i + (1/tau) w_i E_i with
                 E_i = rho + 3 c_i.J~ + sum_{d<=e} kappa_de P_de     (Eqs. collision,
                 equilibrium); kappa_dd = 4.5 c_d^2 - 1.5, kappa_de = 9 c_d c_e
 a7 streaming    f_i <- (x)_d S_d(c_id) f*_i, one axis at a time (x, y, z), each
                 shift an exact MPO (Sec. 2.5) followed by a rounding; on wall axes
                 the non-cyclic shift is used and the last rounding also adds the
                 halfway bounce-back term m_B,i * f*_opp(i)     (Eq. boundaries2),
                 or, with per-face boundary functions (cfg.faces), the terms
                 m_eff * b of boundary_terms
 a8 objects      g_i = f_i * m_O;  f_i <- (f_i - g_i) + S(c_i) g_opp(i)  (Eq. objects),
                 two rounded pairwise sums
 a9 rounding     every sum above is rounded with oracle.mps.round_mps

Products "*" use the single-site fit of Sec. 2.3 with the first factor as the
candidate (hadamard='fit'), the exact Kronecker product of Eq. (mul) followed
by a rounding (hadamard='exact'), or the zip-up pass followed by a rounding
(hadamard='zipup', oracle.mps.hadamard_zipup).

Order of the linear combinations in a6 (the paper does not fix it): shared
partial sums are formed once and reused.
  E0 = ((rho - 1.5 Pxx) - 1.5 Pyy) - 1.5 Pzz
  Q_key: E0 plus the second-order terms of c_i, diagonal ones first (xx, yy, zz),
         then xy, xz, yz; every prefix of such a list is one rounded sum, shared
         by all velocities that have it.
  V_key: sum_d 3 c_id J~_d with the sign normalised so that the first
         coefficient is positive (prefixes shared likewise; a single term is
         just a scaled MPS, no rounding).
  Y_i  = round(Q_i + sigma_i V_i),  f*_i = round((1 - w) f_i + w w_i Y_i).

Parity: pinned through its parts (oracle.mps, oracle.mpo) and by reproducing
oracle.lbm_dense in taylor mode to round-off when nothing is truncated
(tests/test_oracle_mps_lbm.py).
"""

import numpy as np

from . import mps as M
from .mpo import shift_mpo
from .quantics import decode
from .lbm_dense import (second_order_coeffs, velocity_out, face_index, FACE_WALL, FACE_VELOCITY,
                        FACE_PRESSURE)
from .lattice import CS2


class Config:
    def __init__(self, n_bits, lattice, tau, force=(0.0, 0.0, 0.0), periodic=(1, 1, 1),
                 chi_max=16, eps=1e-10, hadamard="fit", sweeps=2, mask=None, faces=None,
                 block_sums=False):
        self.n = n_bits
        self.L = 3 * n_bits
        self.N = 1 << n_bits
        self.lat = lattice
        self.tau = float(tau)
        self.force = tuple(float(x) for x in force)
        self.periodic = tuple(int(p) for p in periodic)
        self.chi = int(chi_max)
        self.eps = float(eps)
        self.hadamard = hadamard
        self.sweeps = int(sweeps)
        self.mask = mask                       # MPS cores of m_O or None
        # None, or six (kind, u_b, rho_b) for the faces x-, x+, y-, y+, z-, z+
        self.faces = faces
        # moments as one rounded block sum of all populations instead of the
        # pairwise tree (the alternative linear fold)
        self.block_sums = bool(block_sums)
        self.n_fluid = float(self.N ** 3) - (M.inner_ones(mask) if mask is not None else 0.0)


# ---------------------------------------------------------------- helpers

def _R(cfg, terms):
    return M.lincomb_round(terms, cfg.chi, cfg.eps)


def _had(cfg, B, C):
    if cfg.hadamard == "fit":
        return M.hadamard_fit(B, C, sweeps=cfg.sweeps)
    if cfg.hadamard == "zipup":
        return M.hadamard_zipup(B, C, cfg.chi, cfg.eps)
    return M.round_mps(M.hadamard_exact(B, C), cfg.chi, cfg.eps)


def tree_sum(cfg, items):
    """Balanced pairwise reduction of [(coef, MPS), ...]; each pair is one
    rounded two-term sum, an odd last item moves up unchanged.  With
    cfg.block_sums: one rounding of the whole block sum (Eq. add over all
    terms, then the rounding sweep once)."""
    items = list(items)
    if cfg.block_sums and len(items) > 1:
        return _R(cfg, items)
    while len(items) > 1:
        nxt = []
        for p in range(0, len(items) - 1, 2):
            nxt.append((1.0, _R(cfg, [items[p], items[p + 1]])))
        if len(items) % 2 == 1:
            nxt.append(items[-1])
        items = nxt
    c, X = items[0]
    return X if c == 1.0 else M.scale(X, c)


def plane_vectors(n_bits, axis, value_bit):
    """Rank-1 indicator of the plane x_axis = 0 (value_bit 0) or N-1 (1)."""
    vecs = []
    for k in range(3 * n_bits):
        if k % 3 == axis:
            vecs.append((1.0, 0.0) if value_bit == 0 else (0.0, 1.0))
        else:
            vecs.append((1.0, 1.0))
    return vecs


def wall_terms(n_bits, c, periodic):
    """m_B for velocity c as a signed sum of rank-1 plane products
    (inclusion-exclusion over the wall axes that c crosses)."""
    W = [d for d in range(3) if c[d] != 0 and not periodic[d]]
    out = []
    for bits in range(1, 1 << len(W)):
        S = [W[t] for t in range(len(W)) if bits >> t & 1]
        coef = 1.0 if len(S) % 2 == 1 else -1.0
        vecs = [(1.0, 1.0)] * (3 * n_bits)
        for d in S:
            pv = plane_vectors(n_bits, d, 0 if c[d] > 0 else 1)
            vecs = [(a[0] * b[0], a[1] * b[1]) for a, b in zip(vecs, pv)]
        out.append((coef, vecs))
    return out


def face_terms(n_bits, c, periodic):
    """[(face, [(sign, vecs)])]: the cells entered through a wall face by
    velocity c, each assigned to the crossed face of lowest axis (as in
    oracle.lbm_dense.face_masks), as signed rank-1 plane products
    m_eff(d) = plane_d prod_{d' < d} (1 - plane_d') expanded."""
    W = [d for d in range(3) if c[d] != 0 and not periodic[d]]
    out = []
    for t, d in enumerate(W):
        lower = W[:t]
        terms = []
        for bits in range(1 << len(lower)):
            S = [lower[q] for q in range(len(lower)) if bits >> q & 1]
            vecs = plane_vectors(n_bits, d, 0 if c[d] > 0 else 1)
            for d2 in S:
                pv = plane_vectors(n_bits, d2, 0 if c[d2] > 0 else 1)
                vecs = [(a[0] * b[0], a[1] * b[1]) for a, b in zip(vecs, pv)]
            terms.append((-1.0 if len(S) % 2 else 1.0, vecs))
        out.append((face_index(d, c[d]), terms))
    return out


def boundary_terms(cfg, i, fstar_opp, one, rho0, P):
    """The (coef, MPS) terms m_eff * b of Eq. (boundaries2) for population i
    with the per-face boundary functions of oracle.lbm_dense.face_value."""
    lat = cfg.lat
    c = lat.c[i]
    w = lat.w[i]
    out = []
    for face, terms in face_terms(cfg.n, c, cfg.periodic):
        kind, u_b, rho_b = cfg.faces[face]
        for sgn, vecs in terms:
            if kind == FACE_WALL:
                out.append((sgn, M.mask_rank1(fstar_opp, vecs)))
            elif kind == FACE_VELOCITY:
                out.append((sgn, M.mask_rank1(fstar_opp, vecs)))
                cu = float(c.astype(np.float64) @ np.asarray(u_b, dtype=np.float64))
                if cu != 0.0:
                    out.append((sgn * 2.0 * w * rho0 * cu / CS2, M.mask_rank1(one, vecs)))
            elif kind == FACE_PRESSURE:
                out.append((-sgn, M.mask_rank1(fstar_opp, vecs)))
                out.append((sgn * 2.0 * w * rho_b, M.mask_rank1(one, vecs)))
                for de, kap in second_order_coeffs(c).items():
                    if kap != 0.0:
                        out.append((sgn * 2.0 * w * rho_b * kap / rho0, M.mask_rank1(P[de], vecs)))
            else:
                raise ValueError(kind)
    return out


def _shift(cfg, X, d, cd):
    """Exact MPO application of (S g)(x) = g(x - cd e_d) (Sec. 2.5)."""
    return M.apply_mpo(shift_mpo(cfg.n, d, -int(cd), bool(cfg.periodic[d])), X)


def fourier_mode_mps(n_bits, k, phase):
    """Exact rank-2 MPS of cos(2 pi k.x / N + phase): each site multiplies the
    running (cos, sin) pair by the rotation of its bit's phase."""
    N = 1 << n_bits
    L = 3 * n_bits
    cores = []
    for s in range(L):
        a, lev = s % 3, s // 3
        core = np.zeros((2, 2, 2))
        for b in range(2):
            th = 2.0 * np.pi * k[a] * (1 << (n_bits - 1 - lev)) * b / N
            core[:, b, :] = [[np.cos(th), np.sin(th)], [-np.sin(th), np.cos(th)]]
        cores.append(core)
    cores[0] = np.einsum("a,asb->sb", np.array([np.cos(phase), np.sin(phase)]), cores[0])[None]
    cores[-1] = cores[-1][:, :, 0:1]
    return cores


# ---------------------------------------------------------------- states

def initial_rest(cfg):
    """f_i = w_i (1 - m_O)."""
    one = M.ones(cfg.L)
    out = []
    for i in range(cfg.lat.Q):
        w = cfg.lat.w[i]
        if cfg.mask is None:
            out.append(_R(cfg, [(w, one)]))
        else:
            out.append(_R(cfg, [(w, one), (-w, cfg.mask)]))
    return out


def initial_perturbed(cfg, modes):
    """f_i = w_i (1 + sum_m (a_rho,m + 3 c_i.a_u,m) cos(2 pi k_m.x/N + phase_m)),
    the linearised equilibrium of smooth density and velocity perturbations,
    rounded once.  `modes` rows: kx, ky, kz, phase, a_rho, a_ux, a_uy, a_uz."""
    one = M.ones(cfg.L)
    mode_mps = [fourier_mode_mps(cfg.n, row[0:3], row[3]) for row in modes]
    out = []
    for i in range(cfg.lat.Q):
        w = cfg.lat.w[i]
        c = cfg.lat.c[i].astype(np.float64)
        terms = [(w, one)]
        for row, X in zip(modes, mode_mps):
            terms.append((w * (row[4] + 3.0 * float(c @ row[5:8])), X))
        out.append(_R(cfg, terms))
    return out


# ---------------------------------------------------------------- the step

def step(cfg, f):
    lat, tau = cfg.lat, cfg.tau
    omega = 1.0 / tau
    Q = lat.Q
    one = M.ones(cfg.L)
    # a1
    rho = tree_sum(cfg, [(1.0, f[i]) for i in range(Q)])
    j = [tree_sum(cfg, [(float(lat.c[i, d]), f[i]) for i in range(Q) if lat.c[i, d] != 0])
         for d in range(3)]
    # a2
    rho0 = M.inner_ones(rho) / cfg.n_fluid
    # a3
    drho = _R(cfg, [(1.0, rho), (-rho0, one)])
    s = _had(cfg, drho, drho)
    inv = _R(cfg, [(1.0 / rho0, one), (-1.0 / rho0 ** 2, drho), (1.0 / rho0 ** 3, s)])
    # a4
    Jt = []
    for d in range(3):
        Fd = cfg.force[d]
        if Fd == 0.0:
            Jt.append(j[d])
        else:
            terms = [(1.0, j[d]), (tau * Fd, one)]
            if cfg.mask is not None:
                terms.append((-tau * Fd, cfg.mask))
            Jt.append(_R(cfg, terms))
    u = [_had(cfg, Jt[d], inv) for d in range(3)]
    # a5
    P = {}
    for d in range(3):
        for e in range(d, 3):
            P[(d, e)] = _had(cfg, Jt[d], u[e])
    # a6
    E0 = rho
    for d in range(3):
        E0 = _R(cfg, [(1.0, E0), (-1.5, P[(d, d)])])
    qcache = {(): E0}

    def qchain(key):
        if key not in qcache:
            prev = qchain(key[:-1])
            de, kap = key[-1]
            qcache[key] = _R(cfg, [(1.0, prev), (kap, P[de])])
        return qcache[key]

    vcache = {}

    def vchain(key):
        # returns (coef, MPS) representing sum of the keyed first-order terms
        if len(key) == 1:
            d, a = key[0]
            return (a, Jt[d])
        if key not in vcache:
            pc, pX = vchain(key[:-1])
            d, a = key[-1]
            vcache[key] = _R(cfg, [(pc, pX), (a, Jt[d])])
        return (1.0, vcache[key])

    fstar = []
    for i in range(Q):
        c = lat.c[i]
        kap = second_order_coeffs(c)
        qkey = []
        for d in range(3):
            if c[d] != 0:
                qkey.append(((d, d), kap[(d, d)] + 1.5))
        for (d, e) in ((0, 1), (0, 2), (1, 2)):
            if c[d] != 0 and c[e] != 0:
                qkey.append(((d, e), kap[(d, e)]))
        Qi = qchain(tuple(qkey))
        first = [(d, 3.0 * float(c[d])) for d in range(3) if c[d] != 0]
        if first:
            sigma = 1.0 if first[0][1] > 0 else -1.0
            vkey = tuple((d, sigma * a) for d, a in first)
            vc, vX = vchain(vkey)
            Y = _R(cfg, [(1.0, Qi), (sigma * vc, vX)])
        else:
            Y = Qi
        fstar.append(_R(cfg, [(1.0 - omega, f[i]), (omega * lat.w[i], Y)]))
    # a7
    fs = []
    for i in range(Q):
        c = lat.c[i]
        axes = [d for d in range(3) if c[d] != 0]
        x = fstar[i]
        walls = wall_terms(cfg.n, c, cfg.periodic)
        for t, d in enumerate(axes):
            terms = [(1.0, _shift(cfg, x, d, c[d]))]
            if t == len(axes) - 1:
                if cfg.faces is None:
                    for coef, vecs in walls:
                        terms.append((coef, M.mask_rank1(fstar[lat.opp[i]], vecs)))
                else:
                    terms += boundary_terms(cfg, i, fstar[lat.opp[i]], one, rho0, P)
            x = _R(cfg, terms)
        fs.append(x)
    if cfg.mask is None:
        return fs
    # a8
    g = [None] + [_had(cfg, fs[i], cfg.mask) for i in range(1, Q)]
    out = [fs[0]]
    for i in range(1, Q):
        c = lat.c[i]
        h = g[lat.opp[i]]
        for d in range(3):
            if c[d] != 0:
                h = _R(cfg, [(1.0, _shift(cfg, h, d, c[d]))])
        t = _R(cfg, [(1.0, fs[i]), (-1.0, g[i])])
        out.append(_R(cfg, [(1.0, t), (1.0, h)]))
    return out


# ---------------------------------------------------------------- outputs

def to_dense_populations(f):
    return np.stack([decode(M.to_tensor(x)) for x in f])


def macroscopic(cfg, f, mask_dense=None):
    """rho and the reported velocity (j + F (1 - m_O)/2)/rho from the contracted
    populations; mask_dense defaults to the contraction of cfg.mask."""
    fd = to_dense_populations(f)
    if mask_dense is None and cfg.mask is not None:
        mask_dense = decode(M.to_tensor(cfg.mask))
    return velocity_out(cfg.lat, fd, cfg.force, mask_dense)
