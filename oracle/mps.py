"""MPS (tensor-train) algebra in float64, Sec. 2.1-2.3.

An MPS is a list of L cores, core k of shape (r_k, 2, r_{k+1}) with
r_0 = r_L = 1 (Eq. MPS with binary physical indices).

Functions and what they follow
  to_tensor        contraction of all cores (Eq. MPS)
  entry            one entry of that contraction (Eq. MPS at fixed indices)
  tt_svd           left-to-right SVD construction with truncation (Eq. svd-comp)
  round_mps        left-orthogonalising QR sweep, then a right-to-left truncated
                   SVD sweep that truncates only at the canonical centre
                   (Eq. lorg, Eq. svd-move; Sec. 3.2 "an iteration of SVD")
  add, lincomb     block-diagonal cores (Eq. add)
  hadamard_exact   per-site Kronecker product via the delta tensor (Eq. mul)
  apply_mpo        site-wise MPO x MPS contraction (Eq. applympo)
  inner_ones       contraction with the rank-1 all-ones MPS (Sec. 3.2, rho_0)
  hadamard_fit     compressed product by single-site variational fit (Sec. 2.3)
  zipup_pass,      compressed product by one left-to-right zip-up pass, then
  hadamard_zipup   a rounding (the alternative to the fit that Sec. 2.3 names)

Truncation rule (the paper fixes only chi): at each bond keep the smallest
r <= chi_max with sqrt(sum_{j>=r} s_j^2) <= eps * ||T|| / sqrt(L-1), r >= 1.

Pinned by tests/test_oracle_mps.py: dense elementwise identities for add,
product and MPO application; Eckart-Young and the eps bound for rounding;
orthogonality (Eq. lorg); exactness and monotone error decrease of the fit.
"""

import numpy as np


# ---------------------------------------------------------------- basics

def ones(L):
    return [np.ones((1, 2, 1)) for _ in range(L)]


def rank1(vectors):
    """Rank-1 MPS from per-site 2-vectors."""
    return [np.asarray(v, dtype=np.float64).reshape(1, 2, 1) for v in vectors]


def ranks(cores):
    return [1] + [c.shape[2] for c in cores]


def copy(cores):
    return [c.copy() for c in cores]


def scale(cores, c):
    out = copy(cores)
    out[0] = out[0] * c
    return out


def to_tensor(cores):
    """Contract all cores (Eq. MPS) into a tensor of shape (2,)*L."""
    t = cores[0].reshape(2, cores[0].shape[2])
    for c in cores[1:]:
        t = np.tensordot(t, c, axes=(t.ndim - 1, 0))
    return t.reshape((2,) * len(cores))


def entry(cores, bits):
    """One entry T[bits_0, ..., bits_{L-1}] of Eq. MPS: the product of the
    per-site matrices A_k[:, bits_k, :] (a 1 x 1 result)."""
    v = np.ones((1,))
    for c, b in zip(cores, bits):
        v = v @ c[:, int(b), :]
    return float(v[0])


def norm(cores):
    return float(np.sqrt(np.sum(to_tensor(cores) ** 2)))


# ---------------------------------------------------------------- factorizations

def qr_pos(M):
    """Reduced QR with non-negative diagonal of R (deterministic gauge)."""
    Q, R = np.linalg.qr(M, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :], R * s[:, None]


def choose_rank(s, chi_max, delta):
    """Smallest r in [1, min(chi_max, len(s))] whose discarded tail
    sqrt(sum_{j>=r} s_j^2) is <= delta; otherwise min(chi_max, len(s))."""
    n = len(s)
    rmax = min(chi_max, n)
    tail2 = 0.0
    tails = np.zeros(n + 1)
    for j in range(n - 1, -1, -1):       # accumulate from the smallest value up
        tail2 += s[j] * s[j]
        tails[j] = tail2
    for r in range(1, rmax + 1):
        if np.sqrt(tails[r]) <= delta:
            return r
    return rmax


def tt_svd(T, chi_max, eps):
    """Eq. (svd-comp): reshape, SVD, keep U as the core, carry S V^T on."""
    T = np.asarray(T, dtype=np.float64)
    L = T.ndim
    nrm = np.sqrt(np.sum(T * T))
    delta = eps * nrm / np.sqrt(max(L - 1, 1))
    cores = []
    r = 1
    M = T.reshape(1, -1)
    for k in range(L - 1):
        M = M.reshape(r * 2, -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        rk = choose_rank(S, chi_max, delta)
        cores.append(U[:, :rk].reshape(r, 2, rk))
        M = S[:rk, None] * Vt[:rk]
        r = rk
    cores.append(M.reshape(r, 2, 1))
    return cores


def left_orthogonalize(cores):
    """QR sweep k = 0..L-2; afterwards cores 0..L-2 satisfy Eq. (lorg) and the
    last core is the canonical centre."""
    A = copy(cores)
    L = len(A)
    for k in range(L - 1):
        r0, d, r1 = A[k].shape
        Q, R = qr_pos(A[k].reshape(r0 * d, r1))
        A[k] = Q.reshape(r0, d, Q.shape[1])
        A[k + 1] = np.tensordot(R, A[k + 1], axes=(1, 0))
    return A


def round_mps(cores, chi_max, eps):
    """TT-rounding: QR sweep to put the centre at the last site, then move the
    centre back to site 0 with truncated SVDs (Eq. svd-move), truncating only
    at the centre (Sec. 2.1)."""
    L = len(cores)
    A = left_orthogonalize(cores)
    if L == 1:
        return A
    nrm = float(np.sqrt(np.sum(A[L - 1] ** 2)))
    delta = eps * nrm / np.sqrt(L - 1)
    for k in range(L - 1, 0, -1):
        r0, d, r1 = A[k].shape
        U, S, Vt = np.linalg.svd(A[k].reshape(r0, d * r1), full_matrices=False)
        rk = choose_rank(S, chi_max, delta)
        A[k] = Vt[:rk].reshape(rk, d, r1)
        A[k - 1] = np.tensordot(A[k - 1], U[:, :rk] * S[None, :rk], axes=(2, 0))
    return A


# ---------------------------------------------------------------- algebra

def add(A, B):
    """Eq. (add): block-diagonal cores; first core concatenated along the right
    bond, last core along the left bond."""
    return lincomb([(1.0, A), (1.0, B)])


def lincomb(terms):
    """sum_t c_t X_t by Eq. (add) applied to all terms at once (block diagonal
    cores, coefficient folded into the first core).  No truncation."""
    L = len(terms[0][1])
    out = []
    for k in range(L):
        blocks = [X[k] * (c if k == 0 else 1.0) for c, X in terms]
        rl = sum(b.shape[0] for b in blocks) if k > 0 else 1
        rr = sum(b.shape[2] for b in blocks) if k < L - 1 else 1
        core = np.zeros((rl, 2, rr))
        ol = orr = 0
        for b in blocks:
            if k == 0:
                core[:, :, orr:orr + b.shape[2]] = b
            elif k == L - 1:
                core[ol:ol + b.shape[0], :, :] = b
            else:
                core[ol:ol + b.shape[0], :, orr:orr + b.shape[2]] = b
            ol += b.shape[0]
            orr += b.shape[2]
        out.append(core)
    return out


def lincomb_round(terms, chi_max, eps):
    return round_mps(lincomb(terms), chi_max, eps)


def hadamard_exact(A, B):
    """Eq. (mul): core (A*B)_k[(a b), s, (a' b')] = A_k[a,s,a'] B_k[b,s,b']."""
    out = []
    for a, b in zip(A, B):
        c = np.einsum("isj,ksl->iksjl", a, b)
        out.append(c.reshape(a.shape[0] * b.shape[0], 2, a.shape[2] * b.shape[2]))
    return out


def mask_rank1(A, vectors):
    """Exact product of A with a rank-1 MPS given by per-site 2-vectors."""
    return [a * np.asarray(v, dtype=np.float64)[None, :, None] for a, v in zip(A, vectors)]


def apply_mpo(O, A):
    """Eq. (applympo): O_k has shape (w_k, 2_out, 2_in, w_{k+1});
    (OA)_k[(w a), s', (w' a')] = sum_s O_k[w, s', s, w'] A_k[a, s, a']."""
    out = []
    for o, a in zip(O, A):
        c = np.einsum("wtsv,asb->watvb", o, a)
        out.append(c.reshape(o.shape[0] * a.shape[0], o.shape[1], o.shape[3] * a.shape[2]))
    return out


def inner_ones(A):
    """<A, 1>: sum of all entries, by a transfer-vector sweep (Sec. 3.2)."""
    v = np.ones(1)
    for c in A:
        v = v @ c.sum(axis=1)
    return float(v[0])


# ---------------------------------------------------------------- Sec. 2.3

# Each contraction below is the plain sum written in three pairwise steps (the
# physical index s is shared by three tensors, so a single einsum call would
# not split it and would cost chi^6 instead of chi^4).

def _env_left(EL, A, B, C):
    # EL'[x,y,z] = sum_{a,b,g,s} EL[a,b,g] A[a,s,x] B[b,s,y] C[g,s,z]
    t = np.einsum("abg,asx->bgsx", EL, A, optimize=True)
    t = np.einsum("bgsx,bsy->gsxy", t, B, optimize=True)
    return np.einsum("gsxy,gsz->xyz", t, C, optimize=True)


def _env_right(ER, A, B, C):
    # ER'[a,b,g] = sum_{s,x,y,z} A[a,s,x] B[b,s,y] C[g,s,z] ER[x,y,z]
    t = np.einsum("gsz,xyz->gsxy", C, ER, optimize=True)
    t = np.einsum("bsy,gsxy->bgsx", B, t, optimize=True)
    return np.einsum("asx,bgsx->abg", A, t, optimize=True)


def _local(EL, B, C, ER):
    # optimal centre: A_c[a,s,x] = sum EL[a,b,g] B[b,s,y] C[g,s,z] ER[x,y,z]
    t = np.einsum("abg,bsy->agsy", EL, B, optimize=True)
    t = np.einsum("agsy,gsz->asyz", t, C, optimize=True)
    return np.einsum("asyz,xyz->asx", t, ER, optimize=True)


def right_orthogonalize(cores):
    """LQ sweep k = L-1..1 (QR of the transposed unfolding): cores 1..L-1 get
    orthonormal rows, the centre ends at site 0."""
    A = copy(cores)
    for k in range(len(A) - 1, 0, -1):
        r0, d, r1 = A[k].shape
        Q, R = qr_pos(A[k].reshape(r0, d * r1).T)
        A[k] = Q.T.reshape(Q.shape[1], d, r1)
        A[k - 1] = np.tensordot(A[k - 1], R.T, axes=(2, 0))
    return A


def hadamard_fit(B, C, sweeps=2, record=None):
    """Compressed product A ~ B*C by the single-site variational fit of
    Sec. 2.3 (Fig. multiplication).

    Candidate A = copy of B, bond dimensions unchanged.  A is brought to
    canonical form with its centre at site 0; right environments are built;
    then `sweeps` round trips c = 0 -> L-1 -> 0.  At each centre the optimal
    core is the contraction of the left environment, the two factor cores and
    the right environment (the local minimiser of ||A - B*C||^2); the centre
    is moved on by QR (rightwards) or LQ (leftwards).  If `record` is a list,
    the squared error ||A - B*C||^2 after every local update is appended
    (a check of the monotone decrease; it contracts densely, tiny L only).
    """
    L = len(B)
    A = right_orthogonalize(B)
    one = np.ones((1, 1, 1))
    EL = [None] * (L + 1)
    ER = [None] * (L + 1)
    EL[0] = one
    ER[L] = one
    for k in range(L - 1, 0, -1):
        ER[k] = _env_right(ER[k + 1], A[k], B[k], C[k])
    target = None
    if record is not None:
        target = to_tensor(B) * to_tensor(C)

    def _rec():
        if record is not None:
            record.append(float(np.sum((to_tensor(A) - target) ** 2)))

    for _ in range(sweeps):
        for c in range(L):                         # left to right
            A[c] = _local(EL[c], B[c], C[c], ER[c + 1])
            _rec()
            if c < L - 1:
                r0, d, r1 = A[c].shape
                Q, R = qr_pos(A[c].reshape(r0 * d, r1))
                A[c] = Q.reshape(r0, d, Q.shape[1])
                A[c + 1] = np.tensordot(R, A[c + 1], axes=(1, 0))
                EL[c + 1] = _env_left(EL[c], A[c], B[c], C[c])
        for c in range(L - 1, -1, -1):             # right to left
            A[c] = _local(EL[c], B[c], C[c], ER[c + 1])
            _rec()
            if c > 0:
                r0, d, r1 = A[c].shape
                Q, R = qr_pos(A[c].reshape(r0, d * r1).T)
                A[c] = Q.T.reshape(Q.shape[1], d, r1)
                A[c - 1] = np.tensordot(A[c - 1], R.T, axes=(2, 0))
                ER[c] = _env_right(ER[c + 1], A[c], B[c], C[c])
    return A


def zipup_pass(B, C, chi_max, eps):
    """One left-to-right zip-up pass over the element-wise product B * C (the
    alternative to the fit named in Sec. 2.3).  A matrix M carries the product
    bond (b, c) of the sites done so far to the new bond a.  At site k the
    product core is contracted into it,
        T[a, s, c', b'] = sum_{b, c} M[a, c, b] B_k[b, s, b'] C_k[c, s, c'],
    T is unfolded as (a s) x (c' b') and factorised by a truncated SVD: U (rank
    r) is the new core, M = S_r V_r^T is carried on.  The last site keeps T.
    Truncation: choose_rank with delta = eps ||T_0|| / sqrt(L-1), T_0 the
    first site's unfolding.  The result is left-orthogonal up to its last
    core.  With C the all-ones MPS (rank 1, cores [1, 1]) this is the
    left-to-right truncated SVD sweep of B (Eq. svd-move run rightwards)."""
    L = len(B)
    M = np.ones((1, 1, 1))
    delta = None
    out = []
    for k in range(L):
        X = np.einsum("acb,bsy->acsy", M, B[k], optimize=True)
        T = np.einsum("acsy,csz->aszy", X, C[k], optimize=True)
        a, _, z, y = T.shape
        Tm = T.reshape(a * 2, z * y)
        if delta is None:
            delta = eps * float(np.sqrt(np.sum(Tm * Tm))) / np.sqrt(max(L - 1, 1))
        if k == L - 1:
            out.append(Tm.reshape(a, 2, 1))
            break
        U, S, Vt = np.linalg.svd(Tm, full_matrices=False)
        r = choose_rank(S, chi_max, delta)
        out.append(U[:, :r].reshape(a, 2, r))
        M = (S[:r, None] * Vt[:r]).reshape(r, z, y)
    return out


def hadamard_zipup(B, C, chi_max, eps):
    """Compressed product by the zip-up pass.  Both factors are first brought
    to right-canonical form (right_orthogonalize: the truncation at each site
    then sees orthonormal rows of each factor's remaining sites; without it
    the pass can lose most of the product), then the pass, then a rounding
    of its result (round_mps: the QR sweep finds the pass's cores already
    left-orthogonal; the right-to-left SVD sweep truncates at the centre and
    leaves the centre at site 0, as the fit and every rounding do)."""
    Z = zipup_pass(right_orthogonalize(B), right_orthogonalize(C), chi_max, eps)
    return round_mps(Z, chi_max, eps)
