"""Python-side marshalling for libtnlbm: device MPS buffers (torch tensors in the
flat layout of include/tnlbm.h), the simulation handle, and the batched
primitives.  No arithmetic of the method happens here."""
import ctypes
import json
import os

import numpy as np
import torch

from . import native as nat

_DT = {nat.FP64: torch.float64, nat.FP32: torch.float32, nat.TF32: torch.float32, nat.MIXED: torch.float32,
       nat.BF16: torch.float32}


def mps_size(L, cap):
    return int(nat.lib().tnlbm_mps_size(L, cap))


def mps_offset(L, cap, k):
    return int(nat.lib().tnlbm_mps_offset(L, cap, k))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptrs(items):
    arr = (ctypes.c_void_p * len(items))()
    for i, t in enumerate(items):
        arr[i] = t.data_ptr()
    return arr


class DeviceMps:
    """One MPS in device memory: `data` holds the flat layout with capacity
    `cap`, `ranks` the realised bonds r[0..L] (int32)."""

    def __init__(self, L, cap, precision=nat.FP64, device="cuda"):
        self.L, self.cap, self.precision = L, cap, precision
        self.data = torch.zeros(mps_size(L, cap), dtype=_DT[precision], device=device)
        self.ranks = torch.ones(L + 1, dtype=torch.int32, device=device)

    @classmethod
    def from_cores(cls, cores, cap=None, precision=nat.FP64, device="cuda"):
        L = len(cores)
        r = [1] + [c.shape[2] for c in cores]
        cap = cap or max(r)
        m = cls(L, cap, precision, device)
        flat = np.zeros(mps_size(L, cap))
        for k, c in enumerate(cores):
            o = mps_offset(L, cap, k)
            flat[o:o + c.size] = np.asarray(c, dtype=np.float64).reshape(-1)
        m.data.copy_(torch.from_numpy(flat).to(_DT[precision]))
        m.ranks.copy_(torch.tensor(r, dtype=torch.int32))
        return m

    def cores(self):
        flat = self.data.double().cpu().numpy()
        r = self.ranks.cpu().numpy().tolist()
        out = []
        for k in range(self.L):
            o = mps_offset(self.L, self.cap, k)
            out.append(flat[o:o + r[k] * 2 * r[k + 1]].reshape(r[k], 2, r[k + 1]).copy())
        return out

    def bonds(self):
        return self.ranks.cpu().numpy().tolist()


def _term(kind, coef=1.0, x=None, y=None, axis=0, offset=1, cyclic=1, mask=None):
    t = nat.Term()
    t.kind = kind
    t.coef = coef
    if x is not None:
        t.x, t.x_ranks, t.x_cap = x.data.data_ptr(), x.ranks.data_ptr(), x.cap
    if y is not None:
        t.y, t.y_ranks, t.y_cap = y.data.data_ptr(), y.ranks.data_ptr(), y.cap
    t.axis, t.offset, t.cyclic = axis, offset, cyclic
    keep = None
    if mask is not None:
        keep = np.ascontiguousarray(mask, dtype=np.float64).reshape(-1)
        t.mask = keep.ctypes.data_as(nat.c_double_p)
    return t, keep


def plain(x, coef=1.0):
    return dict(kind=nat.TERM_PLAIN, coef=coef, x=x)


def ones(coef=1.0):
    return dict(kind=nat.TERM_ONES, coef=coef)


def shift(x, axis, offset, cyclic=True, coef=1.0):
    return dict(kind=nat.TERM_SHIFT, coef=coef, x=x, axis=axis, offset=offset, cyclic=int(cyclic))


def mask1(x, vectors, coef=1.0):
    return dict(kind=nat.TERM_MASK1, coef=coef, x=x, mask=vectors)


def kron(x, y, coef=1.0):
    return dict(kind=nat.TERM_KRON, coef=coef, x=x, y=y)


def _terms_array(batches):
    nterms = len(batches[0])
    arr = (nat.Term * (len(batches) * nterms))()
    keep = []
    for b, terms in enumerate(batches):
        assert len(terms) == nterms
        for t, spec in enumerate(terms):
            tm, k = _term(**spec)
            arr[b * nterms + t] = tm
            keep.append(k)
    return arr, nterms, keep


def lincomb_round(batches, dst, chi_max, eps, stream=None):
    """dst[b] = round(sum of batches[b]) (tnlbm_lincomb_round)."""
    arr, nterms, keep = _terms_array(batches)
    p = dst[0].precision
    rc = nat.lib().tnlbm_lincomb_round(p, dst[0].L // 3, len(dst), nterms, arr,
                                       _ptrs([d.data for d in dst]), _ptrs([d.ranks for d in dst]),
                                       dst[0].cap, chi_max, eps, _stream(stream))
    nat.check(rc, "tnlbm_lincomb_round")


def lincomb_round_noalloc(batches, dst, chi_max, eps, stream=None):
    """As lincomb_round, through the allocation-free entry point
    (tnlbm_lincomb_round_noalloc): for callers that cannot allocate device
    memory at the call; its workspace is the library's fixed static arrays."""
    arr, nterms, keep = _terms_array(batches)
    p = dst[0].precision
    rc = nat.lib().tnlbm_lincomb_round_noalloc(p, dst[0].L // 3, len(dst), nterms, arr,
                                               _ptrs([d.data for d in dst]), _ptrs([d.ranks for d in dst]),
                                               dst[0].cap, chi_max, eps, _stream(stream))
    nat.check(rc, "tnlbm_lincomb_round_noalloc")


def lincomb_round_rsvd(batches, dst, chi_max, eps, targets, omega, oversample=8, power=1, eta=0.2,
                       floor_rel=1e-12, stream=None):
    """lincomb_round with the certified randomized truncation at target ranks
    (tnlbm_lincomb_round_rsvd).  targets: (batch, L + 1) ints, 0 = full SVD;
    omega: device tensor (rows x ld) of the rounding's type.  Returns the
    counts (accepted, fell back, full SVDs)."""
    arr, nterms, keep = _terms_array(batches)
    p = dst[0].precision
    L = dst[0].L
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.int32).reshape(len(dst), L + 1))
    if omega.dtype != (torch.float64 if p == nat.FP64 else torch.float32) or not omega.is_contiguous():
        raise ValueError("omega must be a contiguous tensor of the rounding's type")
    cnt = (ctypes.c_int * 3)()
    rc = nat.lib().tnlbm_lincomb_round_rsvd(p, L // 3, len(dst), nterms, arr,
                                            _ptrs([d.data for d in dst]), _ptrs([d.ranks for d in dst]),
                                            dst[0].cap, chi_max, eps, tg.ctypes.data_as(nat.c_int_p),
                                            ctypes.c_void_p(omega.data_ptr()), omega.shape[0], omega.shape[1],
                                            oversample, power, eta, floor_rel, cnt, _stream(stream))
    nat.check(rc, "tnlbm_lincomb_round_rsvd")
    return tuple(cnt)


# ---------------------------------------------------------------- rank model
MLP_IN = 18
MLP_H = 64


def mlp_param_count():
    return nat.lib().tnlbm_mlp_param_count()


def mlp_flatten(P):
    """Dict of arrays (W1, b1, W2, b2, W3, b3) -> flat float32 vector in the
    library's layout."""
    return np.concatenate([np.asarray(P[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def mlp_unflatten(v):
    v = np.asarray(v, dtype=np.float64)
    shapes = [("W1", (MLP_H, MLP_IN)), ("b1", (MLP_H,)), ("W2", (MLP_H, MLP_H)), ("b2", (MLP_H,)),
              ("W3", (1, MLP_H)), ("b3", (1,))]
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = v[o:o + n].reshape(sh)
        o += n
    return out


def _f32(t):
    if t.dtype != torch.float32 or not t.is_contiguous() or t.device.type != "cuda":
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(params, X, stream=None):
    """Predictions (M,) of the rank model for features X (M x 18); params is the
    flat FP32 device vector."""
    out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
    nat.check(nat.lib().tnlbm_mlp_forward(_f32(params), X.shape[0], _f32(X), _f32(out), _stream(stream)),
              "tnlbm_mlp_forward")
    return out


def mlp_loss_grad(params, X, y, stream=None):
    """(mean squared error, gradient) for the flat FP32 device parameters."""
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    grad = torch.zeros_like(params)
    nat.check(nat.lib().tnlbm_mlp_loss_grad(_f32(params), X.shape[0], _f32(X), _f32(y), _f32(loss),
                                            _f32(grad), _stream(stream)), "tnlbm_mlp_loss_grad")
    return loss, grad


class MlpTrainer:
    """FP32 master parameters with Adam state, trained by tnlbm_mlp_train; the
    FP16 copy (`half`) is what a simulation evaluates."""

    def __init__(self, params):
        self.master = params.detach().clone().contiguous()
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        self.half = self.master.to(torch.float16)
        self.t = 0

    def train(self, X, y, iters, batch=256, lr=1e-3, stream=None):
        hist = torch.zeros(max(iters, 1), dtype=torch.float32, device=X.device)
        rc = nat.lib().tnlbm_mlp_train(_f32(self.master), _f32(self.m), _f32(self.v),
                                       ctypes.c_void_p(self.half.data_ptr()), X.shape[0], _f32(X), _f32(y),
                                       iters, batch, self.t, lr, _f32(hist), _stream(stream))
        nat.check(rc, "tnlbm_mlp_train")
        self.t += iters
        return hist[:iters]


def materialize(terms, dst, stream=None):
    arr, _, keep = _terms_array([[t] for t in terms])
    p = dst[0].precision
    rc = nat.lib().tnlbm_materialize(p, dst[0].L // 3, len(dst), arr, _ptrs([d.data for d in dst]),
                                     _ptrs([d.ranks for d in dst]), dst[0].cap, _stream(stream))
    nat.check(rc, "tnlbm_materialize")


def hadamard_fit(B, C, A, sweeps=2, stream=None):
    p = A[0].precision
    rc = nat.lib().tnlbm_hadamard_fit(p, A[0].L // 3, len(A),
                                      _ptrs([x.data for x in B]), _ptrs([x.ranks for x in B]), B[0].cap,
                                      _ptrs([x.data for x in C]), _ptrs([x.ranks for x in C]), C[0].cap,
                                      _ptrs([x.data for x in A]), _ptrs([x.ranks for x in A]), A[0].cap,
                                      sweeps, _stream(stream))
    nat.check(rc, "tnlbm_hadamard_fit")


def hadamard_zipup(B, C, A, chi_max, eps, stream=None):
    """A[b] ~ B[b] * C[b] by the zip-up pass and a rounding (tnlbm_hadamard_zipup)."""
    p = A[0].precision
    rc = nat.lib().tnlbm_hadamard_zipup(p, A[0].L // 3, len(A),
                                        _ptrs([x.data for x in B]), _ptrs([x.ranks for x in B]), B[0].cap,
                                        _ptrs([x.data for x in C]), _ptrs([x.ranks for x in C]), C[0].cap,
                                        _ptrs([x.data for x in A]), _ptrs([x.ranks for x in A]), A[0].cap,
                                        chi_max, eps, _stream(stream))
    nat.check(rc, "tnlbm_hadamard_zipup")


def inner_ones(X, stream=None):
    out = torch.zeros(len(X), dtype=torch.float64, device=X[0].data.device)
    rc = nat.lib().tnlbm_inner_ones(X[0].precision, X[0].L // 3, len(X), _ptrs([x.data for x in X]),
                                    _ptrs([x.ranks for x in X]), X[0].cap, ctypes.c_void_p(out.data_ptr()),
                                    _stream(stream))
    nat.check(rc, "tnlbm_inner_ones")
    return out


def to_dense(X, stream=None):
    n = X.L // 3
    N = 1 << n
    out = torch.empty((N, N, N), dtype=X.data.dtype, device=X.data.device)
    rc = nat.lib().tnlbm_to_dense(X.precision, n, ctypes.c_void_p(X.data.data_ptr()),
                                  ctypes.c_void_p(X.ranks.data_ptr()), X.cap,
                                  ctypes.c_void_p(out.data_ptr()), _stream(stream))
    nat.check(rc, "tnlbm_to_dense")
    return out


def from_dense(dense, cap, chi_max, eps, stream=None):
    n = int(dense.shape[0]).bit_length() - 1
    p = nat.FP64 if dense.dtype == torch.float64 else nat.FP32
    X = DeviceMps(3 * n, cap, p, dense.device)
    d = dense.contiguous()
    rc = nat.lib().tnlbm_from_dense(p, n, ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(X.data.data_ptr()),
                                    ctypes.c_void_p(X.ranks.data_ptr()), cap, chi_max, eps, _stream(stream))
    nat.check(rc, "tnlbm_from_dense")
    return X


def mask_product(outer, inner, cap, chi_max, eps, stream=None):
    """Combined-scale mask (tnlbm_mask_product): outer and inner are device
    [x][y][z] tensors of the same float type; returns the DeviceMps of the
    inner geometry repeated where the outer mask is one."""
    no = int(outer.shape[0]).bit_length() - 1
    ni = int(inner.shape[0]).bit_length() - 1
    p = nat.FP64 if outer.dtype == torch.float64 else nat.FP32
    if inner.dtype != outer.dtype:
        raise ValueError("outer and inner must have the same type")
    X = DeviceMps(3 * (no + ni), cap, p, outer.device)
    o, i = outer.contiguous(), inner.contiguous()
    rc = nat.lib().tnlbm_mask_product(p, no, ctypes.c_void_p(o.data_ptr()), ni, ctypes.c_void_p(i.data_ptr()),
                                      ctypes.c_void_p(X.data.data_ptr()), ctypes.c_void_p(X.ranks.data_ptr()),
                                      cap, chi_max, eps, _stream(stream))
    nat.check(rc, "tnlbm_mask_product")
    return X


def make_config(n_per_axis, lattice=nat.D3Q19, tau=0.8, periodic=(1, 1, 1), solid=None,
                chi_mask=16, eps_mask=1e-12, mask_cores=None, force=(0.0, 0.0, 0.0), chi_max=16,
                eps=1e-10, precision=nat.FP64, hadamard=nat.HADAMARD_FIT, sweeps=2, modes=None,
                conserve_mass=False, faces=None, block_sums=False, learned_rank=0, seed=0,
                jacobi_max_sweeps=0, wait_limit_ns=0, max_cluster=0):
    """tnlbm_config for the arguments; returns (config, arrays the config
    points to, which must stay alive until the simulation is created).
    faces: None (bounce-back on every wall face) or a dict face -> (kind, u_b,
    rho_b), faces 0..5 = x-, x+, y-, y+, z-, z+, kind nat.FACE_*."""
    c = nat.Config()
    c.n_per_axis = n_per_axis
    c.lattice = lattice
    c.tau = tau
    for d in range(3):
        c.periodic[d] = int(periodic[d])
        c.force[d] = float(force[d])
    keep = []
    if solid is not None:
        sv = np.ascontiguousarray(solid, dtype=np.uint8).reshape(-1)
        keep.append(sv)
        c.solid = sv.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    c.chi_mask = chi_mask
    c.eps_mask = eps_mask
    if mask_cores is not None:
        L = len(mask_cores)
        r = [1] + [x.shape[2] for x in mask_cores]
        cap = max(r)
        flat = np.zeros(mps_size(L, cap))
        for k, x in enumerate(mask_cores):
            o = mps_offset(L, cap, k)
            flat[o:o + x.size] = x.reshape(-1)
        rr = np.array(r, dtype=np.int32)
        keep += [flat, rr]
        c.mask_cores = flat.ctypes.data_as(nat.c_double_p)
        c.mask_ranks = rr.ctypes.data_as(nat.c_int_p)
        c.mask_cap = cap
    c.chi_max = chi_max
    c.eps = eps
    c.precision = precision
    c.hadamard = hadamard
    c.sweeps = sweeps
    c.conserve_mass = int(bool(conserve_mass))
    c.block_sums = int(bool(block_sums))
    c.learned_rank = int(learned_rank)
    c.seed = int(seed)
    c.jacobi_max_sweeps = int(jacobi_max_sweeps)
    c.wait_limit_ns = int(wait_limit_ns)
    c.max_cluster = int(max_cluster)
    for f6, (kind, u_b, rho_b) in (faces or {}).items():
        c.face_kind[f6] = int(kind)
        for d in range(3):
            c.face_u[f6][d] = float(u_b[d])
        c.face_rho[f6] = float(rho_b)
    if modes is not None:
        m = np.ascontiguousarray(modes, dtype=np.float64)
        keep.append(m)
        c.n_modes = m.shape[0]
        c.modes = m.ctypes.data_as(nat.c_double_p)
    return c, keep


def cluster_cache_key(device, configs, jobs):
    """Key of a cluster-size choice in a JSON cache: the device name, each
    simulation's (n_per_axis, lattice, chi_max, precision, max_cluster, fit
    sweeps) and the rounding jobs of every dependency level."""
    sims = [[int(c.n_per_axis), int(c.lattice), int(c.chi_max), int(c.precision), int(c.max_cluster),
             int(c.sweeps)] for c in configs]
    return json.dumps({"device": str(device), "sims": sims, "jobs": [int(j) for j in jobs]}, sort_keys=True)


def load_cluster_cache(path):
    """The {key: sizes} table stored at path ({} if there is none)."""
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return {}
    return d if isinstance(d, dict) else {}


def store_cluster_cache(path, key, sizes):
    """Adds key -> sizes to the table at path (written to a temporary file
    and renamed, so a reader never sees half a file)."""
    d = load_cluster_cache(path)
    d[key] = [int(x) for x in sizes]
    tmp = "%s.%d.tmp" % (path, os.getpid())
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


class _Clusters:
    """Per-level cluster sizes of the rounding launches of a simulation or a
    batch (tnlbm_clusters / tnlbm_set_clusters / tnlbm_tune_clusters)."""
    _fn = ("tnlbm_clusters", "tnlbm_set_clusters", "tnlbm_tune_clusters")

    def clusters(self):
        """(sizes, jobs): per dependency level, the CTAs per rounding job (0
        where the level has no rounding) and the level's rounding jobs."""
        get = getattr(nat.lib(), self._fn[0])
        n = ctypes.c_int()
        nat.check(get(self.h, None, None, 0, ctypes.byref(n)), self._fn[0])
        c = (ctypes.c_int * max(n.value, 1))()
        j = (ctypes.c_int * max(n.value, 1))()
        nat.check(get(self.h, c, j, n.value, ctypes.byref(n)), self._fn[0])
        return list(c)[:n.value], list(j)[:n.value]

    def set_clusters(self, sizes):
        """Sets every level's cluster size (one entry per level) and
        re-captures the step's graph."""
        arr = (ctypes.c_int * max(len(sizes), 1))(*[int(x) for x in sizes])
        nat.check(getattr(nat.lib(), self._fn[1])(self.h, arr, len(sizes)), self._fn[1])

    def tune_clusters(self, reps=2, cache=None):
        """Times each level's rounding launch at the candidate cluster sizes
        and keeps the fastest; the populations and the step count are left as
        they were.  cache: a JSON file; a choice stored there for this device
        and level structure is applied without timing, a new one is stored.
        Returns dict(sizes, jobs, ms: per level {P: ms} or None, cached)."""
        sizes, jobs = self.clusters()
        key = None
        if cache is not None:
            key = cluster_cache_key(torch.cuda.get_device_name(), self._configs(), jobs)
            hit = load_cluster_cache(cache).get(key)
            if hit is not None and len(hit) == len(sizes):
                self.set_clusters(hit)
                return dict(sizes=list(hit), jobs=jobs, ms=None, cached=True)
        stride = nat.CLUSTER_MAX + 1
        buf = (ctypes.c_double * max(len(sizes) * stride, 1))()
        nat.check(getattr(nat.lib(), self._fn[2])(self.h, int(reps), buf, len(buf)), self._fn[2])
        ms = [{P: buf[l * stride + P] for P in range(1, stride) if buf[l * stride + P] >= 0}
              for l in range(len(sizes))]
        sizes, _ = self.clusters()
        if key is not None:
            store_cluster_cache(cache, key, sizes)
        return dict(sizes=sizes, jobs=jobs, ms=ms, cached=False)


class Sim(_Clusters):
    """Handle of a tnlbm_sim (tnlbm_create ... tnlbm_destroy)."""

    def __init__(self, n_per_axis, **kw):
        c, keep = make_config(n_per_axis, **kw)
        self._init_fields(c)
        h = ctypes.c_void_p()
        nat.check(nat.lib().tnlbm_create(ctypes.byref(c), ctypes.byref(h)), "tnlbm_create")
        self.h = h
        self._owned = True
        del keep

    def _configs(self):
        return [self.cfg]

    def _init_fields(self, c):
        self.cfg = c
        self.n = c.n_per_axis
        self.N = 1 << c.n_per_axis
        self.L = 3 * c.n_per_axis
        self.Q = c.lattice
        self.chi = c.chi_max

    @classmethod
    def _borrowed(cls, handle, c):
        obj = cls.__new__(cls)
        obj._init_fields(c)
        obj.h = ctypes.c_void_p(handle)
        obj._owned = False
        return obj

    def step(self, k=1):
        nat.check(nat.lib().tnlbm_step(self.h, k), "tnlbm_step")

    def macroscopic(self):
        N3 = self.N ** 3
        rho = np.empty(N3)
        u = np.empty(3 * N3)
        nat.check(nat.lib().tnlbm_macroscopic(self.h, rho.ctypes.data_as(ctypes.c_void_p),
                                              u.ctypes.data_as(ctypes.c_void_p)), "tnlbm_macroscopic")
        N = self.N
        return rho.reshape(N, N, N), u.reshape(3, N, N, N)

    def macroscopic_slice(self, axis, index):
        """rho (N, N) and u (3, N, N) on the plane coordinate[axis] = index."""
        N = self.N
        rho = np.empty(N * N)
        u = np.empty(3 * N * N)
        nat.check(nat.lib().tnlbm_macroscopic_slice(self.h, int(axis), int(index), rho.ctypes.data_as(ctypes.c_void_p),
                                                    u.ctypes.data_as(ctypes.c_void_p)), "tnlbm_macroscopic_slice")
        return rho.reshape(N, N), u.reshape(3, N, N)

    def get_populations(self):
        ms = mps_size(self.L, self.chi)
        cores = np.empty(self.Q * ms)
        ranks = np.empty(self.Q * (self.L + 1), dtype=np.int32)
        nat.check(nat.lib().tnlbm_get_populations(self.h, cores.ctypes.data_as(ctypes.c_void_p),
                                                  ranks.ctypes.data_as(ctypes.c_void_p)), "get_populations")
        out = []
        for i in range(self.Q):
            r = ranks[i * (self.L + 1):(i + 1) * (self.L + 1)]
            cs = []
            for k in range(self.L):
                o = i * ms + mps_offset(self.L, self.chi, k)
                cs.append(cores[o:o + r[k] * 2 * r[k + 1]].reshape(r[k], 2, r[k + 1]).copy())
            out.append(cs)
        return out

    def set_populations(self, pops):
        ms = mps_size(self.L, self.chi)
        cores = np.zeros(self.Q * ms)
        ranks = np.ones(self.Q * (self.L + 1), dtype=np.int32)
        for i, cs in enumerate(pops):
            for k, c in enumerate(cs):
                o = i * ms + mps_offset(self.L, self.chi, k)
                cores[o:o + c.size] = c.reshape(-1)
                ranks[i * (self.L + 1) + k + 1] = c.shape[2]
        nat.check(nat.lib().tnlbm_set_populations(self.h, cores.ctypes.data_as(ctypes.c_void_p),
                                                  ranks.ctypes.data_as(ctypes.c_void_p)), "set_populations")

    def step_timed(self, k=1):
        """Device milliseconds of k graph launches (CUDA events)."""
        ms = ctypes.c_double()
        nat.check(nat.lib().tnlbm_step_timed(self.h, k, ctypes.byref(ms)), "tnlbm_step_timed")
        return ms.value

    def profile_step(self):
        """One eager step; per kernel class: (ms, algorithmic flops, launches)."""
        n = len(nat.KERNEL_CLASSES)
        ms = (ctypes.c_double * n)()
        fl = (ctypes.c_double * n)()
        la = (ctypes.c_int * n)()
        ph = (ctypes.c_double * len(nat.ROUND_PHASES))()
        nat.check(nat.lib().tnlbm_profile_step(self.h, ms, fl, la, ph), "tnlbm_profile_step")
        out = {c: dict(ms=ms[i], flops=fl[i], launches=la[i]) for i, c in enumerate(nat.KERNEL_CLASSES)}
        out["round"]["phase_cycles"] = {p: ph[i] for i, p in enumerate(nat.ROUND_PHASES)}
        return out

    def learn_configure(self, mode, omega, oversample=8, power=1, eta=0.2, floor_rel=None, dataset_cap=0):
        """Learned rounding: mode 0 off, 1 log spectra, 2 rank model + randomized
        truncation, 3 previous step's rank + randomized truncation
        (tnlbm_learn_configure).  omega: host array (rows x ld)."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        if floor_rel is None:
            floor_rel = 1e-12 if self.cfg.precision == nat.FP64 else 1e-5
        nat.check(nat.lib().tnlbm_learn_configure(self.h, mode, om.ctypes.data_as(nat.c_double_p), om.shape[0],
                                                  om.shape[1], oversample, power, eta, floor_rel, dataset_cap),
                  "tnlbm_learn_configure")

    def learn_set_mlp(self, half_params):
        """half_params: FP16 tensor (device or host) of mlp_param_count() values."""
        t = half_params.contiguous()
        if t.dtype != torch.float16 or t.numel() != mlp_param_count():
            raise ValueError("expected the FP16 parameter vector of the rank model")
        nat.check(nat.lib().tnlbm_learn_set_mlp(self.h, ctypes.c_void_p(t.data_ptr())), "tnlbm_learn_set_mlp")

    def learn_dataset(self, cap, reset=False):
        """(features (n x 18), labels (n,)) logged so far, at most cap rows; and
        the total number of rows logged."""
        out = np.zeros((max(cap, 1), MLP_IN + 1), dtype=np.float32)
        cnt = ctypes.c_int()
        nat.check(nat.lib().tnlbm_learn_dataset(self.h, out.ctypes.data_as(ctypes.c_void_p), cap,
                                                ctypes.byref(cnt), int(reset)), "tnlbm_learn_dataset")
        n = min(cnt.value, cap)
        return out[:n, :MLP_IN].copy(), out[:n, MLP_IN].copy(), cnt.value

    def learn_counters(self, reset=False):
        """(randomized accepted, fell back, full SVDs) since configure / reset."""
        out = (ctypes.c_longlong * 3)()
        nat.check(nat.lib().tnlbm_learn_counters(self.h, out, int(reset)), "tnlbm_learn_counters")
        return tuple(out)

    def set_limits(self, jacobi_max_sweeps=0, wait_limit_ns=0):
        """Jacobi sweep limit and cross-CTA wait limit (ns) of the step's
        roundings from the next step on (0 = defaults 60 and 5 s)."""
        nat.check(nat.lib().tnlbm_set_limits(self.h, int(jacobi_max_sweeps), int(wait_limit_ns)),
                  "tnlbm_set_limits")

    def set_face_velocity(self, face, u):
        """Inlet velocity of a velocity face from the next step on."""
        arr = (ctypes.c_double * 3)(*[float(x) for x in u])
        nat.check(nat.lib().tnlbm_set_face_velocity(self.h, face, arr), "tnlbm_set_face_velocity")

    def stats(self):
        s = nat.Stats()
        nat.check(nat.lib().tnlbm_stats_get(self.h, ctypes.byref(s)), "tnlbm_stats_get")
        return {f: getattr(s, f) for f, _ in nat.Stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
                nat.lib().tnlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch(_Clusters):
    """Several simulations (lattice sizes may differ) stepped together
    (tnlbm_batch_create ... tnlbm_batch_destroy).  configs: list of keyword
    dicts for make_config (each with n_per_axis)."""
    _fn = ("tnlbm_batch_clusters", "tnlbm_batch_set_clusters", "tnlbm_batch_tune_clusters")

    def _configs(self):
        return [s.cfg for s in self.sims]

    def __init__(self, configs):
        made = [make_config(**kw) for kw in configs]
        arr = (nat.Config * len(made))(*[c for c, _ in made])
        h = ctypes.c_void_p()
        nat.check(nat.lib().tnlbm_batch_create(arr, len(made), ctypes.byref(h)), "tnlbm_batch_create")
        self.h = h
        self.sims = [Sim._borrowed(nat.lib().tnlbm_batch_sim(h, i), c) for i, (c, _) in enumerate(made)]
        del made

    def step(self, k=1):
        nat.check(nat.lib().tnlbm_batch_step(self.h, k), "tnlbm_batch_step")

    def step_timed(self, k=1):
        ms = ctypes.c_double()
        nat.check(nat.lib().tnlbm_batch_step_timed(self.h, k, ctypes.byref(ms)), "tnlbm_batch_step_timed")
        return ms.value

    def info(self):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        nat.check(nat.lib().tnlbm_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                  "tnlbm_batch_info")
        return dict(sims=a.value, launches_per_step=b.value, jobs_per_step=c.value)

    def close(self):
        if getattr(self, "h", None):
            for s in self.sims:
                s.h = None
            nat.lib().tnlbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
