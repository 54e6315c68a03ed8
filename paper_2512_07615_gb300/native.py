"""ctypes declarations of the C ABI in include/tnlbm.h.

Loading fails loudly: there is no fallback implementation of any entry point.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtnlbm.so")

FP64, FP32, TF32, MIXED, BF16 = 0, 1, 2, 3, 4
D3Q19, D3Q15 = 19, 15
CLUSTER_MAX = 16   # TNLBM_CLUSTER_MAX
FACE_WALL, FACE_VELOCITY, FACE_PRESSURE = 0, 1, 2
HADAMARD_FIT, HADAMARD_EXACT, HADAMARD_ZIPUP = 0, 1, 2
TERM_PLAIN, TERM_SHIFT, TERM_MASK1, TERM_KRON, TERM_ONES = 0, 1, 2, 3, 4
KERNEL_CLASSES = ("round", "fit_gemm", "fit_qr", "fit_misc", "rho0", "copy", "zipup")
ROUND_PHASES = ("terms", "gemm_rw", "qr", "jacobi", "svd_out", "gemm_qus", "jacobi_sweeps", "svd_count",
                "jacobi_global", "svd_global_count", "svd64_flops", "svd64_exec_flops", "rx_norms", "rx_dots",
                "rx_wait", "rx_angle", "rx_rot", "jacobi32", "newton_schulz", "xv", "sweeps32", "rounds64")

c_int_p = ctypes.POINTER(ctypes.c_int)
c_double_p = ctypes.POINTER(ctypes.c_double)


class Config(ctypes.Structure):
    _fields_ = [
        ("n_per_axis", ctypes.c_int),
        ("lattice", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("periodic", ctypes.c_int * 3),
        ("solid", ctypes.POINTER(ctypes.c_uint8)),
        ("chi_mask", ctypes.c_int),
        ("eps_mask", ctypes.c_double),
        ("mask_cores", c_double_p),
        ("mask_ranks", c_int_p),
        ("mask_cap", ctypes.c_int),
        ("force", ctypes.c_double * 3),
        ("chi_max", ctypes.c_int),
        ("eps", ctypes.c_double),
        ("precision", ctypes.c_int),
        ("hadamard", ctypes.c_int),
        ("sweeps", ctypes.c_int),
        ("n_modes", ctypes.c_int),
        ("modes", c_double_p),
        ("max_jobs_in_flight", ctypes.c_int),
        ("conserve_mass", ctypes.c_int),
        ("face_kind", ctypes.c_int * 6),
        ("face_u", (ctypes.c_double * 3) * 6),
        ("face_rho", ctypes.c_double * 6),
        ("block_sums", ctypes.c_int),
        ("learned_rank", ctypes.c_int),
        ("seed", ctypes.c_uint64),
        ("jacobi_max_sweeps", ctypes.c_int),
        ("wait_limit_ns", ctypes.c_longlong),
        ("max_cluster", ctypes.c_int),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("steps", ctypes.c_int64),
        ("max_bond", ctypes.c_int),
        ("mean_bond", ctypes.c_double),
        ("nvps", ctypes.c_double),
        ("compression_ratio", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("status", ctypes.c_int),
        ("gpu_launches_per_step", ctypes.c_int),
        ("round_jobs_per_step", ctypes.c_int),
        ("product_jobs_per_step", ctypes.c_int),
        ("mass", ctypes.c_double),
        ("discarded2", ctypes.c_double),
        ("round_ctas_per_step", ctypes.c_int),
        ("max_cluster", ctypes.c_int),
    ]


class Term(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("coef", ctypes.c_double),
        ("x", ctypes.c_void_p),
        ("x_ranks", ctypes.c_void_p),
        ("x_cap", ctypes.c_int),
        ("y", ctypes.c_void_p),
        ("y_ranks", ctypes.c_void_p),
        ("y_cap", ctypes.c_int),
        ("axis", ctypes.c_int),
        ("offset", ctypes.c_int),
        ("cyclic", ctypes.c_int),
        ("mask", c_double_p),
    ]


_lib = None

# name -> (restype, argtypes)
SIGNATURES = {
    "tnlbm_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "tnlbm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tnlbm_macroscopic": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_macroscopic_slice": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "tnlbm_get_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_set_populations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "tnlbm_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tnlbm_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "tnlbm_set_limits": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong]),
    "tnlbm_profile_step": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_int_p, c_double_p]),
    "tnlbm_last_error": (ctypes.c_char_p, []),
    "tnlbm_mps_size": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
    "tnlbm_mps_offset": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "tnlbm_lincomb_round": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(Term), ctypes.POINTER(ctypes.c_void_p),
                                           ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_void_p]),
    "tnlbm_lincomb_round_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                   ctypes.POINTER(Term), ctypes.POINTER(ctypes.c_void_p),
                                                   ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                                   ctypes.c_double, ctypes.c_void_p]),
    "tnlbm_lincomb_round_rsvd": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(Term), ctypes.POINTER(ctypes.c_void_p),
                                                ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                                ctypes.c_double, c_int_p, ctypes.c_void_p, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_double, c_int_p, ctypes.c_void_p]),
    "tnlbm_mlp_param_count": (ctypes.c_int, []),
    "tnlbm_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
    "tnlbm_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_learn_configure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int]),
    "tnlbm_learn_set_mlp": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_learn_dataset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, c_int_p,
                                           ctypes.c_int]),
    "tnlbm_learn_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
    "tnlbm_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tnlbm_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "tnlbm_batch_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "tnlbm_batch_sim": (ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int]),
    "tnlbm_batch_info": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p, c_int_p]),
    "tnlbm_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tnlbm_clusters": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p, ctypes.c_int, c_int_p]),
    "tnlbm_set_clusters": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int]),
    "tnlbm_tune_clusters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_int]),
    "tnlbm_batch_clusters": (ctypes.c_int, [ctypes.c_void_p, c_int_p, c_int_p, ctypes.c_int, c_int_p]),
    "tnlbm_batch_set_clusters": (ctypes.c_int, [ctypes.c_void_p, c_int_p, ctypes.c_int]),
    "tnlbm_batch_tune_clusters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p, ctypes.c_int]),
    "tnlbm_mask_product": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    "tnlbm_set_face_velocity": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, c_double_p]),
    "tnlbm_materialize": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Term),
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.c_int, ctypes.c_void_p]),
    "tnlbm_hadamard_fit": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                          ctypes.c_int, ctypes.c_void_p]),
    "tnlbm_hadamard_zipup": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_void_p]),
    "tnlbm_inner_ones": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_to_dense": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "tnlbm_from_dense": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_void_p]),
}


def lib():
    """The loaded libtnlbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtnlbm.so is missing: run __graft_entry__.build() "
                               "(paper_2512_07615_gb300/build.py) first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TnlbmError(RuntimeError):
    def __init__(self, code, where):
        msg = lib().tnlbm_last_error()
        super().__init__("%s failed with code %d: %s" % (where, code, msg.decode() if msg else ""))
        self.code = code


def check(code, where):
    if code != 0:
        raise TnlbmError(code, where)
