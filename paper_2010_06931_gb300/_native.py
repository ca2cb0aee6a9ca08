"""ctypes declarations of the C ABI in include/octmc.h (argument marshalling only)."""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboctmc.so")

OK = 0
NOT_CONVERGED = 1
ERRORS = {-1: "invalid argument", -2: "out of device memory", -3: "CUDA error",
          -4: "objective is not finite", -5: "device wait timed out", -6: "unsupported",
          -7: "grid exceeds the static scratch"}

F32, BF16, F16 = 0, 1, 2
LOSS_PSEUDO_HUBER, LOSS_SSD = 0, 1


class Desc(C.Structure):
    _fields_ = [
        ("w", C.c_int), ("h", C.c_int), ("d", C.c_int), ("storage", C.c_int),
        ("sx", C.c_void_p), ("sy", C.c_void_p), ("ax", C.c_void_p), ("ay", C.c_void_p),
        ("vx", C.c_void_p), ("vy", C.c_void_p), ("tx", C.c_void_p), ("ty", C.c_void_p),
        ("inputs_on_device", C.c_int),
        ("alpha", C.c_double), ("delta0", C.c_double), ("eps_h", C.c_double),
        ("eps_r", C.c_double), ("mu", C.c_double), ("loss", C.c_int),
        ("levels", C.c_int), ("lbfgs_m", C.c_int), ("max_iter", C.c_int), ("max_ls", C.c_int),
        ("gtol", C.c_double), ("ftol", C.c_double), ("stream", C.c_void_p),
        ("persistent_ascans", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [("level", C.c_int), ("iters", C.c_int), ("evals", C.c_int), ("status", C.c_int),
                ("f", C.c_double), ("eta", C.c_double), ("seconds", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

_SIGS = {
    "octmc_desc_defaults": (None, [C.POINTER(Desc)]),
    "octmc_create_problem": (C.c_int, [C.POINTER(Desc), C.POINTER(C.c_void_p)]),
    "octmc_destroy_problem": (None, [C.c_void_p]),
    "octmc_level_shape": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                    C.POINTER(C.c_int)]),
    "octmc_set_eta": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "octmc_compute_eta": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "octmc_eval_objective_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double),
                                            C.c_void_p]),
    "octmc_eval_terms": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "octmc_barrier_selftest": (C.c_int, [C.c_int]),
    "octmc_eval_objective_grad_async": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                                  C.c_void_p]),
    "octmc_eval_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_void_p),
                                   C.POINTER(C.c_void_p), C.POINTER(C.c_double)]),
    "octmc_solve_level": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Stats)]),
    "octmc_solve_full": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(Stats)]),
    "octmc_prolong": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "octmc_level_data": (C.c_int, [C.c_void_p, C.c_int] + [C.c_void_p] * 6),
    "octmc_merge": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double] + [C.c_void_p] * 5),
    "octmc_prealign_disp": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "octmc_prealign_eval": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "octmc_prealign_level": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.POINTER(Stats)]),
    "octmc_prealign_full": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(Stats)]),
    "octmc_saccade_validity": (C.c_int, [C.c_void_p] + [C.c_int] * 4 + [C.c_void_p] * 3),
    "octmc_enface": (C.c_int, [C.c_void_p, C.c_void_p] + [C.c_int] * 4 + [C.c_void_p] + [C.c_double] * 4
                     + [C.c_void_p] * 4),
    "octmc_lbfgs_create": (C.c_int, [C.c_int64, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "octmc_lbfgs_destroy": (None, [C.c_void_p]),
    "octmc_lbfgs_push": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "octmc_lbfgs_direction": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "octmc_lbfgs_reset": (C.c_int, [C.c_void_p]),
    "octmc_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "octmc_profile_read": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    "octmc_data_term_static": (C.c_int, [C.c_void_p] * 6 + [C.c_int] * 3 + [C.c_void_p] + [C.c_double] * 3
                               + [C.c_int] + [C.c_void_p] * 3),
    "octmc_estimate_bytes": (C.c_int64, [C.POINTER(Desc)]),
    "octmc_server_create": (C.c_int, [C.c_int64, C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]),
    "octmc_server_destroy": (None, [C.c_void_p]),
    "octmc_server_submit": (C.c_int, [C.c_void_p, C.POINTER(Desc), C.POINTER(C.c_int64)]),
    "octmc_server_step": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "octmc_server_state": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int)]),
    "octmc_server_poll": (C.c_int, [C.c_void_p, C.c_int64, C.POINTER(C.c_int), C.c_void_p, C.POINTER(Stats),
                                    C.c_int, C.POINTER(C.c_int)]),
    "octmc_status_string": (C.c_char_p, [C.c_int]),
}


def exported_names():
    return sorted(_SIGS)


def lib():
    """The loaded liboctmc.so.  Raises if it has not been built: there is no fallback."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liboctmc.so is not built (run __graft_entry__.build() or "
                              "python paper_2010_06931_gb300/build.py); no CPU fallback exists")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class OctmcError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (%d)" % (where, ERRORS.get(code, "error"), code))


def check(code, where):
    if code < 0:
        raise OctmcError(code, where)
    return code
