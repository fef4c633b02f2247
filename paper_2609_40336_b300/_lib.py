"""ctypes declarations of the C ABI in include/lrh.h (argument marshalling only).

Loading fails loudly when ``liblrh.so`` has not been built: there is no CPU
fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblrh.so")

LRH_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOTHERM", -3: "EPOSET", -4: "ENOMEM", -5: "ECUDA",
          -6: "ETIMEOUT", -7: "ENUMERIC", -8: "EUNSUPPORTED", -9: "ENOCONV", -10: "EDEADLINE"}
EINVAL, ENOTHERM, EPOSET, ENOMEM, ECUDA, ETIMEOUT, ENUMERIC, EUNSUPPORTED = -1, -2, -3, -4, -5, -6, -7, -8
ENOCONV, EDEADLINE = -9, -10
SUBGRADIENT, NESTEROV = 0, 1
STEP_CONST, STEP_INV_SQRT = 0, 1
MSG_NU, MSG_ZETA, MSG_NU_BEST, MSG_GRAD = 0, 1, 2, 3
BOUND_CERTIFIED, BOUND_LAST, BOUND_BEST = 0, 1, 2


class ProblemDesc(C.Structure):
    _fields_ = [
        ("n_sites", C.c_int32),
        ("n_regions", C.c_int32),
        ("region_ptr", C.POINTER(C.c_int64)),
        ("region_sites", C.POINTER(C.c_int32)),
        ("n_terms", C.c_int32),
        ("term_ptr", C.POINTER(C.c_int64)),
        ("term_sites", C.POINTER(C.c_int32)),
        ("term_mat_off", C.POINTER(C.c_int64)),
        ("term_mat_total", C.c_int64),
        ("term_mats", C.POINTER(C.c_double)),
        ("n_instances", C.c_int32),
        ("n_pairs", C.c_int64),
        ("pair_parent", C.POINTER(C.c_int32)),
        ("pair_child", C.POINTER(C.c_int32)),
        ("term_region", C.POINTER(C.c_int32)),
        ("region_ghost", C.POINTER(C.c_uint8)),
    ]


class HaloItem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("id", C.c_int32)]


HALO_STATE = 0
HALO_TRACE = 1


class Options(C.Structure):
    _fields_ = [
        ("variant", C.c_int32),
        ("step_rule", C.c_int32),
        ("alpha", C.c_double),
        ("beta", C.c_double),
        ("lhat", C.c_double),
        ("degen_tol", C.c_double),
        ("max_sweeps", C.c_int32),
        ("loop", C.c_int32),
        ("cert_sweeps", C.c_int32),
        ("n_beta", C.c_int32),
        ("beta_sched", C.POINTER(C.c_double)),
        ("iters_per_stage", C.c_int32),
        ("certify_every", C.c_int32),
        ("deadline_s", C.c_double),
        ("tune_cache", C.c_char_p),
        ("target", C.POINTER(C.c_double)),
        ("screen_tol", C.c_double),
        ("cold_start", C.c_int32),
    ]


class Info(C.Structure):
    _fields_ = [
        ("n_instances", C.c_int32),
        ("n_regions", C.c_int32),
        ("n_pairs", C.c_int32),
        ("max_region_sites", C.c_int32),
        ("msg_elems", C.c_int64),
        ("lambda_G", C.c_double),
        ("gamma_G", C.c_double),
        ("iteration", C.c_int64),
        ("n_classes", C.c_int32),
        ("class_sites", C.c_int32 * 8),
        ("class_regions", C.c_int32 * 8),
        ("sweeps", C.c_uint64 * 8),
        ("class_block", C.c_int32 * 8),
        ("concurrent_classes", C.c_int32),
        ("loop", C.c_int32),
        ("persistent_grid", C.c_int32),
        ("persistent_tiles", C.c_int64),
        ("sweep_capped", C.c_uint64 * 8),
        ("n_sites", C.c_int32),
        ("kappa_G", C.c_int32),
        ("warm_bytes", C.c_int64),
    ]


class Params(C.Structure):
    _fields_ = [
        ("beta", C.c_double), ("lhat", C.c_double), ("alpha", C.c_double), ("c", C.c_double),
        ("lambda_G", C.c_double), ("gamma_G", C.c_double),
        ("kappa_G", C.c_int32), ("n_sites", C.c_int32),
        ("T_nesterov", C.c_int64), ("T_subgradient", C.c_int64),
    ]


class Record(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("seconds", C.c_double), ("beta", C.c_double)]


class LrhError(RuntimeError):
    def __init__(self, code: int, fn: str, detail: str):
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)} ({detail})")
        self.code = code


# name -> (restype, argtypes)
SIGNATURES = {
    "lrh_create": (C.c_int, [C.POINTER(ProblemDesc), C.POINTER(Options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "lrh_destroy": (None, [C.c_void_p]),
    "lrh_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "lrh_get_pairs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lrh_set_options": (C.c_int, [C.c_void_p, C.POINTER(Options)]),
    "lrh_restart": (C.c_int, [C.c_void_p]),
    "lrh_step": (C.c_int, [C.c_void_p, C.c_int32]),
    "lrh_evaluate": (C.c_int, [C.c_void_p]),
    "lrh_launch_region_pass": (C.c_int, [C.c_void_p, C.c_int32]),
    "lrh_bound": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "lrh_get_region_values": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "lrh_get_messages": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32]),
    "lrh_set_messages": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32]),
    "lrh_selftest_barrier_timeout": (C.c_int, [C.c_void_p]),
    "lrh_set_class_mode": (C.c_int, [C.c_void_p, C.c_int32]),
    "lrh_synchronize": (C.c_int, [C.c_void_p]),
    "lrh_set_terms": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lrh_autotune": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int32]),
    "lrh_set_launch_shape": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32]),
    "lrh_state_bytes": (C.c_int64, [C.c_void_p]),
    "lrh_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "lrh_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "lrh_vjp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32]),
    "lrh_level1_eval_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lrh_theorem_parameters": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.POINTER(Params)]),
    "lrh_reset": (C.c_int, [C.c_void_p]),
    "lrh_solve": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lrh_plan_poset": (C.c_int, [C.POINTER(ProblemDesc), C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "lrh_halo_set": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "lrh_halo_pass": (C.c_int, [C.c_void_p]),
    "lrh_halo_pack": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lrh_halo_unpack": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lrh_halo_update": (C.c_int, [C.c_void_p]),
    "lrh_strerror": (C.c_char_p, [C.c_int]),
    "lrh_last_error": (C.c_char_p, []),
}

_lib = None


def load() -> C.CDLL:
    """Load liblrh.so (built in-tree by ``paper_2609_40336_b300.build``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2609_40336_b300.build`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int, fn: str) -> None:
    if code != LRH_OK:
        detail = load().lrh_last_error().decode(errors="replace")
        raise LrhError(code, fn, detail)
