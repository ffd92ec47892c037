"""ctypes declarations of librsr's C ABI (include/rsr.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librsr.so")

RSR_OK = 0
RSR_ERR_INVALID_ARG = -1
RSR_ERR_CUDA = -2
RSR_ERR_WORKSPACE = -3
RSR_ERR_TIMEOUT = -4
RSR_ERR_UNSUPPORTED = -5
RSR_ERR_NOT_PREPARED = -6

RSR_PATH_AUTO = 0
RSR_PATH_POPC = 1
RSR_PATH_TC = 2

RSR_FLAG_DENSE = 1
RSR_FLAG_NO_INDEX = 2
RSR_FLAG_TEST_STALL = 0x100
RSR_FLAG_TEST_DEEP_CAP = 0x200
RSR_FLAG_TEST_TWO_PASS = 0x400
RSR_FLAG_TEST_TILES3 = 0x800


class rsr_problem(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("pmf", ctypes.c_void_p),
        ("R_L", ctypes.c_int64),
        ("R_U", ctypes.c_int64),
        ("ref_L", ctypes.c_void_p),
        ("ref_U", ctypes.c_void_p),
        ("path", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]


RSR_PHI_ST_CONNECTIVITY = 0
RSR_PHI_ST_MAXFLOW_LEVELS = 1
RSR_PHI_GLOBAL_CONNECTIVITY = 2
RSR_PHI_GLOBAL_CONN_LEVEL = 3

RSR_SEARCH_INDEX_ORDER = 0
RSR_SEARCH_PERMUTED = 1


class rsr_system(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("n_nodes", ctypes.c_int32),
        ("src", ctypes.c_void_p),
        ("dst", ctypes.c_void_p),
        ("s", ctypes.c_int32),
        ("t", ctypes.c_int32),
        ("n_levels", ctypes.c_int32),
        ("level_thr", ctypes.c_int32 * 8),
        ("m_prime", ctypes.c_int32),
    ]


class rsr_stage1_opts(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("N", ctypes.c_int64),
        ("max_starts", ctypes.c_int64),
        ("eps_u", ctypes.c_double),
        ("R_max", ctypes.c_int64),
        ("max_rounds", ctypes.c_int32),
        ("search_order", ctypes.c_int32),
    ]


class rsr_stage1_result(ctypes.Structure):
    _fields_ = [
        ("rounds", ctypes.c_int32),
        ("stop", ctypes.c_int32),
        ("R_L", ctypes.c_int64),
        ("R_U", ctypes.c_int64),
        ("n_u_last", ctypes.c_int64),
        ("phi_evals", ctypes.c_int64),
    ]


class rsr_estimate_out(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in (
        "pL", "pU", "pu", "P_lower", "P_upper", "cov_pL", "cov_pU", "cov_pu", "cov_lower", "cov_upper")]


# (name, restype, argtypes) of every entry point declared in include/rsr.h
_P, _S = ctypes.c_void_p, ctypes.c_size_t
_I32, _I64, _U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_PROB = ctypes.POINTER(rsr_problem)
SIGNATURES = {
    "rsr_measure_int_peak": (ctypes.c_int, [_P, _P, _P]),
    "rsr_measure_philox_rate": (ctypes.c_int, [_P, _P]),
    "rsr_measure_fp8_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, _P, _P, _P]),
    "rsr_classify_plan": (ctypes.c_int, [_PROB, _I64, ctypes.c_size_t, _P]),
    "rsr_workspace_size": (ctypes.c_size_t, [_PROB, _I64]),
    "rsr_prepare": (ctypes.c_int, [_PROB, _P, _S, _P]),
    "rsr_update_pmf": (ctypes.c_int, [_PROB, _P, _S, _P]),
    "rsr_classify": (ctypes.c_int, [_PROB, _U64, _U64, _I64, _P, _P, _P, _P, _P, _P, _S, _P]),
    "rsr_estimate": (ctypes.c_int, [_P, _I64, _I64, ctypes.POINTER(rsr_estimate_out)]),
    "rsr_grad": (ctypes.c_int, [_PROB, _U64, _U64, _I64, _P, _P, _I64, _P, _P, _P, _S, _P]),
    "rsr_sample": (ctypes.c_int, [_PROB, _U64, _U64, _I64, _P, _P, _S, _P]),
    "rsr_workspace_status": (ctypes.c_int, [_P, _P, _P]),
    "rsr_batch_workspace_size": (ctypes.c_size_t, [_PROB, _I32, _P]),
    "rsr_batch_prepare": (ctypes.c_int, [_PROB, _I32, _P, _P, _P, _P, _P, _P, _P, _S, _P]),
    "rsr_batch": (ctypes.c_int, [_PROB, _I32, _P, _P, _P, _P, _P, _P, _P, _S, _P]),
    "rsr_batch_autotune": (ctypes.c_int, [_PROB, _I32, _P, _P, _P, _P, _P, _P, _P, _S, _P, _P]),
    "rsr_batch_profile": (ctypes.c_int, [_PROB, _I32, _P, _P, _P, _P, _P, _P, _P, _S, _P, _P]),
    "rsr_autotune": (ctypes.c_int, [_PROB, _P, _S, _P, _P]),
    "rsr_batch_grad": (ctypes.c_int, [_PROB, _I32, _P, _P, _P, _P, _P]),
    "rsr_classify_static": (ctypes.c_int, [_PROB, _U64, _U64, _I64, _P, _P, _P, _P, _P]),
    "rsr_resolve": (ctypes.c_int, [_PROB, ctypes.POINTER(rsr_system), _U64, _U64, _I64, _P, _P, _I64, _P, _P, _S,
                                   _P]),
    "rsr_level_pmf": (ctypes.c_int, [_PROB, _I32, _P, _P, ctypes.POINTER(rsr_system), _U64, _U64, _I64, _P, _P, _P,
                                     _P, _P, _P]),
    "rsr_search_workspace_size": (ctypes.c_size_t, [_PROB]),
    "rsr_boundary_search": (ctypes.c_int, [_PROB, ctypes.POINTER(rsr_system), _U64, _U64, _P, _I64, _P, _P, _P,
                                           _I32, _P, _S, _P]),
    "rsr_nondominated_scratch_size": (ctypes.c_size_t, [_I32, _I32, _I64]),
    "rsr_nondominated": (ctypes.c_int, [_I32, _I32, _I64, _P, _I32, _P, _P, _P, _S, _P]),
    "rsr_stage1_workspace_size": (ctypes.c_size_t, [_PROB, ctypes.POINTER(rsr_stage1_opts)]),
    "rsr_stage1": (ctypes.c_int, [_PROB, ctypes.POINTER(rsr_system), ctypes.POINTER(rsr_stage1_opts), _P, _P, _P,
                                  ctypes.POINTER(rsr_stage1_result), _P, _S, _P]),
    "rsr_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "rsr_last_cuda_error": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librsr.so; raise if it is missing (there is no fallback path)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    "librsr.so is not built (%s); run paper_2604_17066_gb300.build.build() "
                    "or __graft_entry__.build()" % path)
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class RSRError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.rsr_status_string(status).decode()
        if status == RSR_ERR_CUDA:
            msg += ": " + lib.rsr_last_cuda_error().decode()
        super().__init__("%s failed: %s (%d)" % (where, msg, status))
        self.status = status


def check(status: int, where: str) -> None:
    if status != RSR_OK:
        raise RSRError(status, where)
