"""ctypes declarations of the C ABI in include/rcp.h (argument marshalling only).

``load()`` opens ``librcp.so`` built next to this file and raises if it is
missing: there is no CPU fallback for any entry point.
"""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librcp.so")

MAX_NDIM = 8

RCP_OK, RCP_EINVAL, RCP_ENOMEM, RCP_ECUDA, RCP_ESINGULAR, RCP_ENAN, RCP_ETIMEOUT, \
    RCP_EORDER, RCP_ENOTCONV = range(9)
RCP_DTYPE_F64, RCP_DTYPE_F32 = 0, 1
RCP_PREC_F64, RCP_PREC_MIXED = 0, 1
RCP_FLAG_HOST_STAGING, RCP_FLAG_NO_SHIFT, RCP_FLAG_MODE_OVERSAMPLE, RCP_FLAG_LU_NORM = 1, 2, 4, 8
RCP_FLAG_INDEPENDENT = 16
RCP_INIT_RANDN, RCP_INIT_LEARNED, RCP_INIT_EIG = 0, 1, 2
RCP_SOLVER_ALS, RCP_SOLVER_BCD = 0, 1
RCP_ARITH_DW_ADD, RCP_ARITH_DW_MUL, RCP_ARITH_DW_RCP, RCP_ARITH_DW_SQRT, RCP_ARITH_RSQRT64 = range(5)
RCP_INFO_SHIFTED_QR, RCP_INFO_ALS_REGULARISED, RCP_INFO_LEARNED_INIT = 1, 2, 4
WS_LPAD, WS_RPAD = 24, 16
MLP_IN, MLP_HIDDEN, MLP_OUT = 13824, 512, 1152
RCP_KT_SKETCH, RCP_KT_APPLY, RCP_KT_PROJECT, RCP_KT_TTM, RCP_KT_ALS, RCP_KT_ALL = range(6)


class RcpConfig(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32),
                ("dims", ctypes.c_int64 * MAX_NDIM),
                ("in_dtype", ctypes.c_int32),
                ("rank", ctypes.c_int32),
                ("oversample", ctypes.c_int32),
                ("power_iters", ctypes.c_int32),
                ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32),
                ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int32),
                ("flags", ctypes.c_int32),
                ("init", ctypes.c_int32),
                ("solver", ctypes.c_int32),
                ("skip_modes", ctypes.c_int32),
                ("mode_oversample", ctypes.c_int32 * MAX_NDIM),
                ("wait_budget", ctypes.c_int64)]


class RcpResult(ctypes.Structure):
    _fields_ = [("fit", ctypes.c_double),
                ("iters", ctypes.c_int32),
                ("info", ctypes.c_int32),
                ("norm_x2", ctypes.c_double),
                ("norm_b2", ctypes.c_double),
                ("rel_err", ctypes.c_double),
                ("device_status", ctypes.c_int32),
                ("widths", ctypes.c_int32 * MAX_NDIM)]


# name -> (restype, argtypes); every symbol declared in include/rcp.h
P = ctypes.c_void_p
DP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "rcp_plan": (ctypes.c_int, [ctypes.POINTER(RcpConfig), P, ctypes.POINTER(P)]),
    "rcp_plan_destroy": (ctypes.c_int, [P]),
    "rcp_width": (ctypes.c_int32, [P, ctypes.c_int32]),
    "rcp_sketch": (ctypes.c_int, [P, P, ctypes.c_int32, P]),
    "rcp_compress": (ctypes.c_int, [P, P, ctypes.c_int32]),
    "rcp_als_init": (ctypes.c_int, [P, ctypes.POINTER(P)]),
    "rcp_als": (ctypes.c_int, [P, DP, DP, ctypes.POINTER(ctypes.c_int32)]),
    "rcp_project": (ctypes.c_int, [P, ctypes.POINTER(P), P]),
    "rcp_decompose": (ctypes.c_int, [P, P, ctypes.POINTER(P), P]),
    "rcp_decompose_host": (ctypes.c_int, [P, P, ctypes.POINTER(P), DP, ctypes.POINTER(RcpResult)]),
    "rcp_result_get": (ctypes.c_int, [P, ctypes.POINTER(RcpResult)]),
    "rcp_get_core": (ctypes.c_int, [P, P]),
    "rcp_get_compressed_factors": (ctypes.c_int, [P, ctypes.POINTER(P), P]),
    "rcp_last_error": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
    "rcp_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "rcp_profile_enable": (ctypes.c_int, [P, ctypes.c_int32]),
    "rcp_profile_read": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_int64), DP]),
    "rcp_plan_batched": (ctypes.c_int, [ctypes.POINTER(RcpConfig), ctypes.c_int32, P,
                                        ctypes.POINTER(P)]),
    "rcp_batched_run": (ctypes.c_int, [P, ctypes.POINTER(P)]),
    "rcp_batched_autotune": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(ctypes.c_int32)]),
    "rcp_batched_result": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(P), P,
                                          ctypes.POINTER(RcpResult)]),
    "rcp_batched_destroy": (ctypes.c_int, [P]),
    "rcp_batched_intermediates": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(P), P,
                                                 ctypes.POINTER(P), P]),
    "rcp_mlp_param_count": (ctypes.c_int64, []),
    "rcp_mlp_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, P, ctypes.POINTER(P)]),
    "rcp_mlp_destroy": (ctypes.c_int, [P]),
    "rcp_mlp_get_params": (ctypes.c_int, [P, P, P, P, ctypes.POINTER(ctypes.c_int64)]),
    "rcp_mlp_set_params": (ctypes.c_int, [P, P, P, P, ctypes.c_int64]),
    "rcp_mlp_forward": (ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int32, P]),
    "rcp_mlp_backward": (ctypes.c_int, [P, P, P]),
    "rcp_mlp_adam": (ctypes.c_int, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float]),
    "rcp_mlp_status": (ctypes.c_int, [P]),
    "rcp_ws_canonicalize": (ctypes.c_int, [P, P, ctypes.c_int32, P, P, P]),
    "rcp_ws_loss": (ctypes.c_int, [P, P, P, ctypes.c_int32, ctypes.c_float, P, P, P]),
    "rcp_mlp_train_step": (ctypes.c_int, [P, P, P, P, ctypes.c_int32, ctypes.c_float, P]),
    "rcp_batched_export": (ctypes.c_int, [P, P, P, P, P, P]),
    "rcp_batched_set_warm_start": (ctypes.c_int, [P, P]),
    "rcp_set_warm_start": (ctypes.c_int, [P, P]),
    "rcp_synth_cp": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                    ctypes.POINTER(P), P, ctypes.c_float, ctypes.c_uint64, P, P]),
    "rcp_sketch_mode1_static": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                               ctypes.c_int32, ctypes.c_uint64, P, P, P]),
    "rcp_measure_fma_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                            ctypes.c_void_p]),
    "rcp_test_arith": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "rcp_test_normals": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_int64, ctypes.c_int64, P, P, P, P]),
}

_LIB = None


class RcpError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _LIB.rcp_status_str(code).decode() if _LIB is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")


def load():
    """Open librcp.so (built by ``paper_1703_09074_gb300.build``); no fallback."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librcp.so not found at {LIB_PATH}: build it with "
                           "`python -m paper_1703_09074_gb300.build` (nvcc, sm_103a)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(code, where, ok=(RCP_OK,)):
    if code not in ok:
        raise RcpError(code, where)
    return code
