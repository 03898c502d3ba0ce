"""ctypes binding of ``libiwfpm.so`` (declared in ``include/iwfpm.h``): argument marshalling only.

Every entry point of the header is exposed under the same name. No computation happens
here; if the shared library is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libiwfpm.so")

IWF_OK = 0
STATUS = {0: "IWF_OK", -1: "IWF_ERR_ARG", -2: "IWF_ERR_SINGULAR_PI", -3: "IWF_ERR_ALLOC",
          -4: "IWF_ERR_CUDA", -5: "IWF_ERR_NONFINITE", -6: "IWF_ERR_BREAKDOWN",
          -7: "IWF_ERR_NOCONV", -8: "IWF_ERR_TIMEOUT", -9: "IWF_ERR_WINDOW_TIE",
          -10: "IWF_ERR_UNSUPPORTED"}
IWF_METHOD_IWFPM, IWF_METHOD_PM = 0, 1
IWF_SHIFT_EXACT, IWF_SHIFT_ROUND = 0, 1
IWF_PREC_F64, IWF_PREC_C64, IWF_PREC_F64_EXACT, IWF_PREC_F64_DF = 0, 1, 2, 3
IWF_CONTRACT_TENSOR, IWF_CONTRACT_DF, IWF_CONTRACT_F64 = 0, 1, 2
IWF_PATH_AUTO, IWF_PATH_TILED, IWF_PATH_PENCIL = 0, 1, 2


class IwfError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class iwf_plan_opts(C.Structure):
    _fields_ = [("method", C.c_int), ("shift_round", C.c_int), ("device", C.c_int)]


class iwf_solve_opts(C.Structure):
    _fields_ = [("nev", C.c_int), ("block", C.c_int), ("maxit", C.c_int), ("tol", C.c_double),
                ("precision", C.c_int), ("c64_tol", C.c_double), ("seed", C.c_ulonglong)]


class iwf_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("iters_c64", C.c_int), ("applies", C.c_longlong),
                ("converged", C.c_int), ("max_resid", C.c_double), ("seconds", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run python -m paper_2404_04507_gb300.build")
    return C.CDLL(LIB_PATH)


lib = _load()

_vp, _i, _ll = C.c_void_p, C.c_int, C.c_longlong
_PROTOS = {
    "iwf_version": (_i, []),
    "iwf_last_error": (C.c_char_p, []),
    "iwf_plan_create": (_i, [C.POINTER(_vp), _i, _i, C.POINTER(C.c_double), C.POINTER(_i),
                             C.POINTER(_i), C.POINTER(iwf_plan_opts)]),
    "iwf_plan_destroy": (None, [_vp]),
    "iwf_coef_extent": (_i, [_vp, _vp, C.c_double, C.POINTER(C.c_int), _vp]),
    "iwf_plan_set_arith": (_i, [_vp, _i]),
    "iwf_plan_trim": (None, [_vp]),
    "iwf_plan_size": (_i, [_vp, C.POINTER(_ll)]),
    "iwf_plan_lens": (_i, [_vp, C.POINTER(_i)]),
    "iwf_window": (_i, [_vp, C.POINTER(_i)]),
    "iwf_kinetic": (_i, [_vp, C.POINTER(C.c_double)]),
    "iwf_set_potential": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(C.c_double),
                               C.POINTER(C.c_double)]),
    "iwf_apply": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "iwf_preconditioner": (_i, [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "iwf_apply_profile": (_i, [_vp, _i, _vp, _vp, _i, _vp, C.POINTER(C.c_double),
                               C.POINTER(_i)]),
    "iwf_kernel_launches": (_ll, []),
    "iwf_apply_noalloc": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "iwf_apply_host": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "iwf_apply_stencil": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "iwf_evaluate": (_i, [_vp, _vp, _vp, _ll, _vp, _vp]),
    "iwf_evaluate_grid": (_i, [_vp, _vp, C.POINTER(C.c_double), C.POINTER(C.c_double),
                               C.POINTER(C.c_int), _vp, _vp]),
    "iwf_field_normalize": (_i, [_vp, _vp, _ll, _ll, _vp, _vp, _vp]),
    "iwf_field_distance": (_i, [_vp, _vp, _vp, _ll, _vp, _vp]),
    "iwf_plan_autotune": (_i, [_vp, _i, _i, C.POINTER(C.c_double), C.POINTER(_i), _vp]),
    "iwf_plan_set_schedule": (_i, [_vp, _i, _i, _i, _i]),
    "iwf_plan_set_path": (_i, [_vp, _i, _i]),
    "iwf_plan_get_schedule": (_i, [_vp, _i, C.POINTER(_i)]),
    "iwf_eigensolve": (_i, [_vp, C.POINTER(iwf_solve_opts), _vp, C.POINTER(C.c_double), _vp,
                            C.POINTER(C.c_double), C.POINTER(iwf_solve_info), _vp]),
    "iwf_batch_eigensolve": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(iwf_solve_opts), _vp,
                                  C.POINTER(C.c_double), _vp, C.POINTER(C.c_double),
                                  C.POINTER(_i), C.POINTER(iwf_solve_info), _vp]),
    "iwf_ws_create": (_i, [C.POINTER(_vp), _i, C.POINTER(_i), C.c_ulonglong, _i]),
    "iwf_ws_destroy": (None, [_vp]),
    "iwf_ws_num_params": (_i, [_vp, C.POINTER(_ll)]),
    "iwf_ws_get_params": (_i, [_vp, C.POINTER(C.c_float)]),
    "iwf_ws_set_params": (_i, [_vp, C.POINTER(C.c_float)]),
    "iwf_ws_predict": (_i, [_vp, _i, _vp, _vp, _vp]),
    "iwf_ws_loss_grad": (_i, [_vp, _i, _vp, _vp, _i, _i, C.POINTER(C.c_float),
                              C.POINTER(C.c_float), _vp]),
    "iwf_ws_train": (_i, [_vp, _i, _vp, _vp, _i, _i, _i, _i, C.c_float, C.c_float,
                          C.c_ulonglong, C.POINTER(C.c_float), _vp]),
    "iwf_ws_embed": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp]),
    "iwf_ws_phase": (_i, [_vp, _i, _i, C.POINTER(C.c_double), _i, _vp, _vp]),
    "iwf_plan_check": (_i, [_vp, _vp]),
    "iwf_batch_solve": (_i, [_i, C.POINTER(_vp), C.POINTER(iwf_solve_opts), C.POINTER(_vp),
                             C.POINTER(C.c_double), C.POINTER(_vp), C.POINTER(C.c_double),
                             C.POINTER(_i), C.POINTER(iwf_solve_info), _vp]),
    "iwf_gram": (_i, [_i, _ll, _vp, _i, _vp, _i, _vp, _i, _vp]),
    "iwf_block_update": (_i, [_i, _ll, _vp, _i, _vp, _i, _vp, _i, _i, _vp]),
    "iwf_plan_set_wait_limit": (_i, [_vp, _ll]),
}
for _name, (_res, _args) in _PROTOS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args
    globals()[_name] = _fn


def check(status: int, where: str) -> None:
    if status != IWF_OK:
        raise IwfError(status, where, lib.iwf_last_error().decode(errors="replace"))
