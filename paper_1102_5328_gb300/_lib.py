"""ctypes binding of libtileqr.so: the C ABI of include/tileqr.h with the
same names, argument marshalling only. Every computation runs in the CUDA
library; there is no Python or CPU fallback: if the library cannot be built
or loaded, loading raises."""
import ctypes
import os

from . import build as _build

_lib = None

c_i64 = ctypes.c_int64
c_int = ctypes.c_int
c_vp = ctypes.c_void_p
c_dbl = ctypes.c_double

# (name, restype, argtypes) for every symbol of include/tileqr.h
SIGNATURES = [
    ("qr_workspace", c_int, [c_i64, c_i64, c_int, c_int, c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("qr_factor_d", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("qr_factor_s", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("qr_factor_d_noalloc", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_vp]),
    ("qr_apply_qt_d", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp]),
    ("qr_apply_qt_s", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp]),
    ("qr_status", c_int, [c_vp, ctypes.POINTER(c_int), c_vp]),
    ("qr_workspace_p", c_int, [c_i64, c_i64, c_int, c_int, c_int, c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("qr_factor_p_d", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("qr_factor_p_s", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("qr_apply_workspace_p", c_int, [c_i64, c_i64, c_i64, c_int, c_int, ctypes.POINTER(c_i64)]),
    ("qr_apply_qt_p_d", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp,
                                c_i64, c_vp]),
    ("qr_apply_qt_p_s", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp,
                                c_i64, c_vp]),
    ("qr_apply_workspace", c_int, [c_i64, c_i64, c_i64, c_int, ctypes.POINTER(c_i64)]),
    ("qr_apply_qt_ws_d", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp, c_i64,
                                 c_vp]),
    ("qr_apply_qt_ws_s", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_vp, c_vp, c_i64, c_int, c_vp, c_i64,
                                 c_vp]),
    ("qr_batched_plan", c_int, [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_int, c_int, c_int,
                                ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("qr_factor_batched_d", c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("qr_factor_batched_s", c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("qr_batched_set_class", c_int, [c_int, c_int, c_int, c_int]),
    ("qr_batched_clear_classes", c_int, [c_int]),
    ("qr_batched_status", c_int, [c_vp, ctypes.POINTER(c_int), c_vp]),
    ("qr_solve_ls_workspace", c_int, [c_i64, c_i64, c_i64, c_int, c_int, c_int, c_int, ctypes.POINTER(c_i64)]),
    ("qr_solve_ls", c_int, [c_i64, c_i64, c_i64, c_vp, c_i64, c_vp, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_int,
                            c_int, c_dbl, ctypes.POINTER(c_int), c_vp, c_i64, c_vp]),
    ("qr_set_option", c_int, [c_int, c_i64]),
    ("qr_set_trace", c_int, [c_vp, c_i64]),
    ("qr_set_task_costs", c_int, [c_int, c_int, c_int, ctypes.POINTER(c_dbl)]),
    ("qr_get_option", c_i64, [c_int]),
    ("qr_task_count", c_i64, [c_i64, c_i64, c_int, c_int, c_int]),
    ("qr_last_kernel_ms", c_int, [ctypes.POINTER(ctypes.c_float)]),
    ("qr_load_table", c_int, [ctypes.c_char_p]),
    ("qr_mlp_workspace", c_int, [c_int, ctypes.POINTER(c_i64)]),
    ("qr_mlp_forward", c_int, [c_int, c_vp, c_vp, c_vp, c_vp]),
    ("qr_mlp_grad", c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    ("qr_mlp_adam_step", c_int, [c_vp, c_vp, c_vp, c_vp, c_int, ctypes.c_float, c_vp]),
    ("qr_mlp_train", c_int, [c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_int, ctypes.c_float, c_vp, c_vp, c_vp]),
    ("qr_clear_tables", c_int, []),
    ("qr_lookup", c_int, [c_i64, c_i64, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    ("qr_lookup_sms", c_int, [c_i64, c_i64, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                              ctypes.POINTER(c_int)]),
    ("qr_lookup_p", c_int, [c_i64, c_i64, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    ("qr_tune_grid", c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    ("qr_tune_preselect", c_int, [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), ctypes.POINTER(c_dbl), c_int,
                                  c_int, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    ("qr_tune_payg", c_int, [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_dbl), ctypes.POINTER(c_int)]),
    ("qr_tune_nearest", c_i64, [c_i64, ctypes.POINTER(c_i64), c_int]),
    ("qr_step1_workspace", c_int, [c_int, c_int, c_int, ctypes.POINTER(c_i64)]),
    ("qr_step1_time", c_int, [c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp,
                              c_i64, c_vp]),
    ("qr_tune_workspace", c_int, [c_i64, c_i64, c_int, ctypes.POINTER(c_i64)]),
    ("qr_time_factor", c_int, [c_i64, c_i64, c_int, c_int, c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl),
                               c_vp, c_i64, c_vp]),
    ("qr_time_factor_p", c_int, [c_i64, c_i64, c_int, c_int, c_int, c_int, c_int, ctypes.POINTER(c_dbl),
                                 ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("qr_tune", c_int, [ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), c_int, c_int, c_int, c_int, c_int, c_int,
                        ctypes.c_char_p, ctypes.c_char_p, c_vp, c_i64, ctypes.POINTER(c_dbl), c_vp]),
    ("qr_factor_mixed_s", c_int, [c_i64, c_i64, c_vp, c_i64, c_int, c_int, c_int, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("chol_workspace", c_int, [c_i64, c_int, ctypes.POINTER(c_i64)]),
    ("chol_factor_d", c_int, [c_i64, c_vp, c_i64, c_int, c_vp, c_i64, c_vp]),
    ("chol_status", c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_i64), c_vp]),
    ("chol_task_count_n", c_i64, [c_i64, c_int]),
    ("chol_step1_workspace", c_int, [c_int, ctypes.POINTER(c_i64)]),
    ("chol_step1_time", c_int, [c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("chol_time_factor", c_int, [c_i64, c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("chol_tune_workspace", c_int, [c_i64, ctypes.POINTER(c_i64)]),
    ("chol_tune", c_int, [ctypes.POINTER(c_i64), c_int, c_int, c_int, ctypes.c_char_p, ctypes.c_char_p, c_vp, c_i64,
                          ctypes.POINTER(c_dbl), c_vp]),
    ("chol_load_table", c_int, [ctypes.c_char_p]),
    ("chol_lookup", c_int, [c_i64, ctypes.POINTER(c_int)]),
    ("lu_workspace", c_int, [c_i64, c_int, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    ("lu_factor_d", c_int, [c_i64, c_vp, c_i64, c_int, c_vp, c_vp, c_i64, c_vp]),
    ("lu_status", c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_i64), c_vp]),
    ("lu_task_count_n", c_i64, [c_i64, c_int]),
    ("lu_step1_workspace", c_int, [c_int, ctypes.POINTER(c_i64)]),
    ("lu_step1_time", c_int, [c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("lu_time_factor", c_int, [c_i64, c_int, c_int, ctypes.POINTER(c_dbl), ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("lu_tune_workspace", c_int, [c_i64, ctypes.POINTER(c_i64)]),
    ("lu_tune", c_int, [ctypes.POINTER(c_i64), c_int, c_int, c_int, ctypes.c_char_p, ctypes.c_char_p, c_vp, c_i64,
                        ctypes.POINTER(c_dbl), c_vp]),
    ("lu_load_table", c_int, [ctypes.c_char_p]),
    ("lu_lookup", c_int, [c_i64, ctypes.POINTER(c_int)]),
    ("lu_clear_table", c_int, []),
    ("qr_model_propose", c_int, [c_i64, c_i64, c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                 ctypes.POINTER(c_dbl), c_vp, c_i64, c_vp]),
    ("qr_peak_fp64", c_int, [ctypes.POINTER(c_dbl), c_vp]),
]


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load (building first if needed) libtileqr.so and set its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libtileqr.so is not built (run __graft_entry__.build())")
    L = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(rc, what):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (what, rc))
    return rc
