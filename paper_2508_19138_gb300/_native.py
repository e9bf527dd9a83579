"""ctypes mirror of include/bt_selinv.h and the loader of libbt_selinv.so.

The library is the product: if it is missing this module raises (there is no fallback)."""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

BT_OK, BT_ERR_INVALID_ARG, BT_ERR_OOM, BT_ERR_BUDGET, BT_ERR_CUDA = 0, 1, 2, 3, 4
BT_ERR_SINGULAR, BT_ERR_NOT_CONVERGED, BT_ERR_NONFINITE, BT_ERR_TIMEOUT, BT_ERR_UNSUPPORTED = 5, 6, 7, 8, 9
BT_ERR_CANCELLED = 10
STATUS_NAMES = {0: "BT_OK", 1: "BT_ERR_INVALID_ARG", 2: "BT_ERR_OOM", 3: "BT_ERR_BUDGET", 4: "BT_ERR_CUDA",
                5: "BT_ERR_SINGULAR", 6: "BT_ERR_NOT_CONVERGED", 7: "BT_ERR_NONFINITE", 8: "BT_ERR_TIMEOUT",
                9: "BT_ERR_UNSUPPORTED", 10: "BT_ERR_CANCELLED"}
BT_SYS_G, BT_SYS_W = 0, 1
BT_CONV_REVERSE_B, BT_CONV_CONJ_B = 1, 2
BT_FP64, BT_SPLIT = 0, 1
BT_LAYOUT_BLOCKS, BT_LAYOUT_DIAGVEC, BT_LAYOUT_PACKED_UPPER = 0, 1, 2
BT_SYM_GENERAL, BT_SYM_HERMITIAN, BT_SYM_ANTIHERMITIAN = 0, 1, 2
BT_OP_N, BT_OP_C = 0, 1


class bt_bt(C.Structure):
    _fields_ = [("diag", C.c_void_p), ("upper", C.c_void_p), ("lower", C.c_void_p), ("layout", C.c_int),
                ("symmetry", C.c_int), ("per_energy", C.c_int)]


class bt_bt_out(C.Structure):
    _fields_ = [("diag", C.c_void_p), ("upper", C.c_void_p), ("lower", C.c_void_p), ("layout", C.c_int)]


class bt_selinv_desc(C.Structure):
    _fields_ = [("nb", C.c_int), ("bs", C.c_int), ("max_energies", C.c_int), ("system", C.c_int),
                ("precision", C.c_int), ("split_slices", C.c_int), ("symmetrize", C.c_int), ("obc", C.c_int),
                ("eta", C.c_double), ("kT", C.c_double), ("mu_left", C.c_double), ("mu_right", C.c_double),
                ("decim_tol", C.c_double), ("decim_maxit", C.c_int), ("hbm_budget_bytes", C.c_size_t),
                ("obc_memo", C.c_int), ("memo_nfpi", C.c_int), ("memo_capacity", C.c_int), ("split_scope", C.c_int),
                ("graph", C.c_int), ("decim_newton_after", C.c_int), ("gemm_tile", C.c_int), ("inv_panel", C.c_int)]


class bt_stats(C.Structure):
    _fields_ = [("solves", C.c_longlong), ("energies", C.c_longlong), ("decim_iterations", C.c_longlong),
                ("flops_model", C.c_double), ("workspace_bytes", C.c_size_t), ("kernel_launches", C.c_longlong),
                ("lead_iterations", C.c_longlong), ("fpi_iterations", C.c_longlong), ("memo_hits", C.c_longlong),
                ("newton_leads", C.c_longlong), ("newton_iterations", C.c_longlong)]


# exported names and their ctypes signatures (restype is bt_status unless noted)
_P = C.c_void_p
_I = C.c_int
_LL = C.c_longlong
_D = C.c_double
_SZ = C.c_size_t
SIGNATURES = {
    "bt_selinv_workspace_bytes": [C.POINTER(bt_selinv_desc), C.POINTER(C.c_size_t)],
    "bt_selinv_create": [C.POINTER(bt_selinv_desc), _P, C.POINTER(_P)],
    "bt_selinv_solve": [_P, C.POINTER(bt_bt), C.POINTER(bt_bt), C.POINTER(bt_bt), C.POINTER(bt_bt),
                        C.POINTER(bt_bt), C.POINTER(_D), _I, C.POINTER(bt_bt_out), C.POINTER(bt_bt_out),
                        C.POINTER(bt_bt_out), _P],
    "bt_selinv_solve_host": [_P, C.POINTER(bt_bt), C.POINTER(bt_bt), C.POINTER(bt_bt), C.POINTER(bt_bt),
                             C.POINTER(bt_bt), C.POINTER(_D), _I, C.POINTER(bt_bt_out), C.POINTER(bt_bt_out),
                             C.POINTER(bt_bt_out), _P],
    "bt_selinv_get_stats": [_P, C.POINTER(bt_stats)],
    "bt_selinv_destroy": [_P],
    "bt_selinv_last_error": [_P],
    "bt_zgemm_batched": [_I, _I, _I, _D, _D, _P, _I, _LL, _I, _P, _I, _LL, _I, _D, _D, _P, _I, _LL, _I, _P],
    "bt_split_zgemm_workspace_bytes": [_I, _I, _I, _I, _I, C.POINTER(C.c_size_t)],
    "bt_split_zgemm_batched": [_I, _I, _I, _D, _D, _P, _I, _LL, _I, _P, _I, _LL, _I, _D, _D, _P, _I, _LL, _I, _I,
                               _P, _SZ, _P],
    "bt_zinv_workspace_bytes": [_I, _I, C.POINTER(C.c_size_t)],
    "bt_zinv_batched": [_I, _P, _LL, _I, _P, _P, _SZ, _P],
    "bt_zinv_batched_noalloc": [_I, _P, _LL, _I, _P, _P],
    "bt_debug_split_stall": [C.c_ulonglong, C.c_longlong],
    "bt_debug_fp64_rate": [_I, _I, C.POINTER(_D), C.POINTER(_D), _P],
    "bt_debug_panel_cluster": [_I],
    "bt_debug_split_profile": [_I, C.POINTER(C.c_ulonglong), _I],
    "bt_debug_cache_config": [_I],
    "bt_debug_split_pair": [_I],
    "bt_debug_split_sched": [_I],
    "bt_debug_split_schedule": [_I, _I, _I, C.POINTER(_I), _I, C.POINTER(_I), _I, C.POINTER(_I)],
    "bt_debug_mma_issue_rate": [_I, _I, C.POINTER(_D), _P],
    "bt_energy_convolve": [_I, _I, _I, _I, _I, _P, _LL, _P, _LL, _P, _LL, _D, _D, _I, _P],
    "bt_decimate_workspace_bytes": [_I, _I, C.POINTER(C.c_size_t)],
    "bt_decimate_batched": [_I, _I, _P, _P, _P, _D, _I, _P, _P, _P, _P, _P, _SZ, _P],
}
RESTYPES = {"bt_selinv_last_error": C.c_char_p, "bt_debug_split_stall": None, "bt_debug_panel_cluster": None, "bt_debug_split_pair": None,
            "bt_debug_split_sched": None}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Load libbt_selinv.so (building it first if asked); raises if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError(f"{path} is missing: run paper_2508_19138_gb300.build.build() first "
                               "(the CUDA library is required; there is no CPU fallback)")
    lib = C.CDLL(path)
    for name, args in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = RESTYPES.get(name, C.c_int)
    _lib = lib
    return lib


# ---- serving ----
class bt_server_desc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int), ("max_energies_per_chunk", C.c_int),
                ("precision", C.c_int), ("split_slices", C.c_int), ("device", C.c_int), ("split_scope", C.c_int),
                ("max_retries", C.c_int), ("max_skips", C.c_int), ("graph", C.c_int)]


class bt_request(C.Structure):
    _fields_ = [("nb", C.c_int), ("bs", C.c_int), ("n_energies", C.c_int), ("H", bt_bt), ("S", bt_bt),
                ("sigR", bt_bt), ("sigL", bt_bt), ("sigG", bt_bt), ("energies_host", C.POINTER(C.c_double)),
                ("eta", C.c_double), ("kT", C.c_double), ("mu_left", C.c_double), ("mu_right", C.c_double),
                ("obc", C.c_int), ("outR", bt_bt_out), ("outL", bt_bt_out), ("outG", bt_bt_out),
                ("status_device", C.c_void_p)]


class bt_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("rejected", C.c_longlong), ("energies_done", C.c_longlong), ("queued", C.c_longlong),
                ("active", C.c_int), ("peak_active", C.c_int), ("p50_latency_s", C.c_double),
                ("p99_latency_s", C.c_double), ("mean_latency_s", C.c_double), ("busy_seconds", C.c_double),
                ("energies_per_s", C.c_double), ("peak_bytes", C.c_size_t), ("units_done", C.c_longlong),
                ("retries", C.c_longlong)]


SIGNATURES.update({
    "bt_server_create": [C.POINTER(bt_server_desc), C.POINTER(_P)],
    "bt_server_submit": [_P, C.POINTER(bt_request), C.POINTER(C.c_longlong)],
    "bt_server_poll": [_P, C.c_longlong, C.POINTER(C.c_int)],
    "bt_server_wait": [_P, C.c_longlong, C.c_double, C.POINTER(C.c_int)],
    "bt_server_get_stats": [_P, C.POINTER(bt_server_stats)],
    "bt_server_destroy": [_P],
})
