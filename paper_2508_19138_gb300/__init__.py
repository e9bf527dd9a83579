"""GB300 (sm_103a) block-tridiagonal selected inversion: recursive Green's function sweeps for
the G and W systems of NEGF+GW with Sancho-Rubio contacts.

The compute is in libbt_selinv.so (hand-written CUDA behind a C ABI, include/bt_selinv.h);
this package is a thin ctypes binding with the same entry-point names.  PyTorch provides device
memory and streams only."""
from .api import *  # noqa: F401,F403
from ._native import (BT_ERR_BUDGET, BT_ERR_CANCELLED, BT_ERR_CUDA, BT_ERR_INVALID_ARG, BT_ERR_NONFINITE,  # noqa: F401
                      BT_ERR_NOT_CONVERGED, BT_ERR_OOM, BT_CONV_CONJ_B, BT_CONV_REVERSE_B, BT_ERR_SINGULAR, BT_ERR_TIMEOUT, BT_ERR_UNSUPPORTED,
                      BT_FP64, BT_LAYOUT_BLOCKS, BT_LAYOUT_DIAGVEC, BT_LAYOUT_PACKED_UPPER, BT_OK, BT_OP_C, BT_OP_N, BT_SPLIT,
                      BT_SYM_ANTIHERMITIAN, BT_SYM_GENERAL, BT_SYM_HERMITIAN, BT_SYS_G, BT_SYS_W, STATUS_NAMES)
from .serving import (Server, bt_server_create, bt_server_destroy, bt_server_get_stats,  # noqa: F401,E402
                      bt_server_poll, bt_server_submit, bt_server_wait)
