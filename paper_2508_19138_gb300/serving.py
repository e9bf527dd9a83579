"""Binding of the serving entry points (bt_server_*): argument marshalling only."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _native as N
from .api import BT, BTError, BTOut, _ptr

__all__ = ["Server", "bt_server_create", "bt_server_submit", "bt_server_poll", "bt_server_wait",
           "bt_server_get_stats", "bt_server_destroy"]


class Server:
    """Owns a bt_server handle and keeps each request's tensors alive until it is done."""

    def __init__(self, handle):
        self.handle = handle
        self.keep = {}

    def close(self):
        if self.handle:
            N.load().bt_server_destroy(self.handle)
            self.handle = None
            self.keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bt_server_create(hbm_budget_bytes: int, max_active: int = 4, max_energies_per_chunk: int = 16,
                     precision: int = N.BT_FP64, split_slices: int = 0, device: int = 0, split_scope: int = 0,
                     max_retries: int = 1, max_skips: int = 0, graph: bool = False) -> Server:
    d = N.bt_server_desc(hbm_budget_bytes, max_active, max_energies_per_chunk, precision, split_slices, device,
                         split_scope, max_retries, max_skips, 1 if graph else 0)
    h = C.c_void_p(None)
    rc = N.load().bt_server_create(C.byref(d), C.byref(h))
    if rc != N.BT_OK:
        raise BTError(rc, "bt_server_create")
    return Server(h.value)


def _bt_struct(b: Optional[BT]) -> N.bt_bt:
    return b.struct("cuda") if b is not None else N.bt_bt()


def _out_struct(o: Optional[BTOut]) -> N.bt_bt_out:
    return o.struct("cuda") if o is not None else N.bt_bt_out()


def bt_server_submit(srv: Server, nb: int, bs: int, H: BT, energies, status, outR: Optional[BTOut] = None,
                     outL: Optional[BTOut] = None, outG: Optional[BTOut] = None, S: Optional[BT] = None,
                     sigR: Optional[BT] = None, sigL: Optional[BT] = None, sigG: Optional[BT] = None,
                     eta: float = 1e-6, kT: float = 0.025, mu_left: float = 0.0, mu_right: float = 0.0,
                     obc: bool = True) -> int:
    import torch
    E = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    r = N.bt_request(nb, bs, len(E), _bt_struct(H), _bt_struct(S), _bt_struct(sigR), _bt_struct(sigL),
                     _bt_struct(sigG), E.ctypes.data_as(C.POINTER(C.c_double)), eta, kT, mu_left, mu_right,
                     1 if obc else 0, _out_struct(outR), _out_struct(outL), _out_struct(outG),
                     _ptr(status, torch.int32))
    t = C.c_longlong(0)
    rc = N.load().bt_server_submit(srv.handle, C.byref(r), C.byref(t))
    if rc != N.BT_OK:
        raise BTError(rc, "bt_server_submit")
    srv.keep[t.value] = (H, S, sigR, sigL, sigG, outR, outL, outG, status)
    return t.value


def bt_server_poll(srv: Server, ticket: int) -> int:
    st = C.c_int(0)
    rc = N.load().bt_server_poll(srv.handle, ticket, C.byref(st))
    if st.value >= 2:  # done or failed: the server no longer touches the request's tensors
        srv.keep.pop(ticket, None)
    if rc != N.BT_OK:
        raise BTError(rc, "bt_server_poll")
    return st.value


def bt_server_wait(srv: Server, ticket: int, timeout_s: float = 600.0) -> int:
    st = C.c_int(0)
    rc = N.load().bt_server_wait(srv.handle, ticket, timeout_s, C.byref(st))
    if st.value >= 2:
        srv.keep.pop(ticket, None)
    if rc != N.BT_OK:
        raise BTError(rc, f"bt_server_wait (state {st.value})")
    return st.value


def bt_server_get_stats(srv: Server) -> dict:
    s = N.bt_server_stats()
    rc = N.load().bt_server_get_stats(srv.handle, C.byref(s))
    if rc != N.BT_OK:
        raise BTError(rc, "bt_server_get_stats")
    return {k: getattr(s, k) for k, _ in N.bt_server_stats._fields_}


def bt_server_destroy(srv: Server) -> None:
    srv.close()
