"""Convenience layer over the C ABI: owns a context, device copies of the inputs and the output
tensors for one device size.  Pure marshalling: every arithmetic step runs in libbt_selinv.so."""
from __future__ import annotations

from typing import Optional

import numpy as np

from . import _native as N
from .api import (BT, BTOut, bt_selinv_create, bt_selinv_get_stats, bt_selinv_solve, bt_selinv_solve_host,
                  make_desc)


def _t(x, device):
    import torch
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.complex128).contiguous()
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex128))).to(device)


class GSolver:
    """Selected inversion of the electron system (Table 2, left column) for one device shape.

    Inputs: H_diag [nb,bs,bs], H_upper [nb-1,bs,bs] (Hermitian H), optional scattering
    self-energies as diagonal vectors [E,nb,bs] or full per-energy blocks [E,nb,bs,bs]."""

    def __init__(self, nb: int, bs: int, max_energies: int, eta: float, kT: float = 0.025, mu_left: float = 0.0,
                 mu_right: float = 0.0, obc: bool = True, precision: int = N.BT_FP64, split_slices: int = 0,
                 symmetrize: bool = True, decim_tol: float = 1e-14, decim_maxit: int = 100, stream=None,
                 hbm_budget_bytes: int = 0, device: str = "cuda", obc_memo: bool = False, memo_nfpi: int = 0,
                 memo_capacity: int = 0, split_scope: int = 0, graph: bool = False, decim_newton_after: int = 0,
                 gemm_tile: int = 0, inv_panel: int = 0):
        self.nb, self.bs, self.max_energies = nb, bs, max_energies
        self.device = device
        self.desc = make_desc(nb, bs, max_energies, N.BT_SYS_G, precision, split_slices, symmetrize, obc, eta, kT,
                              mu_left, mu_right, decim_tol, decim_maxit, hbm_budget_bytes, obc_memo, memo_nfpi,
                              memo_capacity, split_scope, graph, decim_newton_after, gemm_tile, inv_panel)
        self._own_stream = None
        self.graph = bool(graph)
        if graph and stream is None:
            import torch
            stream = torch.cuda.Stream()  # stream capture needs a non-default stream
            self._own_stream = stream
        self.stream = stream
        self.ctx = bt_selinv_create(self.desc, stream)
        self.H = self.S = self.sigR = self.sigL = self.sigG = None

    def set_inputs(self, H_diag, H_upper, sigR=None, sigL=None, sigG=None, H_lower=None):
        dev = self.device
        sym = N.BT_SYM_HERMITIAN if H_lower is None else N.BT_SYM_GENERAL
        self.H = BT(_t(H_diag, dev), _t(H_upper, dev) if self.nb > 1 else None,
                    _t(H_lower, dev) if H_lower is not None else None, N.BT_LAYOUT_BLOCKS, sym, False)

        def sig(x, symmetry):
            if x is None:
                return None
            x = _t(x, dev)
            if x.dim() == 3:
                return BT(x, None, None, N.BT_LAYOUT_DIAGVEC, symmetry, True)
            return BT(x, None, None, N.BT_LAYOUT_BLOCKS, symmetry, True)

        self.sigR = sig(sigR, N.BT_SYM_GENERAL)
        self.sigL = sig(sigL, N.BT_SYM_ANTIHERMITIAN)
        self.sigG = sig(sigG, N.BT_SYM_ANTIHERMITIAN)
        return self

    def energy_slice(self, e0: int, e1: int):
        """Inputs restricted to energies [e0, e1) (per-energy operands are views)."""
        out = []
        for s in (self.sigR, self.sigL, self.sigG):
            out.append(None if s is None else BT(s.diag[e0:e1], None, None, s.layout, s.symmetry, True))
        return out

    def allocate_outputs(self, n_energies: int, which=("R", "L", "G"), lower_R: bool = True, packed_lg: bool = False):
        """Device output tensors; packed_lg: lesser/greater diagonal blocks in packed upper-triangle
        storage ([E][nb][bs (bs + 1) / 2], BT_LAYOUT_PACKED_UPPER)."""
        import torch
        nb, bs, dev = self.nb, self.bs, self.device
        shape_d = (n_energies, nb, bs, bs)
        shape_p = (n_energies, nb, bs * (bs + 1) // 2)
        shape_o = (n_energies, max(nb - 1, 0), bs, bs)
        outs = {}
        for w in which:
            packed = packed_lg and w in ("L", "G")
            outs[w] = BTOut(torch.empty(shape_p if packed else shape_d, dtype=torch.complex128, device=dev),
                            torch.empty(shape_o, dtype=torch.complex128, device=dev) if nb > 1 else None,
                            torch.empty(shape_o, dtype=torch.complex128, device=dev)
                            if (w == "R" and lower_R and nb > 1) else None,
                            N.BT_LAYOUT_PACKED_UPPER if packed else N.BT_LAYOUT_BLOCKS)
        status = torch.empty(n_energies, dtype=torch.int32, device=dev)
        return outs, status

    def solve(self, energies, outs=None, status=None, sig_range=None):
        """Device solve (asynchronous).  Returns (outs, status)."""
        energies = np.asarray(energies, dtype=np.float64)
        if outs is None:
            outs, status = self.allocate_outputs(len(energies))
        sR, sL, sG = (self.sigR, self.sigL, self.sigG) if sig_range is None else self.energy_slice(*sig_range)
        if self._own_stream is not None:
            # the private stream of graph mode runs after what the caller queued on its stream (the
            # staging copies below and the solve read inputs the caller may just have produced), and
            # the caller's stream waits for the solve at the end
            import torch
            self._own_stream.wait_stream(torch.cuda.current_stream())
        bt_selinv_solve(self.ctx, self.H, self.S, sR, sL, sG, energies, outs.get("R"), outs.get("L"),
                        outs.get("G"), status)
        if self._own_stream is not None:
            torch.cuda.current_stream().wait_stream(self._own_stream)
        return outs, status

    def stats(self):
        return bt_selinv_get_stats(self.ctx)

    def close(self):
        self.ctx.close()


def g_solve_host(ctx, H_diag, H_upper, energies, sigR=None, sigL=None, sigG=None, which=("R", "L", "G"), pin=True):
    """Host-buffer solve through bt_selinv_solve_host; all tensors on the CPU."""
    import torch
    nb, bs = H_diag.shape[0], H_diag.shape[1]
    n = len(energies)

    def host(x):
        if x is None:
            return None
        t = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
        t = t.to(torch.complex128).contiguous()
        return t.pin_memory() if pin else t

    H = BT(host(H_diag), host(H_upper) if nb > 1 else None, None, N.BT_LAYOUT_BLOCKS, N.BT_SYM_HERMITIAN, False)

    def sig(x, symm):
        if x is None:
            return None
        t = host(x)
        return BT(t, None, None, N.BT_LAYOUT_DIAGVEC if t.dim() == 3 else N.BT_LAYOUT_BLOCKS, symm, True)

    outs = {}
    for w in which:
        mk = (lambda shape: torch.empty(shape, dtype=torch.complex128).pin_memory()) if pin else \
            (lambda shape: torch.empty(shape, dtype=torch.complex128))
        outs[w] = BTOut(mk((n, nb, bs, bs)), mk((n, nb - 1, bs, bs)) if nb > 1 else None,
                        mk((n, nb - 1, bs, bs)) if (w == "R" and nb > 1) else None)
    status = torch.zeros(n, dtype=torch.int32)
    bt_selinv_solve_host(ctx, H, None, sig(sigR, N.BT_SYM_GENERAL), sig(sigL, N.BT_SYM_ANTIHERMITIAN),
                         sig(sigG, N.BT_SYM_ANTIHERMITIAN), energies, outs.get("R"), outs.get("L"), outs.get("G"),
                         status)
    return outs, status
