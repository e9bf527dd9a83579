"""Thin Python binding of include/bt_selinv.h: the same entry-point names, argument marshalling only.

Tensors are passed by pointer (``tensor.data_ptr()``); device entry points require CUDA tensors
and use the current torch stream unless one is given.  Every call raises BTError on a non-OK
status (with the library's last-error text)."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _native as N

__all__ = [
    "BTError", "BT", "BTOut", "Context", "make_desc", "bt_selinv_workspace_bytes", "bt_selinv_create",
    "bt_selinv_solve", "bt_selinv_solve_host", "bt_selinv_destroy", "bt_selinv_last_error", "bt_selinv_get_stats",
    "bt_zgemm_batched", "bt_split_zgemm_workspace_bytes", "bt_split_zgemm_batched", "bt_zinv_workspace_bytes",
    "bt_zinv_batched", "bt_zinv_batched_noalloc", "bt_decimate_workspace_bytes", "bt_decimate_batched", "library",
    "bt_debug_split_stall", "bt_debug_fp64_rate", "bt_debug_panel_cluster", "bt_debug_split_profile", "bt_debug_cache_config", "bt_debug_split_pair", "bt_debug_split_sched", "bt_debug_split_schedule", "bt_debug_mma_issue_rate", "bt_energy_convolve",
]


class BTError(RuntimeError):
    def __init__(self, status: int, msg: str = ""):
        self.status = status
        super().__init__(f"{N.STATUS_NAMES.get(status, status)}: {msg}")


def library():
    """The loaded libbt_selinv.so (ctypes.CDLL)."""
    return N.load()


def _torch():
    import torch
    return torch


def _ptr(t, dtype=None, device: Optional[str] = "cuda"):
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if device == "cuda" and not t.is_cuda:
        raise ValueError("device entry point needs a CUDA tensor")
    if device == "cpu" and t.is_cuda:
        raise ValueError("host entry point needs a CPU tensor")
    return t.data_ptr()


def _stream(stream):
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(rc: int, ctx=None, what: str = ""):
    if rc != N.BT_OK:
        msg = bt_selinv_last_error(ctx) if ctx is not None or what == "create" else ""
        raise BTError(rc, f"{what}: {msg}" if what else msg)


class BT:
    """A block-tridiagonal input operand (keeps its tensors alive)."""

    def __init__(self, diag, upper=None, lower=None, layout: int = N.BT_LAYOUT_BLOCKS,
                 symmetry: int = N.BT_SYM_HERMITIAN, per_energy: bool = False):
        self.diag, self.upper, self.lower = diag, upper, lower
        self.layout, self.symmetry, self.per_energy = layout, symmetry, per_energy

    def struct(self, device="cuda") -> N.bt_bt:
        torch = _torch()
        return N.bt_bt(_ptr(self.diag, torch.complex128, device), _ptr(self.upper, torch.complex128, device),
                       _ptr(self.lower, torch.complex128, device), self.layout, self.symmetry,
                       1 if self.per_energy else 0)


class BTOut:
    """Output operand: [E][nb][bs][bs] diag, [E][nb-1][bs][bs] upper / lower (None = not written);
    layout BT_LAYOUT_DIAGVEC: diag is [E][nb][bs] (diagonal entries of the diagonal blocks);
    BT_LAYOUT_PACKED_UPPER (lesser/greater, symmetrised): diag is [E][nb][bs (bs + 1) / 2], the upper
    triangle of each anti-Hermitian block row by row (entry (r, c >= r) at r bs - r (r - 1) / 2 + (c - r))."""

    def __init__(self, diag=None, upper=None, lower=None, layout: int = N.BT_LAYOUT_BLOCKS):
        self.diag, self.upper, self.lower, self.layout = diag, upper, lower, layout

    def struct(self, device="cuda") -> N.bt_bt_out:
        torch = _torch()
        return N.bt_bt_out(_ptr(self.diag, torch.complex128, device), _ptr(self.upper, torch.complex128, device),
                           _ptr(self.lower, torch.complex128, device), self.layout)


def make_desc(nb: int, bs: int, max_energies: int, system: int = N.BT_SYS_G, precision: int = N.BT_FP64,
              split_slices: int = 0, symmetrize: bool = True, obc: bool = True, eta: float = 1e-6,
              kT: float = 0.025, mu_left: float = 0.0, mu_right: float = 0.0, decim_tol: float = 1e-14,
              decim_maxit: int = 100, hbm_budget_bytes: int = 0, obc_memo: bool = False, memo_nfpi: int = 0,
              memo_capacity: int = 0, split_scope: int = 0, graph: bool = False,
              decim_newton_after: int = 0, gemm_tile: int = 0, inv_panel: int = 0) -> N.bt_selinv_desc:
    return N.bt_selinv_desc(nb, bs, max_energies, system, precision, split_slices, 1 if symmetrize else 0,
                            1 if obc else 0, eta, kT, mu_left, mu_right, decim_tol, decim_maxit, hbm_budget_bytes,
                            1 if obc_memo else 0, memo_nfpi, memo_capacity, split_scope, 1 if graph else 0,
                            decim_newton_after, gemm_tile, inv_panel)


class Context:
    """Owns a bt_ctx handle (destroyed on close / garbage collection)."""

    def __init__(self, handle: int, desc: N.bt_selinv_desc):
        self.handle = handle
        self.desc = desc

    def close(self):
        if self.handle:
            N.load().bt_selinv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def bt_selinv_workspace_bytes(desc: N.bt_selinv_desc) -> int:
    out = C.c_size_t(0)
    _check(N.load().bt_selinv_workspace_bytes(C.byref(desc), C.byref(out)), what="workspace_bytes")
    return out.value


def bt_selinv_create(desc: N.bt_selinv_desc, stream=None) -> Context:
    h = C.c_void_p(None)
    st = _stream(stream) if (stream is not None or _cuda_ok()) else 0
    rc = N.load().bt_selinv_create(C.byref(desc), C.c_void_p(st), C.byref(h))
    if rc != N.BT_OK:
        raise BTError(rc, "create: " + bt_selinv_last_error(None))
    return Context(h.value, desc)


def _cuda_ok() -> bool:
    try:
        return _torch().cuda.is_available()
    except Exception:
        return False


def _ref(x, device):
    return C.byref(x.struct(device)) if x is not None else None


def _solve(fn, ctx: Context, H, S, sigR, sigL, sigG, energies, outR, outL, outG, status, device):
    torch = _torch()
    E = np.ascontiguousarray(np.asarray(energies, dtype=np.float64))
    n = int(E.shape[0])
    structs = [x.struct(device) if x is not None else None for x in (H, S, sigR, sigL, sigG, outR, outL, outG)]
    refs = [C.byref(s) if s is not None else None for s in structs]
    st_ptr = _ptr(status, torch.int32, device)
    rc = fn(ctx.handle, refs[0], refs[1], refs[2], refs[3], refs[4], E.ctypes.data_as(C.POINTER(C.c_double)), n,
            refs[5], refs[6], refs[7], st_ptr)
    _check(rc, ctx, "solve")


def bt_selinv_solve(ctx: Context, H: BT, S: Optional[BT], sigR: Optional[BT], sigL: Optional[BT], sigG: Optional[BT],
                    energies: Sequence[float], outR: Optional[BTOut], outL: Optional[BTOut], outG: Optional[BTOut],
                    status) -> None:
    """Asynchronous device solve on the context's stream (see include/bt_selinv.h)."""
    _solve(N.load().bt_selinv_solve, ctx, H, S, sigR, sigL, sigG, energies, outR, outL, outG, status, "cuda")


def bt_selinv_solve_host(ctx: Context, H: BT, S: Optional[BT], sigR: Optional[BT], sigL: Optional[BT],
                         sigG: Optional[BT], energies: Sequence[float], outR: Optional[BTOut], outL: Optional[BTOut],
                         outG: Optional[BTOut], status) -> None:
    """Synchronous solve on HOST tensors (copied to the device inside the call)."""
    _solve(N.load().bt_selinv_solve_host, ctx, H, S, sigR, sigL, sigG, energies, outR, outL, outG, status, "cpu")


def bt_selinv_destroy(ctx: Context) -> None:
    ctx.close()


def bt_selinv_last_error(ctx: Optional[Context]) -> str:
    h = ctx.handle if isinstance(ctx, Context) else None
    s = N.load().bt_selinv_last_error(h)
    return s.decode() if s else ""


def bt_selinv_get_stats(ctx: Context) -> dict:
    st = N.bt_stats()
    _check(N.load().bt_selinv_get_stats(ctx.handle, C.byref(st)), ctx, "get_stats")
    return {k: getattr(st, k) for k, _ in N.bt_stats._fields_}


def bt_zgemm_batched(m, n, k, alpha, A, lda, strideA, opA, B, ldb, strideB, opB, beta, Cm, ldc, strideC, batch,
                     stream=None) -> None:
    torch = _torch()
    alpha, beta = complex(alpha), complex(beta)
    rc = N.load().bt_zgemm_batched(m, n, k, alpha.real, alpha.imag, _ptr(A, torch.complex128), lda, strideA, opA,
                                   _ptr(B, torch.complex128), ldb, strideB, opB, beta.real, beta.imag,
                                   _ptr(Cm, torch.complex128), ldc, strideC, batch, _stream(stream))
    _check(rc, None, "zgemm")


def bt_split_zgemm_workspace_bytes(m, n, k, slices, batch) -> int:
    out = C.c_size_t(0)
    _check(N.load().bt_split_zgemm_workspace_bytes(m, n, k, slices, batch, C.byref(out)), None, "split ws")
    return out.value


def bt_split_zgemm_batched(m, n, k, alpha, A, lda, strideA, opA, B, ldb, strideB, opB, beta, Cm, ldc, strideC, batch,
                           slices, workspace=None, stream=None) -> None:
    torch = _torch()
    alpha, beta = complex(alpha), complex(beta)
    nbytes = bt_split_zgemm_workspace_bytes(m, n, k, slices, batch)
    if workspace is None and nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=Cm.device)
    rc = N.load().bt_split_zgemm_batched(m, n, k, alpha.real, alpha.imag, _ptr(A, torch.complex128), lda, strideA, opA,
                                         _ptr(B, torch.complex128), ldb, strideB, opB, beta.real, beta.imag,
                                         _ptr(Cm, torch.complex128), ldc, strideC, batch, slices,
                                         _ptr(workspace), nbytes if workspace is not None else 0, _stream(stream))
    _check(rc, None, "split_zgemm")


def bt_zinv_workspace_bytes(n, batch) -> int:
    out = C.c_size_t(0)
    _check(N.load().bt_zinv_workspace_bytes(n, batch, C.byref(out)), None, "zinv ws")
    return out.value


def bt_zinv_batched(n, A, strideA, batch, info, workspace=None, stream=None) -> None:
    torch = _torch()
    nbytes = bt_zinv_workspace_bytes(n, batch)
    if workspace is None and nbytes:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=A.device)
    rc = N.load().bt_zinv_batched(n, _ptr(A, torch.complex128), strideA, batch, _ptr(info, torch.int32),
                                  _ptr(workspace), nbytes if workspace is not None else 0, _stream(stream))
    _check(rc, None, "zinv")


def bt_zinv_batched_noalloc(n, A, strideA, batch, info, stream=None) -> None:
    """In-place batched inverse whose scratch is a fixed array inside the library (for callers
    that must not allocate device memory at this point); raises BTError(BT_ERR_BUDGET) when the
    request needs more than BT_ZINV_NOALLOC_SCRATCH_BYTES of scratch."""
    torch = _torch()
    rc = N.load().bt_zinv_batched_noalloc(n, _ptr(A, torch.complex128), strideA, batch, _ptr(info, torch.int32),
                                          _stream(stream))
    _check(rc, None, "zinv_noalloc")


def bt_energy_convolve(n_elem, na, nb, A, lda, B, ldb, C, ldc, scale=1.0, m0=0, n_out=None, flags=0,
                       stream=None) -> None:
    """Element-wise energy convolution (Sec. 4.4, Eq. 3) of energy-major complex128 device arrays:
    C[m - m0][e] = scale * sum_k A[m - k][e] * B'[k][e] for m0 <= m < m0 + n_out (see the header)."""
    torch = _torch()
    if n_out is None:
        n_out = na + nb - 1 - m0
    sc = complex(scale)
    rc = N.load().bt_energy_convolve(n_elem, na, nb, m0, n_out, _ptr(A, torch.complex128), lda,
                                     _ptr(B, torch.complex128), ldb, _ptr(C, torch.complex128), ldc, sc.real, sc.imag,
                                     flags, _stream(stream))
    _check(rc, None, "energy_convolve")


def bt_debug_fp64_rate(which: int, iters: int = 4096, stream=None) -> dict:
    """FP64 multiply-add rate on registers only: which 0 = DFMA, 1 = DMMA (mma.sync m8n8k4 f64)."""
    t, ms = C.c_double(0.0), C.c_double(0.0)
    _check(N.load().bt_debug_fp64_rate(which, iters, C.byref(t), C.byref(ms), _stream(stream)), None, "fp64_rate")
    return {"tflops": t.value, "ms": ms.value}


SPLIT_PROFILE_SLOTS = ("mma_wait_full", "mma_wait_acc", "mma_loop", "tma_wait_empty", "epi_drain", "epi_write",
                       "tiles")


def bt_debug_split_profile(enable: bool):
    """Measurement aid: start (True) or stop (False) the tensor-core GEMM's wait counters; on stop
    returns them as a dict of SM cycles summed over CTAs (SPLIT_PROFILE_SLOTS)."""
    buf = (C.c_ulonglong * len(SPLIT_PROFILE_SLOTS))()
    _check(N.load().bt_debug_split_profile(1 if enable else 0, buf, len(SPLIT_PROFILE_SLOTS)), None, "split_profile")
    return None if enable else dict(zip(SPLIT_PROFILE_SLOTS, [int(v) for v in buf]))


def bt_debug_mma_issue_rate(busy_warps: int, wait: bool = False, stream=None) -> float:
    """Measurement aid: tensor-pipe busy fraction of one MMA-issuing thread per SM next to
    busy_warps warps of multiply-add chains (wait: a ring-stage wait per K block)."""
    f = C.c_double(0.0)
    _check(N.load().bt_debug_mma_issue_rate(int(busy_warps), 1 if wait else 0, C.byref(f), _stream(stream)), None,
           "mma_issue_rate")
    return f.value


def bt_debug_split_pair(mode: int) -> None:
    """Measurement aid: tensor-core GEMM CTA arrangement (1 = single CTAs, 2 = CTA pairs, 3 = CTA pairs
    with two K blocks per stage, 0 = default)."""
    N.load().bt_debug_split_pair(int(mode))


def bt_debug_split_sched(mode: int) -> None:
    """Measurement aid: tensor-core GEMM accumulation schedule (0 = merged weight classes, the
    default; 1 = one slice pair per accumulator)."""
    N.load().bt_debug_split_sched(int(mode))


def bt_debug_split_schedule(slices: int, k_blocks: int, mode: int = 0):
    """Host-only query of the tensor-core GEMM's accumulation schedule: (jobs, items, F) with jobs
    as rows (dual, first item, end item, first K block, end K block, cvt lane 0, cvt lane 1, 0)
    and items as rows (s, s2, t); None for unsupported arguments."""
    cap_j, cap_i = 256, 256
    jobs = (C.c_int * (8 * cap_j))()
    items = (C.c_int * (3 * cap_i))()
    F = C.c_int(0)
    n = N.load().bt_debug_split_schedule(int(slices), int(k_blocks), int(mode), jobs, cap_j, items, cap_i,
                                         C.byref(F))
    if n < 0:
        return None
    rows = [tuple(jobs[8 * g:8 * g + 8]) for g in range(n)]
    n_items = rows[-1][2] if rows else 0
    return rows, [tuple(items[3 * i:3 * i + 3]) for i in range(n_items)], F.value


def bt_debug_cache_config(config: int) -> None:
    """Measurement aid: preferred L1 / shared split (0 none, 1 shared, 2 L1, 3 equal)."""
    _check(N.load().bt_debug_cache_config(int(config)), None, "cache_config")


def bt_debug_panel_cluster(cl: int) -> None:
    """Measurement aid: force the Gauss-Jordan panel cluster size (2, 4 or 8; 0 = default)."""
    N.load().bt_debug_panel_cluster(int(cl))


def bt_debug_split_stall(ns: int, launches: int = -1) -> None:
    """Test hook: the next `launches` tensor-core GEMM launches (all when negative) first stall
    their MMA warp up to ns nanoseconds on a barrier nothing completes, so that the bounded-wait
    timeout path runs (ns = 0: off)."""
    N.load().bt_debug_split_stall(int(ns), int(launches))


def bt_decimate_workspace_bytes(bs, batch) -> int:
    out = C.c_size_t(0)
    _check(N.load().bt_decimate_workspace_bytes(bs, batch, C.byref(out)), None, "decimate ws")
    return out.value


def bt_decimate_batched(bs, batch, m, n, n_prime, tol, maxit, x, sigma, iters, info, workspace=None,
                        stream=None) -> None:
    torch = _torch()
    nbytes = bt_decimate_workspace_bytes(bs, batch)
    if workspace is None:
        workspace = torch.empty(nbytes, dtype=torch.uint8, device=m.device)
    rc = N.load().bt_decimate_batched(bs, batch, _ptr(m, torch.complex128), _ptr(n, torch.complex128),
                                      _ptr(n_prime, torch.complex128), tol, maxit, _ptr(x, torch.complex128),
                                      _ptr(sigma, torch.complex128), _ptr(iters, torch.int32), _ptr(info, torch.int32),
                                      _ptr(workspace), nbytes, _stream(stream))
    _check(rc, None, "decimate")
