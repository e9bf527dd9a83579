"""Project-written autotuner for the batching and kernel-shape parameters of a solve.

The throughput of a solve depends on how many energies one batched launch carries
(`max_energies`, the chunk: small chunks leave SMs idle in the per-matrix inversion panels and
in the GEMM grids, large ones cost workspace), on the output tile of the FP64 products
(`gemm_tile`, 16 or 32) and on the panel width of the blocked inversions (`inv_panel`: narrow
panels shorten the serial column loop, wide ones need fewer update launches).  The tuner times
the candidates on the actual device shape one parameter at a time (the chunk first, then the tile
with the chosen chunk, then the panel), keeps the fastest within an HBM budget, and caches the
choice in a JSON file keyed by (GPU name, nb, bs, precision, split scope), so later runs reuse it
without timing."""
from __future__ import annotations

import json
import os
import time
from typing import Callable, Dict, Iterable, Optional

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune.json")


def cache_key(gpu: str, nb: int, bs: int, precision: int, split_scope: int) -> str:
    return f"{gpu}|nb={nb}|bs={bs}|p={precision}|scope={split_scope}"


def load_cache(path: str = DEFAULT_CACHE) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict], path: str = DEFAULT_CACHE) -> None:
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def choose(measure: Callable[[int], float], candidates: Iterable[int], fits: Callable[[int], bool]) -> dict:
    """measure(chunk) -> seconds per energy; returns {"best": chunk, "table": {chunk: s/energy}}.
    Candidates that do not fit the budget are skipped; ties keep the smaller chunk."""
    table = {}
    for c in sorted(set(int(x) for x in candidates)):
        if c < 1 or not fits(c):
            continue
        table[c] = float(measure(c))
    if not table:
        raise ValueError("no candidate chunk fits the budget")
    best = min(table, key=lambda c: (table[c], c))
    return {"best": best, "table": {str(k): v for k, v in table.items()}}


def coordinate_descent(measure: Callable[[dict], float], space: Dict[str, Iterable], start: dict,
                       fits: Callable[[dict], bool]) -> dict:
    """Tunes one parameter at a time in the order of `space` (name -> candidates), the others
    held at their best values so far; measure(params) -> seconds per energy.  Returns
    {"best": params, "table": {name: {value: s/energy}}}; ties keep the earlier candidate."""
    best = dict(start)
    tables = {}
    for name, cands in space.items():
        table = {}
        for v in cands:
            trial = dict(best, **{name: v})
            if not fits(trial):
                continue
            table[v] = float(measure(trial))
        if not table:
            raise ValueError(f"no candidate of {name} fits the budget")
        best[name] = min(table, key=lambda v: (table[v], list(table).index(v)))
        tables[name] = {str(k): t for k, t in table.items()}
    return {"best": best, "table": tables}


def tune_g(nb: int, bs: int, H_diag, H_upper, energies, sigR=None, sigL=None, sigG=None, eta: float = 1e-6,
           kT: float = 0.025, mu_left: float = 0.0, mu_right: float = 0.0, precision: int = 0, split_scope: int = 0,
           chunks=(4, 8, 16, 32), tiles=(32, 16), panels=(0, 8), hbm_budget_bytes: Optional[int] = None,
           cache_path: str = DEFAULT_CACHE, reuse: bool = True) -> dict:
    """Chunk, FP64 output tile and inversion panel width for this device shape (coordinate
    descent, each candidate timed by a warm-up solve and a timed solve of 2 chunks of energies).
    Returns {"best": {"max_energies", "gemm_tile", "inv_panel"}, "table": ..., "cached": bool}."""
    import torch

    from . import api
    from .highlevel import GSolver
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, nb, bs, precision, split_scope) + "|shape"
    cache = load_cache(cache_path)
    if reuse and key in cache:
        return dict(cache[key], cached=True)

    def fits(p):
        if hbm_budget_bytes is None:
            return True
        d = api.make_desc(nb, bs, p["max_energies"], precision=precision, split_scope=split_scope, eta=eta, kT=kT)
        return api.bt_selinv_workspace_bytes(d) <= hbm_budget_bytes

    def measure(p):
        c = p["max_energies"]
        solver = GSolver(nb, bs, c, eta, kT, mu_left, mu_right, precision=precision, split_scope=split_scope,
                         gemm_tile=p["gemm_tile"], inv_panel=p["inv_panel"])
        solver.set_inputs(H_diag, H_upper, sigR, sigL, sigG)
        n = min(len(energies), 2 * c)
        outs, status = solver.allocate_outputs(n)
        rng = (0, n) if sigR is not None else None
        solver.solve(energies[:n], outs, status, sig_range=rng)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.solve(energies[:n], outs, status, sig_range=rng)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n
        solver.close()
        return dt

    res = coordinate_descent(measure, {"max_energies": chunks, "gemm_tile": tiles, "inv_panel": panels},
                             {"max_energies": chunks[0], "gemm_tile": 0, "inv_panel": 0}, fits)
    cache[key] = res
    save_cache(cache, cache_path)
    return dict(res, cached=False)


def tune_g_chunk(nb: int, bs: int, H_diag, H_upper, energies, sigR=None, sigL=None, sigG=None, eta: float = 1e-6,
                 kT: float = 0.025, mu_left: float = 0.0, mu_right: float = 0.0, precision: int = 0,
                 split_scope: int = 0, candidates=(4, 8, 16, 32), hbm_budget_bytes: Optional[int] = None,
                 cache_path: str = DEFAULT_CACHE, reuse: bool = True) -> dict:
    """Times bt_selinv_solve on `energies` (one solve per candidate chunk, after a warm-up solve)
    and returns {"best": chunk, "table": {...}, "cached": bool}."""
    import torch

    from . import api
    from .highlevel import GSolver
    gpu = torch.cuda.get_device_name()
    key = cache_key(gpu, nb, bs, precision, split_scope)
    cache = load_cache(cache_path)
    if reuse and key in cache:
        return dict(cache[key], cached=True)

    def fits(c):
        if hbm_budget_bytes is None:
            return True
        d = api.make_desc(nb, bs, c, precision=precision, split_scope=split_scope, eta=eta, kT=kT)
        return api.bt_selinv_workspace_bytes(d) <= hbm_budget_bytes

    def measure(c):
        solver = GSolver(nb, bs, c, eta, kT, mu_left, mu_right, precision=precision, split_scope=split_scope)
        solver.set_inputs(H_diag, H_upper, sigR, sigL, sigG)
        n = min(len(energies), 2 * c)
        outs, status = solver.allocate_outputs(n)
        solver.solve(energies[:n], outs, status, sig_range=(0, n) if sigR is not None else None)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solver.solve(energies[:n], outs, status, sig_range=(0, n) if sigR is not None else None)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / n
        solver.close()
        return dt

    res = choose(measure, candidates, fits)
    cache[key] = res
    save_cache(cache, cache_path)
    return dict(res, cached=False)
