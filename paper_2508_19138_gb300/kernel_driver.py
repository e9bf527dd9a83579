"""Runs one building-block kernel of the library at a given launch shape, for profiling:

    python -m paper_2508_19138_gb300.kernel_driver --kernel zgemm --bs 416 --batch 32 --reps 3
    python -m paper_2508_19138_gb300.kernel_driver --kernel split --bs 416 --batch 32 --slices 6
    python -m paper_2508_19138_gb300.kernel_driver --kernel zinv --bs 416 --batch 32
    python -m paper_2508_19138_gb300.kernel_driver --kernel cublas --bs 416 --batch 16   # library reference
    python -m paper_2508_19138_gb300.kernel_driver --kernel conv --bs 416 --batch 512    # energy convolution of
        # the bs^2 element series of one diagonal block over `batch` energies (na = nb = batch)
    python -m paper_2508_19138_gb300.kernel_driver --kernel fp64rate --reps 4   # DFMA vs DMMA (FP64 tensor) rates
    python -m paper_2508_19138_gb300.kernel_driver --kernel mmaissue   # tcgen05.mma issue rate next to busy warps
    python -m paper_2508_19138_gb300.kernel_driver --kernel steptrace --precision split --split-scope 1 --batch 32
        # launch list of one solve step of the 40 x 416 nanoribbon (`batch` energies) from CUPTI
        # activity records (csrc/launch_trace.cpp): kernels, launches, device time, share

Inputs are random complex128 blocks already on the device; each kernel is launched `--reps`
times on the current stream and its mean time is printed (CUDA events)."""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    import paper_2508_19138_gb300 as pkg
    ap = argparse.ArgumentParser()
    ap.add_argument("--kernel", choices=["zgemm", "split", "zinv", "cublas", "conv", "fp64rate", "steptrace",
                                                 "mmaissue"],
                    required=True)
    ap.add_argument("--bs", type=int, default=416)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--slices", type=int, default=6)
    ap.add_argument("--k", type=int, default=0, help="inner dimension of the products (default: --bs)")
    ap.add_argument("--precision", choices=["fp64", "split"], default="split", help="steptrace: solve precision")
    ap.add_argument("--split-scope", type=int, default=1, help="steptrace: split scope")
    ap.add_argument("--graph", choices=["on", "off"], default="on", help="steptrace: graph mode")
    ap.add_argument("--warmup", type=int, default=2, help="steptrace: untraced steps first")
    ap.add_argument("--inv-panel", type=int, default=0, help="steptrace: inversion panel width (0 = default)")
    ap.add_argument("--cache-config", type=int, default=-1,
                    help="preferred L1 / shared split for the run (0 none, 1 shared, 2 L1, 3 equal; -1 untouched)")
    ap.add_argument("--split-pair", type=int, default=0,
                    help="split: 1 = single CTAs, 2 = CTA pairs (cta_group::2), 3 = pairs with two K blocks per "
                         "stage, 0 = default; with --check all three")
    ap.add_argument("--split-sched", type=int, default=0,
                    help="split: accumulation schedule, 0 = merged weight classes (default), 1 = one slice pair "
                         "per accumulator; --check compares both")
    ap.add_argument("--check", action="store_true",
                    help="split: compare the result of single CTAs and CTA pairs bitwise, and with torch")
    ap.add_argument("--split-profile", action="store_true",
                    help="split: also report the GEMM's wait counters (bt_debug_split_profile)")
    ap.add_argument("--panel-cluster", type=int, default=0,
                    help="zinv: force the panel cluster size (2, 4 or 8; 0 = default rule)")
    a = ap.parse_args()
    if a.kernel == "cublas":
        return cublas_reference(a)
    pkg.library()
    if a.panel_cluster:
        pkg.bt_debug_panel_cluster(a.panel_cluster)
    if a.cache_config >= 0:
        pkg.bt_debug_cache_config(a.cache_config)
    if a.kernel == "conv":
        return conv_driver(a, pkg)
    if a.kernel == "steptrace":
        return step_trace(a, pkg)
    if a.kernel == "mmaissue":
        rows = [{"busy_warps": bw, "wait": wt, "tensor_busy": pkg.bt_debug_mma_issue_rate(bw, wt)}
                for wt in (False, True) for bw in (0, 4, 8, 16)]
        print(json.dumps({"kernel": "mmaissue", "rows": rows}))
        return None
    if a.kernel == "fp64rate":
        out = {"kernel": "fp64rate"}
        for which, name in ((0, "dfma"), (1, "dmma")):
            r = pkg.bt_debug_fp64_rate(which, iters=max(1, a.reps) * 4096)
            out[name + "_tflops"], out[name + "_ms"] = r["tflops"], r["ms"]
        print(json.dumps(out))
        return None
    b, n = a.batch, a.bs
    kk = a.k if a.k > 0 and a.kernel != "zinv" else n
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(b, n, kk, dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn(b, kk, n, dtype=torch.complex128, device="cuda", generator=g)
    C = torch.empty(b, n, n, dtype=torch.complex128, device="cuda")
    ws = None
    if a.kernel == "split":
        ws = torch.empty(pkg.bt_split_zgemm_workspace_bytes(n, n, kk, a.slices, b), dtype=torch.uint8, device="cuda")
    info = torch.zeros(b, dtype=torch.int32, device="cuda")
    if a.kernel == "zinv":
        A += 4.0 * torch.eye(n, dtype=torch.complex128, device="cuda")
        ws = torch.empty(max(1, pkg.bt_zinv_workspace_bytes(n, b)), dtype=torch.uint8, device="cuda")
    Ainv = A.clone()

    if a.kernel == "split" and a.split_pair:
        pkg.bt_debug_split_pair(a.split_pair)
    if a.kernel == "split":
        pkg.bt_debug_split_sched(a.split_sched)
    check = None
    if a.kernel == "split" and a.check:
        outs = {}
        for mode in (1, 2, 3):
            pkg.bt_debug_split_pair(mode)
            C.zero_()
            pkg.bt_split_zgemm_batched(n, n, kk, 1.0, A, kk, n * kk, 0, B, n, kk * n, 0, 0.0, C, n, n * n, b,
                                       a.slices, workspace=ws)
            torch.cuda.synchronize()
            outs[mode] = C.clone()
        ref = torch.matmul(A, B)
        rel = (torch.linalg.norm(outs[2] - ref) / torch.linalg.norm(ref)).item()
        check = {"bitwise_equal": bool(torch.equal(outs[1], outs[2])),
                 "bitwise_equal_pair_kps2": bool(torch.equal(outs[1], outs[3])),
                 "max_abs_diff": (outs[1] - outs[2]).abs().max().item(), "rel_err_vs_torch_pair": rel,
                 "rel_err_vs_torch_single": (torch.linalg.norm(outs[1] - ref) / torch.linalg.norm(ref)).item()}
        # the other accumulation schedule (same CTA arrangement as the run)
        pkg.bt_debug_split_pair(a.split_pair)
        pkg.bt_debug_split_sched(1 - a.split_sched)
        C.zero_()
        pkg.bt_split_zgemm_batched(n, n, kk, 1.0, A, kk, n * kk, 0, B, n, kk * n, 0, 0.0, C, n, n * n, b,
                                   a.slices, workspace=ws)
        torch.cuda.synchronize()
        other = C.clone()
        pkg.bt_debug_split_sched(a.split_sched)
        C.zero_()
        pkg.bt_split_zgemm_batched(n, n, kk, 1.0, A, kk, n * kk, 0, B, n, kk * n, 0, 0.0, C, n, n * n, b,
                                   a.slices, workspace=ws)
        torch.cuda.synchronize()
        check["rel_err_vs_torch_other_sched"] = (torch.linalg.norm(other - ref) / torch.linalg.norm(ref)).item()
        check["rel_diff_between_scheds"] = (torch.linalg.norm(other - C) / torch.linalg.norm(C)).item()

    def run():
        if a.kernel == "zgemm":
            pkg.bt_zgemm_batched(n, n, kk, 1.0, A, kk, n * kk, 0, B, n, kk * n, 0, 0.0, C, n, n * n, b)
        elif a.kernel == "split":
            pkg.bt_split_zgemm_batched(n, n, kk, 1.0, A, kk, n * kk, 0, B, n, kk * n, 0, 0.0, C, n, n * n, b,
                                       a.slices, workspace=ws)
        else:
            Ainv.copy_(A)
            pkg.bt_zinv_batched(n, Ainv, n * n, b, info, workspace=ws)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    prof = None
    if a.kernel == "split" and a.split_profile:
        pkg.bt_debug_split_profile(True)
        for _ in range(a.reps):
            run()
        c = pkg.bt_debug_split_profile(False)
        loop = max(1, c["mma_loop"])
        prof = dict(c, frac_mma_wait_full=c["mma_wait_full"] / loop, frac_mma_wait_acc=c["mma_wait_acc"] / loop,
                    frac_tma_wait_empty=c["tma_wait_empty"] / loop, frac_epi_drain=c["epi_drain"] / loop,
                    frac_epi_write=c["epi_write"] / loop)
    flops = 8.0 * n * n * kk * b
    print(json.dumps({"kernel": a.kernel, "bs": n, "k": kk, "batch": b, "ms": ms, "fp64_eq_tflops": flops / ms / 1e9,
                      "slices": a.slices if a.kernel == "split" else None,
                      "panel_cluster": a.panel_cluster if a.kernel == "zinv" else None, "split_profile": prof,
                      "split_pair": a.split_pair if a.kernel == "split" else None,
                      "split_sched": a.split_sched if a.kernel == "split" else None, "check": check}))


def conv_flops(L):
    """Flops of one series' convolution by FFT: three transforms of 5 L log2 L and the spectral
    product (6 L), the usual count for radix-2 complex FFTs."""
    import math
    return 3 * 5 * L * math.log2(L) + 6 * L


def conv_driver(a, pkg):
    """bt_energy_convolve on bs^2 element series (one diagonal block) of `batch` energies each."""
    import torch
    n_elem, ne = a.bs * a.bs, a.batch
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(ne, n_elem, dtype=torch.complex128, device="cuda", generator=g)
    B = torch.randn(ne, n_elem, dtype=torch.complex128, device="cuda", generator=g)
    C = torch.empty(2 * ne - 1, n_elem, dtype=torch.complex128, device="cuda")

    def run():
        pkg.bt_energy_convolve(n_elem, ne, ne, A, n_elem, B, n_elem, C, n_elem)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    L = 1 << (2 * ne - 2).bit_length()
    flops = conv_flops(L) * n_elem
    moved = 16.0 * n_elem * (ne + ne + 2 * ne - 1)
    print(json.dumps({"kernel": "conv", "series": n_elem, "energies": ne, "L": L, "ms": ms,
                      "fp64_tflops": flops / ms / 1e9, "hbm_gbs": moved / ms / 1e6}))


def _short_name(name: str) -> str:
    """Kernel name without its argument list and namespaces (template arguments kept)."""
    name = name.replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
    depth, cut = 0, len(name)
    for i, ch in enumerate(name):  # the argument list: the first '(' outside template brackets
        if ch == "<":
            depth += 1
        elif ch == ">":
            depth -= 1
        elif ch == "(" and depth == 0 and i > 0:
            cut = i
            break
    head = name[:cut]
    if head.startswith("void "):
        head = head[5:]
    base, _, targs = head.partition("<")
    base = base.split("::")[-1]
    return (base + ("<" + targs if targs else "")).strip()


def _load_tracer():
    """Builds (once) and loads the CUPTI activity collector csrc/launch_trace.cpp: g++ against the
    toolkit's libcupti, next to the solver library."""
    import ctypes as C
    import os
    import subprocess
    here = os.path.dirname(os.path.abspath(__file__))
    so = os.path.join(here, "libbt_trace.so")
    src = os.path.join(here, "csrc", "launch_trace.cpp")
    if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
        libdirs = [d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "extras", "CUPTI", "lib64"))
                   if os.path.isdir(d)]
        incs = [d for d in (os.path.join(cuda, "include"), os.path.join(cuda, "extras", "CUPTI", "include"))
                if os.path.isdir(d)]
        cmd = (["g++", "-O2", "-std=c++17", "-shared", "-fPIC", src, "-o", so] + [f"-I{d}" for d in incs] +
               [f"-L{d}" for d in libdirs] + [f"-Wl,-rpath,{d}" for d in libdirs] + ["-lcupti"])
        subprocess.run(cmd, check=True)
    lib = C.CDLL(so)
    lib.bt_trace_get.argtypes = [C.c_int, C.c_char_p, C.c_int, C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]
    return lib


def step_trace(a, pkg):
    """One solve step of the 40 x 416 nanoribbon G system (a.batch energies strided across the
    512-energy grid, as the bench steps) after a.warmup untraced steps: the step's kernels from
    CUPTI activity records (device start / end of every kernel, memcpy and memset, graph-launched
    kernels included), aggregated per kernel; plus the step's time untraced (CUDA events).
    Kernels that run inside the body of a device-side conditional loop of a graph (the
    decimation, Newton and Stein loops of graph mode) produce no records: their time shows as
    one idle gap at the loop's entry.  --graph off lists every kernel (the loops then run from
    the host)."""
    import numpy as np
    import torch

    import synthetic
    from paper_2508_19138_gb300.highlevel import GSolver
    sysg = synthetic.nanoribbon_40x416()
    nE, eps = len(sysg.energies), a.batch
    nbat = max(1, nE // eps)
    perm = (np.arange(nbat)[:, None] + nbat * np.arange(eps)[None, :]).ravel()
    sysg = sysg.subset(perm)
    precision = pkg.BT_SPLIT if a.precision == "split" else pkg.BT_FP64
    stream = torch.cuda.Stream()
    solver = GSolver(sysg.nb, sysg.bs, eps, sysg.eta, sysg.kT, sysg.mu_left, sysg.mu_right, obc=True,
                     precision=precision, split_slices=a.slices, stream=stream, split_scope=a.split_scope,
                     graph=a.graph == "on", inv_panel=a.inv_panel)
    with torch.cuda.stream(stream):
        solver.set_inputs(sysg.H_diag, sysg.H_upper, sysg.sigR_diag, sysg.sigL_diag, sysg.sigG_diag)
        outs, status = solver.allocate_outputs(eps)
    torch.cuda.synchronize()

    def step(j):
        e0 = (j % nbat) * eps
        solver.solve(sysg.energies[e0:e0 + eps], outs, status, sig_range=(e0, e0 + eps))

    for j in range(a.warmup):
        step(j)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    step(a.warmup)
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1)
    import ctypes as C
    tr = _load_tracer()
    if tr.bt_trace_start() != 0:
        raise SystemExit("CUPTI activity tracing could not be enabled")
    step(a.warmup + 1)
    torch.cuda.synchronize()
    if tr.bt_trace_stop() != 0:
        raise SystemExit("CUPTI activity flush failed")
    agg = {}
    first, last = None, None
    name = C.create_string_buffer(1024)
    t0, t1 = C.c_ulonglong(0), C.c_ulonglong(0)
    recs = []
    for i in range(tr.bt_trace_count()):
        if tr.bt_trace_get(i, name, 1024, C.byref(t0), C.byref(t1)) < 0:
            continue
        s_ns, e_ns = t0.value, t1.value
        first = s_ns if first is None else min(first, s_ns)
        last = e_ns if last is None else max(last, e_ns)
        k = _short_name(name.value.decode(errors="replace"))
        recs.append((s_ns, e_ns, k))
        n, us = agg.get(k, (0, 0.0))
        agg[k] = (n + 1, us + (e_ns - s_ns) / 1e3)
    # device time between consecutive records (by start) with no record running, attributed to the
    # record after the gap: launch waits, or (graph mode) the device-side loop bodies
    recs.sort()
    gaps, idle, busy_to = {}, 0.0, None
    big = []  # (gap us, index of the record after it)
    for i, (s_ns, e_ns, k) in enumerate(recs):
        if busy_to is not None and s_ns > busy_to:
            g = (s_ns - busy_to) / 1e3
            idle += g
            n, us = gaps.get(k, (0, 0.0))
            gaps[k] = (n + 1, us + g)
            big.append((g, i))
        busy_to = e_ns if busy_to is None else max(busy_to, e_ns)
    big.sort(reverse=True)
    largest = [{"gap_ms": g / 1e3, "at_ms": (recs[i][0] - first) / 1e6,
                "before": [recs[j][2] for j in range(max(0, i - 3), i)],
                "after": [recs[j][2] for j in range(i, min(len(recs), i + 3))]} for g, i in big[:6]]
    total = sum(us for _, us in agg.values())
    rows = sorted(agg.items(), key=lambda kv: -kv[1][1])
    print(json.dumps({"kernel": "steptrace", "workload": f"nanoribbon G 40x416, {eps} energies per step",
                      "precision": a.precision, "split_scope": a.split_scope if a.precision == "split" else None,
                      "graph": a.graph, "cache_config": a.cache_config, "inv_panel": a.inv_panel,
                      "step_ms_plain": plain_ms,
                      "traced_span_ms": (last - first) / 1e6 if rows else 0,
                      "device_ms": total / 1e3, "launches": sum(n for n, _ in agg.values()),
                      "idle_ms": idle / 1e3,
                      "kernels": [{"name": k, "launches": n, "ms": us / 1e3, "share": us / total if total else 0}
                                  for k, (n, us) in rows],
                      "largest_gaps": largest,
                      "idle_before": [{"name": k, "gaps": n, "ms": us / 1e3}
                                      for k, (n, us) in sorted(gaps.items(), key=lambda kv: -kv[1][1])[:20]]}))
    status_bad = int((status != 0).sum().item())
    if status_bad:
        raise SystemExit(f"{status_bad} energies with a non-zero status")


def cublas_reference(a):
    """Library FP64 rates for comparison (not this library's kernels): cuBLAS DGEMM and ZGEMM
    through torch.matmul, batched over --batch matrices of --bs, mean of --reps after a warm-up."""
    import torch
    n, b = a.bs, a.batch
    out = {"kernel": "cublas", "bs": n, "batch": b}
    for name, dt, flop in (("dgemm", torch.float64, 2.0), ("zgemm", torch.complex128, 8.0)):
        x = torch.randn(b, n, n, dtype=dt, device="cuda")
        y = torch.randn(b, n, n, dtype=dt, device="cuda")
        torch.matmul(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(a.reps):
            torch.matmul(x, y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        out[name + "_ms"] = ms
        out[name + "_tflops"] = flop * n ** 3 * b / ms / 1e9
    print(json.dumps(out))


if __name__ == "__main__":
    main()
