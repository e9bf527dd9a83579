"""Shared helpers of the GPU parity tests: run a synthetic system through the C ABI and compare
block by block with the CPU oracle (relative Frobenius error per block, at the fixed tolerances
below; lesser / greater blocks with the absolute allowance of lesser_floor).  The oracle's lead
surface functions come from the eigen route (Eq. 6), which the CPU tests pin against an
extended-precision decimation; FP64 decimation alone is up to ~1e-8 off near band edges."""
import numpy as np

import oracle

TOL_FP64 = 1e-10   # per-block relative Frobenius error, FP64 path
TOL_SPLIT = 1e-8   # split-precision path


def lesser_floor(ref):
    """Absolute error scale of lesser/greater blocks set by FP64 rounding of the boundary
    broadening: B^<> ~ (Sigma - Sigma^H) cancels to ~eta-level outside the lead bands, so a
    rounding of u*|Sigma| in Sigma becomes an error ~ u*|X^R|^2*|Sigma| in X^<>.  Returns
    A = max_i |X^R_ii|_F^2 * max(|B^R_OBC,L|_F, |B^R_OBC,R|_F); blocks are compared with
    denominator max(|ref|, 0.01*A), i.e. an absolute allowance of 1e-12*A at tol 1e-10
    (1e4 unit roundoffs of the uncancelled magnitude)."""
    xr = max(np.linalg.norm(b) for b in ref["R_diag"])
    info = ref.get("info") or {}
    sig = max([np.linalg.norm(info[k]) for k in ("R_L", "R_R") if k in info] + [0.0])
    return xr * xr * sig


def unpack_upper(packed, bs):
    """Full anti-Hermitian blocks from BT_LAYOUT_PACKED_UPPER storage, for the comparisons:
    packed [..., bs (bs + 1) / 2] -> [..., bs, bs] with X_cr = -conj(X_rc) (Sec. 5.2)."""
    packed = np.asarray(packed)
    iu = np.triu_indices(bs)
    out = np.zeros(packed.shape[:-1] + (bs, bs), dtype=np.complex128)
    out[..., iu[0], iu[1]] = packed
    low = -np.conj(np.swapaxes(out, -1, -2))
    il = np.tril_indices(bs, -1)
    out[..., il[0], il[1]] = low[..., il[0], il[1]]
    return out


def block_errors(gpu, ref, floor_frac=1e-14, abs_floor=0.0):
    """Per-block relative Frobenius errors; the denominator is max(|ref block|,
    floor_frac * max block norm, abs_floor)."""
    ref = np.asarray(ref)
    gpu = np.asarray(gpu)
    norms = np.linalg.norm(ref.reshape(ref.shape[0], -1), axis=1)
    floor = max(floor_frac * norms.max() if norms.size else 0.0, abs_floor)
    errs = []
    for k in range(ref.shape[0]):
        den = max(norms[k], floor)
        num = np.linalg.norm(gpu[k] - ref[k])
        errs.append(num / den if den > 0 else num)
    return np.array(errs)


def run_g(sysg, max_energies=None, precision=0, split_slices=0, symmetrize=True, energies_idx=None,
          which=("R", "L", "G"), decim_maxit=100, sig_blocks=None):
    """Solve a synthetic.GSystem on the GPU; returns dict of numpy arrays and the status."""
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    E = sysg.energies if energies_idx is None else sysg.energies[energies_idx]
    pick = (lambda a: a) if energies_idx is None else (lambda a: None if a is None else a[energies_idx])
    n = len(E)
    solver = GSolver(sysg.nb, sysg.bs, max_energies or n, sysg.eta, sysg.kT, sysg.mu_left, sysg.mu_right,
                     obc=sysg.obc, precision=precision, split_slices=split_slices, symmetrize=symmetrize,
                     decim_maxit=decim_maxit)
    if sig_blocks is not None:
        sR, sL, sG = sig_blocks
    else:
        sR, sL, sG = pick(sysg.sigR_diag), pick(sysg.sigL_diag), pick(sysg.sigG_diag)
    solver.set_inputs(sysg.H_diag, sysg.H_upper, sR, sL, sG)
    outs, status = solver.allocate_outputs(n, which)
    solver.solve(E, outs, status)
    torch.cuda.synchronize()
    res = {}
    for w, o in outs.items():
        res[w + "_diag"] = o.diag.cpu().numpy()
        if o.upper is not None:
            res[w + "_upper"] = o.upper.cpu().numpy()
        if o.lower is not None:
            res[w + "_lower"] = o.lower.cpu().numpy()
    res["status"] = status.cpu().numpy()
    res["stats"] = solver.stats()
    solver.close()
    return res


# Every comparison of the parity tests is recorded here; conftest prints a summary at the end of
# the run: blocks compared per output, the largest relative error, and how many blocks passed
# only through the absolute lesser/greater allowance of lesser_floor (with the largest own-norm
# relative error among them).
PARITY_LOG = []


def record(test, key, e, own_rel, judged, tol, floor_used):
    PARITY_LOG.append(dict(test=test, key=key, energy=int(e), own_rel=float(own_rel), judged=float(judged),
                           tol=float(tol), floor_used=bool(floor_used)))


def _current_test():
    import os
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def compare_blocks(got, ref_blocks, key, e, tol, abs_floor=0.0):
    """Per-block comparison of one output with the oracle: the error judged is relative to
    max(|ref block|, 1e-14 max |ref|, abs_floor); every block is recorded in PARITY_LOG with its
    error relative to its own norm.  Returns the worst judged error."""
    judged = block_errors(got, ref_blocks, abs_floor=abs_floor)
    own = block_errors(got, ref_blocks)
    t = _current_test()
    for j, o in zip(judged, own):
        record(t, key, e, o, j, tol, floor_used=(o > tol and j <= tol))
    return float(judged.max()) if judged.size else 0.0


def compare_g(res, sysg, e_gpu, e_ref, tol=TOL_FP64, symmetrize=True, keys=None, surface="eig"):
    """Worst per-block error of one energy against the dense oracle (contacts by the eigen route,
    which the CPU tests check against extended precision).  Returns ({key: worst}, {key: worst}
    for the outputs above tol)."""
    ref = oracle.solve_g(sysg, e_ref, symmetrize=symmetrize, surface=surface)
    lg_floor = 0.01 * lesser_floor(ref)
    worst = {}
    for k in (keys or ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")):
        if k not in res or ref[k].shape[0] == 0:
            continue
        worst[k] = compare_blocks(res[k][e_gpu], ref[k], k, e_ref, tol, abs_floor=lg_floor if k[0] in "LG" else 0.0)
    bad = {k: v for k, v in worst.items() if not v <= tol}
    return worst, bad
