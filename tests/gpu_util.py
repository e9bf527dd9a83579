"""Shared helpers of the GPU parity tests: run a synthetic system through the C ABI and compare
block by block with the CPU oracle (relative Frobenius error with the C1 floor)."""
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


def compare_g(res, sysg, e_gpu, e_ref, tol=TOL_FP64, symmetrize=True, keys=None):
    """Max per-block error of one energy against the dense oracle."""
    ref = oracle.solve_g(sysg, e_ref, symmetrize=symmetrize)
    lg_floor = 0.01 * lesser_floor(ref)
    worst = {}
    for k in (keys or ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")):
        if k not in res or ref[k].shape[0] == 0:
            continue
        errs = block_errors(res[k][e_gpu], ref[k], abs_floor=lg_floor if k[0] in "LG" else 0.0)
        worst[k] = float(errs.max())
    bad = {k: v for k, v in worst.items() if not v <= tol}
    return worst, bad


def route_discrepancy(sysg, e, symmetrize=True):
    """Per-output disagreement of two independent FP64 routes of the oracle at energy index e:
    contacts by Sancho-Rubio decimation vs by the eigen (polynomial eigenproblem) route.  It
    measures how far FP64 rounding alone moves the exact answer at this energy (large near
    band edges at small eta).  Returns {key: max per-block relative difference} or {} when the
    system has no contacts or the eigen route is not applicable."""
    if not sysg.obc:
        return {}
    ref = oracle.solve_g(sysg, e, symmetrize=symmetrize)
    orig = oracle.negf.sancho_rubio
    oracle.negf.sancho_rubio = lambda m, n, np_, tol=1e-14, maxit=100: (oracle.surface_gf_eig(m, n, np_), 0, True)
    try:
        alt = oracle.solve_g(sysg, e, symmetrize=symmetrize)
    except ValueError:
        return {}
    finally:
        oracle.negf.sancho_rubio = orig
    floor = 0.01 * lesser_floor(ref)
    out = {}
    for k in ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper"):
        if ref[k].shape[0] == 0:
            continue
        out[k] = float(block_errors(alt[k], ref[k], abs_floor=floor if k[0] in "LG" else 0.0).max())
    return out


def compare_g_derived(res, sysg, e_gpu, e_ref, tol=TOL_FP64, symmetrize=True, margin=10.0):
    """compare_g with the tolerance of each output raised to margin x the FP64 route
    discrepancy of the oracle at that energy (never below tol)."""
    worst, _ = compare_g(res, sysg, e_gpu, e_ref, tol=np.inf, symmetrize=symmetrize)
    disc = route_discrepancy(sysg, e_ref, symmetrize=symmetrize)
    bad = {}
    for k, v in worst.items():
        lim = max(tol, margin * disc.get(k, 0.0))
        if not v <= lim:
            bad[k] = (v, lim)
    return worst, bad
