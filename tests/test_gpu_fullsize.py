"""Parity at the benchmark's full size and launch configuration: the 40 x 416 nanoribbon, one
chunk of 32 energies strided over the grid, graph mode — exactly what bench.py times — checked on
sampled outputs that the oracle computes without a dense inverse (banded LU of the whole
16,640 x 16,640 system for block rows 0, 19 and 38, Sancho-Rubio contacts): FP64, the split with
sliced sweep products, and the split with every product sliced."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import TOL_FP64, TOL_SPLIT, block_errors

pytestmark = pytest.mark.gpu

BLOCKS = (0, 19, 38)
ENERGY = 256          # E = 0.0078 (between the Fermi levels); the bench's batch 0 of 16 (energies 0, 16, ..., 496)
EPS = 32


@pytest.fixture(scope="module")
def reference():
    s = synthetic.nanoribbon_40x416()
    ref = oracle.solve_g_sampled(s, ENERGY, list(BLOCKS))
    o = oracle.obc_self_energies(s, ENERGY)
    xr = max(np.linalg.norm(ref[i]["R_diag"]) for i in ref)
    floor = 0.01 * xr * xr * max(np.linalg.norm(o["R_L"]), np.linalg.norm(o["R_R"]))  # R12 (a)
    return s, ref, floor


@pytest.mark.parametrize("precision,scope,tol", [(0, 0, TOL_FP64), (1, 0, TOL_SPLIT), (1, 1, TOL_SPLIT)])
def test_fullsize_nanoribbon_sampled(reference, precision, scope, tol):
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    s, ref, floor = reference
    nE = len(s.energies)
    nbat = nE // EPS
    j = ENERGY % nbat
    idx = j + nbat * np.arange(EPS)
    pos = int(np.nonzero(idx == ENERGY)[0][0])
    solver = GSolver(s.nb, s.bs, EPS, s.eta, s.kT, s.mu_left, s.mu_right, obc=True, precision=precision,
                     split_scope=scope, graph=True)
    sub = s.subset(idx)
    solver.set_inputs(sub.H_diag, sub.H_upper, sub.sigR_diag, sub.sigL_diag, sub.sigG_diag)
    outs, status = solver.allocate_outputs(EPS)
    for _ in range(2):  # capture, then replay
        solver.solve(sub.energies, outs, status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    worst = {}
    for i in BLOCKS:
        for key, t in (("R_diag", outs["R"].diag), ("L_diag", outs["L"].diag), ("G_diag", outs["G"].diag),
                       ("R_upper", outs["R"].upper), ("R_lower", outs["R"].lower),
                       ("L_upper", outs["L"].upper), ("G_upper", outs["G"].upper)):
            if key not in ref[i]:
                continue
            got = t[pos, i].cpu().numpy()
            err = block_errors(got[None], ref[i][key][None], abs_floor=floor if key[0] in "LG" else 0.0).max()
            worst[(i, key)] = err
    bad = {k: v for k, v in worst.items() if not v <= tol}
    assert not bad, bad
    solver.close()
