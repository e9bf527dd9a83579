"""Parity at the benchmark's full sizes and launch configurations.

* The 40 x 416 nanoribbon, one chunk of 32 energies strided over the grid, graph mode (what
  bench.py times), checked on sampled outputs that the oracle computes without a dense inverse
  (banded LU of the whole 16,640 x 16,640 system for block rows 0, 19 and 38, contacts by the
  eigen route): FP64, the split with sliced sweep products, and the split with every product
  sliced.
* The W system of 16 cells of 1024 atoms, one chunk of 4 energies (the bench's W step), against
  stored oracle values (tests/golden/w16x1024_e64.npz, written by tests/golden/make_golden.py from
  oracle.solve_w_sampled): per sampled block its Frobenius norm and 512 seeded entries.  And the
  identity W^> - W^< = W^R - W^A on every block."""
import os

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
    ref = oracle.solve_g_sampled(s, ENERGY, list(BLOCKS), surface="eig")
    o = oracle.obc_self_energies(s, ENERGY, surface="eig")
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


def _w_chunk(ws, idx, precision):
    """Solves the W system for the energies idx (one chunk) through the C ABI; returns the outputs."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import BT, BTOut
    nb, bs = ws.nb, ws.bs
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    R0d, R0u, R1d, R1u, Gd, Gu = (t(x) for x in (ws.R0_diag, ws.R0_upper, ws.R1_diag, ws.R1_upper, ws.Gam_diag,
                                                   ws.Gam_upper))
    R0l, R1l, Gl = (x.transpose(1, 2).conj().contiguous() for x in (R0u, R1u, Gu))
    r1 = torch.tensor(ws.r1[idx], device="cuda").view(-1, 1, 1, 1)
    s1 = torch.tensor(1.0 + ws.g1[idx], device="cuda").view(-1, 1, 1, 1)
    a = torch.tensor(ws.a[idx], device="cuda").view(-1, 1, 1, 1)
    PR = BT((R0d + r1 * R1d - 0.5j * s1 * Gd).contiguous(), (R0u + r1 * R1u - 0.5j * s1 * Gu).contiguous(),
            (R0l + r1 * R1l - 0.5j * s1 * Gl).contiguous(), pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_GENERAL, True)
    PL = BT((-1j * a * s1 * Gd).contiguous(), (-1j * a * s1 * Gu).contiguous(), None, pkg.BT_LAYOUT_BLOCKS,
            pkg.BT_SYM_ANTIHERMITIAN, True)
    PG = BT((-1j * (1 + a) * s1 * Gd).contiguous(), (-1j * (1 + a) * s1 * Gu).contiguous(), None,
            pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_ANTIHERMITIAN, True)
    V = BT(t(ws.V_diag), t(ws.V_upper), None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_HERMITIAN, False)
    E = len(idx)
    mk = lambda *sh: torch.empty(sh, dtype=torch.complex128, device="cuda")
    oR = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), mk(E, nb - 1, bs, bs))
    oL = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs))
    oG = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs))
    status = torch.zeros(E, dtype=torch.int32, device="cuda")
    ctx = pkg.bt_selinv_create(pkg.make_desc(nb, bs, E, system=pkg.BT_SYS_W, precision=precision, obc=False,
                                             eta=0.0))
    pkg.bt_selinv_solve(ctx, V, None, PR, PL, PG, ws.energies[idx], oR, oL, oG, status)
    torch.cuda.synchronize()
    ctx.close()
    assert (status.cpu().numpy() == 0).all()
    return oR, oL, oG


@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_fullsize_w_sampled_against_oracle(precision, tol):
    """The bench's W step (4 energies strided over the 256-energy grid: 0, 64, 128, 192), energy 64
    against the stored oracle values of block rows 0, 7 and 15: the block's Frobenius norm, every
    sampled entry within tol of the block norm, and the Frobenius error estimated from the 512
    sampled entries (root-mean-square error times bs) within tol."""
    import importlib.util
    here = os.path.dirname(os.path.abspath(__file__))
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(here, "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    gold = np.load(os.path.join(here, "golden", "w16x1024_e64.npz"))
    ws = synthetic.w_system_16x1024()
    idx = np.array([0, 64, 128, 192])
    pos = int(np.nonzero(idx == int(gold["energy"]))[0][0])
    oR, oL, oG = _w_chunk(ws, idx, precision)
    outs = {"R": oR, "L": oL, "G": oG}
    worst = {}
    for name, fro, vals in zip(gold["names"], gold["fro"], gold["vals"]):
        i, key = str(name).split(":")
        i = int(i)
        o = outs[key[0]]
        blk = getattr(o, key.split("_")[1])[pos, i].cpu().numpy()
        got = blk.reshape(-1)[mg.w_sample_indices(ws.bs, i, key)]
        d = np.abs(got - vals)
        est = np.sqrt(np.mean(d * d)) * ws.bs / fro
        worst[name] = (est, d.max() / fro, abs(np.linalg.norm(blk) - fro) / fro)
    bad = {k: v for k, v in worst.items() if not max(v) <= tol}
    assert not bad, bad
    print("worst (estimated Frobenius, max entry, norm) errors:", {k: f"{max(v):.2e}" for k, v in worst.items()})


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-7)])
def test_fullsize_w_identity(precision, tol):
    """W system at full size (16 cells of 1024 atoms, the bench's W workload), two energies: the
    identity W^> - W^< = W^R - W^A, exact when P^> - P^< = P^R - P^A and V = V^H (Table 2), on every
    diagonal and upper block, relative to the largest W^R block."""
    import torch
    ws = synthetic.w_system_16x1024()
    oR, oL, oG = _w_chunk(ws, np.array([40, 200]), precision)
    scale = torch.linalg.matrix_norm(oR.diag).max().item()
    lhs_d = oG.diag - oL.diag
    rhs_d = oR.diag - oR.diag.transpose(-1, -2).conj()
    lhs_u = oG.upper - oL.upper
    rhs_u = oR.upper - oR.lower.transpose(-1, -2).conj()
    err = max(torch.linalg.matrix_norm(lhs_d - rhs_d).max().item(), torch.linalg.matrix_norm(lhs_u - rhs_u).max().item())
    assert err <= tol * scale, (err / scale, tol)
