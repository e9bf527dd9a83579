"""Parity of the W (screened interaction) path with the dense oracle: M~ = I - V P^R and
B^<> = V P^<> V^H assembled as block-tridiagonal products on the GPU, RGF sweep, W^R = X^R V
on the selected blocks (needs X^R_{i,i+-2}), W^<> = X^<>; and with contacts (Sec. 4.2: leads
repeating the edge cells, retarded boundary by decimation, lesser / greater boundary by the Stein
equation of Eq. 7) against the oracle's folded-lead route."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import TOL_FP64, TOL_SPLIT, block_errors, compare_blocks

pytestmark = pytest.mark.gpu


def run_w(ws, idx, precision=0, max_energies=None, symmetrize=True, obc=False, split_scope=0):
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import BT, BTOut
    nb, bs = ws.nb, ws.bs
    E = len(idx)
    parts = [ws.P_blocks(e) for e in idx]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    PRd = t(np.stack([p[0] for p in parts]))
    PRu = t(np.stack([p[1] for p in parts]))
    PRl = t(np.stack([p[2] for p in parts]))
    PLd = t(np.stack([p[3] for p in parts]))
    PLu = t(np.stack([p[4] for p in parts]))
    PGd = t(np.stack([p[5] for p in parts]))
    PGu = t(np.stack([p[6] for p in parts]))
    desc = pkg.make_desc(nb, bs, max_energies or E, system=pkg.BT_SYS_W, precision=precision,
                         symmetrize=symmetrize, obc=obc, eta=0.0, split_scope=split_scope)
    ctx = pkg.bt_selinv_create(desc)
    V = BT(t(ws.V_diag), t(ws.V_upper), None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_HERMITIAN, False)
    PR = BT(PRd, PRu, PRl, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_GENERAL, True)
    PL = BT(PLd, PLu, None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_ANTIHERMITIAN, True)
    PG = BT(PGd, PGu, None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_ANTIHERMITIAN, True)
    mk = lambda *sh: torch.empty(sh, dtype=torch.complex128, device="cuda")
    oR = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), mk(E, nb - 1, bs, bs))
    oL = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
    oG = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
    status = torch.zeros(E, dtype=torch.int32, device="cuda")
    pkg.bt_selinv_solve(ctx, V, None, PR, PL, PG, ws.energies[idx], oR, oL, oG, status)
    torch.cuda.synchronize()
    ctx.close()
    out = {"R_diag": oR.diag, "R_upper": oR.upper, "R_lower": oR.lower, "L_diag": oL.diag, "L_upper": oL.upper,
           "G_diag": oG.diag, "G_upper": oG.upper}
    return {k: v.cpu().numpy() for k, v in out.items()}, status.cpu().numpy()


@pytest.mark.parametrize("geom", [dict(nb=4, ny=2, nz=2, nx=8, r_cut=5.0),
                                  dict(nb=5, ny=3, nz=2, nx=6, r_cut=4.0)])
@pytest.mark.parametrize("precision,tol", [(0, TOL_FP64), (1, TOL_SPLIT)])
def test_w_system_matches_dense(geom, precision, tol):
    ws = synthetic.w_system(spacing=2.2, n_energies=5, **geom)
    idx = np.arange(5)
    res, status = run_w(ws, idx, precision=precision, max_energies=3)
    assert (status == 0).all()
    for j, e in enumerate(idx):
        ref = oracle.solve_w(ws, e)
        for k in ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper"):
            errs = block_errors(res[k][j], ref[k])
            assert errs.max() < tol, (k, e, errs.max())


def test_w_identity_on_gpu_output():
    """W^> - W^< = W^R - W^A (exact for P^> - P^< = P^R - P^A, V Hermitian) on the diagonal."""
    ws = synthetic.w_system(nb=4, ny=2, nz=2, nx=8, spacing=2.2, r_cut=5.0, n_energies=2)
    res, status = run_w(ws, np.arange(2))
    for j in range(2):
        for i in range(ws.nb):
            R = res["R_diag"][j, i]
            lhs = res["G_diag"][j, i] - res["L_diag"][j, i]
            assert np.abs(lhs - (R - R.conj().T)).max() <= 1e-11 * np.abs(R).max()


@pytest.mark.parametrize("geom", [dict(nb=3, ny=2, nz=2, nx=8, r_cut=5.0),
                                  dict(nb=5, ny=3, nz=2, nx=6, r_cut=4.0)])
@pytest.mark.parametrize("precision,scope,tol", [(0, 0, TOL_FP64), (1, 0, TOL_SPLIT), (1, 1, TOL_SPLIT)])
def test_w_contacts_match_oracle(geom, precision, scope, tol):
    """W system with both leads attached (obc = 1), chunks of 3 over 5 energies: every selected
    block against oracle.solve_w_contacts (edge cells with the first lead cell's products, the
    folded lead blocks B^R_OBC and B^<>_OBC, W^R's lead-column terms)."""
    ws = synthetic.w_system(spacing=2.2, n_energies=5, **geom)
    idx = np.arange(5)
    res, status = run_w(ws, idx, precision=precision, max_energies=3, obc=True, split_scope=scope)
    assert (status == 0).all()
    for j, e in enumerate(idx):
        ref = oracle.solve_w_contacts(ws, e)
        for k in ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper"):
            worst = compare_blocks(res[k][j], ref[k], k, e, tol)
            assert worst <= tol, (k, e, worst)


def test_w_contacts_change_the_edge_blocks():
    """The contacts matter: the device without leads differs from the one with leads in the edge
    blocks by far more than the tolerance (so the test above cannot pass on the closed device)."""
    ws = synthetic.w_system(spacing=2.2, n_energies=2, nb=3, ny=2, nz=2, nx=8, r_cut=5.0)
    res, _ = run_w(ws, np.arange(2), obc=True)
    closed = oracle.solve_w(ws, 1)
    assert block_errors(res["L_diag"][1][:1], closed["L_diag"][:1]).max() > 1e-3
    assert block_errors(res["R_diag"][1][:1], closed["R_diag"][:1]).max() > 1e-3


def test_packed_polarization_inputs():
    """P^<> diagonal blocks given by their upper triangles (Sec. 5.2): the same W^R, W^<> as with
    the full blocks, bitwise (P^<> here is exactly anti-Hermitian)."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import BT, BTOut
    ws = synthetic.w_system(spacing=2.2, n_energies=3, nb=4, ny=2, nz=2, nx=8, r_cut=5.0)
    nb, bs, E = ws.nb, ws.bs, 3
    parts = [ws.P_blocks(e) for e in range(E)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P = [np.stack([p[j] for p in parts]) for j in range(7)]
    iu = np.triu_indices(bs)
    pack = lambda A: np.ascontiguousarray(A[..., iu[0], iu[1]])
    got = {}
    for packed in (False, True):
        lay = pkg.BT_LAYOUT_PACKED_UPPER if packed else pkg.BT_LAYOUT_BLOCKS
        V = BT(t(ws.V_diag), t(ws.V_upper), None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_HERMITIAN, False)
        PR = BT(t(P[0]), t(P[1]), t(P[2]), pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_GENERAL, True)
        PL = BT(t(pack(P[3]) if packed else P[3]), t(P[4]), None, lay, pkg.BT_SYM_ANTIHERMITIAN, True)
        PG = BT(t(pack(P[5]) if packed else P[5]), t(P[6]), None, lay, pkg.BT_SYM_ANTIHERMITIAN, True)
        mk = lambda *sh: torch.empty(sh, dtype=torch.complex128, device="cuda")
        oR = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), mk(E, nb - 1, bs, bs))
        oL = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
        oG = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
        status = torch.zeros(E, dtype=torch.int32, device="cuda")
        ctx = pkg.bt_selinv_create(pkg.make_desc(nb, bs, E, system=pkg.BT_SYS_W, obc=False, eta=0.0))
        pkg.bt_selinv_solve(ctx, V, None, PR, PL, PG, ws.energies[:E], oR, oL, oG, status)
        torch.cuda.synchronize()
        ctx.close()
        got[packed] = [x.cpu().numpy() for x in (oR.diag, oR.upper, oR.lower, oL.diag, oL.upper, oG.diag, oG.upper)]
    for a, b in zip(got[False], got[True]):
        assert np.array_equal(a, b)
    ref = oracle.solve_w(ws, 1)
    assert block_errors(got[True][3][1], ref["L_diag"]).max() < TOL_FP64
