"""Parity of the GPU RGF path (G system) with the dense CPU oracle, block by block, FP64:
relative Frobenius error <= 1e-10 per block (C1 floor for underflowing blocks)."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import TOL_FP64, TOL_SPLIT, block_errors, compare_g, run_g

pytestmark = pytest.mark.gpu


def test_random_device_8x32_all_energies():
    """The 8 x 32, 64-energy random device: every block of every energy."""
    s = synthetic.random_device_8x32()
    res = run_g(s)
    assert (res["status"] == 0).all()
    worst_all = {}
    for e in range(len(s.energies)):
        worst, bad = compare_g(res, s, e, e)
        assert not bad, f"energy {e}: {bad}"
        for k, v in worst.items():
            worst_all[k] = max(worst_all.get(k, 0.0), v)
    print("worst per-block errors:", worst_all)


@pytest.mark.parametrize("nb,bs", [(5, 33), (3, 100), (4, 130), (2, 17), (6, 1)])
def test_ragged_sizes(nb, bs):
    s = synthetic.random_device(100 + bs, nb, bs, 5)
    res = run_g(s)
    assert (res["status"] == 0).all()
    for e in range(5):
        _, bad = compare_g(res, s, e, e)
        assert not bad, f"nb={nb} bs={bs} e={e}: {bad}"


def test_chunking_ragged_last_chunk():
    s = synthetic.random_device(7, 4, 16, 11)
    res = run_g(s, max_energies=4)  # chunks 4 + 4 + 3
    assert (res["status"] == 0).all()
    for e in range(11):
        _, bad = compare_g(res, s, e, e)
        assert not bad


def test_single_block_no_contacts():
    s = synthetic.random_device(8, 1, 20, 3)
    s.obc = False
    s.eta = 0.05
    res = run_g(s)
    for e in range(3):
        M, BL, BG, _ = oracle.assemble_g(s, e)
        assert np.linalg.norm(res["R_diag"][e, 0] - np.linalg.inv(M)) / np.linalg.norm(np.linalg.inv(M)) < 1e-12


def test_nanoribbon_wide_blocks_cluster_panels():
    """b = 200 >= 192: the inversions use the cluster-parallel panels; FP64 and split."""
    s = synthetic.nanoribbon(nb=3, n_puc=2, puc=100, n_energies=3)
    for precision, tol in ((0, TOL_FP64), (1, TOL_SPLIT)):
        res = run_g(s, precision=precision)
        assert (res["status"] == 0).all()
        for e in range(3):
            _, bad = compare_g(res, s, e, e, tol=tol)
            assert not bad, f"precision={precision} e={e}: {bad}"


def test_nanoribbon_diagonal_sigma():
    """Nanoribbon structure (sparse-in-dense H, periodic, diagonal scattering self-energies)."""
    s = synthetic.nanoribbon(nb=6, n_puc=2, puc=26, n_energies=6)
    res = run_g(s)
    assert (res["status"] == 0).all()
    for e in range(6):
        _, bad = compare_g(res, s, e, e)
        assert not bad, f"e={e}: {bad}"


def test_block_sigma_with_off_diagonals():
    """Full per-energy Sigma blocks with off-diagonal blocks: exercises the assembled M~ off-diagonal
    blocks and the y, Y terms of Eq. 10 / 11 (B^<> with off-diagonal blocks)."""
    rng = np.random.default_rng(17)
    s = synthetic.random_device(17, 5, 12, 4)
    nb, bs, E = s.nb, s.bs, 4
    # retarded: -i * (PSD banded Gamma)/2 ; lesser/greater anti-Hermitian by fluctuation-dissipation
    G = synthetic.cn(rng, (E, nb * bs, nb * bs)) * 0.02
    mask = np.zeros((nb * bs, nb * bs))
    for i in range(nb):
        for j in range(max(0, i - 1), min(nb, i + 2)):
            mask[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = 1
    Gam = np.stack([(g @ g.conj().T) * mask for g in G])
    sR = -0.5j * Gam
    f = 0.3
    sL = 1j * f * Gam
    sG = -1j * (1 - f) * Gam

    def blocks(A):
        d, u, l = zip(*[oracle.selected_blocks(a, nb, bs) for a in A])
        return np.stack(d), np.stack(u), np.stack(l)

    Rd, Ru, Rl = blocks(sR)
    Ld, Lu, _ = blocks(sL)
    Gd, Gu, _ = blocks(sG)
    import torch
    from paper_2508_19138_gb300 import highlevel, BT, BT_LAYOUT_BLOCKS, BT_SYM_GENERAL, BT_SYM_ANTIHERMITIAN
    solver = highlevel.GSolver(nb, bs, E, s.eta, s.kT, s.mu_left, s.mu_right, obc=True)
    solver.set_inputs(s.H_diag, s.H_upper)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    solver.sigR = BT(t(Rd), t(Ru), t(Rl), BT_LAYOUT_BLOCKS, BT_SYM_GENERAL, True)
    solver.sigL = BT(t(Ld), t(Lu), None, BT_LAYOUT_BLOCKS, BT_SYM_ANTIHERMITIAN, True)
    solver.sigG = BT(t(Gd), t(Gu), None, BT_LAYOUT_BLOCKS, BT_SYM_ANTIHERMITIAN, True)
    outs, status = solver.allocate_outputs(E)
    solver.solve(s.energies, outs, status)
    torch.cuda.synchronize()
    assert (status.cpu().numpy() == 0).all()
    for e in range(E):
        # dense reference with the full Sigma (lead blocks from M - Sigma^R edge blocks)
        z = s.energies[e] + 1j * s.eta
        M = oracle.bt_dense(z * np.eye(bs)[None] - s.H_diag - Rd[e], -s.H_upper - Ru[e],
                            -np.conj(np.swapaxes(s.H_upper, 1, 2)) - Rl[e])
        Mb = lambda i, j: M[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]
        xL = oracle.surface_gf_eig(Mb(0, 0), Mb(1, 0), Mb(0, 1))
        xR = oracle.surface_gf_eig(Mb(nb - 1, nb - 1), Mb(nb - 2, nb - 1), Mb(nb - 1, nb - 2))
        SL = Mb(1, 0) @ xL @ Mb(0, 1)
        SR = Mb(nb - 2, nb - 1) @ xR @ Mb(nb - 1, nb - 2)
        fL = float(oracle.fermi(s.energies[e], s.mu_left, s.kT))
        fR = float(oracle.fermi(s.energies[e], s.mu_right, s.kT))
        Mt = M.copy()
        Mt[:bs, :bs] -= SL
        Mt[-bs:, -bs:] -= SR
        BL = sL[e].copy()
        BL[:bs, :bs] += -fL * (SL - SL.conj().T)
        BL[-bs:, -bs:] += -fR * (SR - SR.conj().T)
        XR = np.linalg.inv(Mt)
        XL = oracle.symmetrize_lesser(XR @ BL @ XR.conj().T)
        rd, ru, rl = oracle.selected_blocks(XR, nb, bs)
        ld, lu, _ = oracle.selected_blocks(XL, nb, bs)
        xr = max(np.linalg.norm(b) for b in rd)
        lg = 0.01 * xr * xr * max(np.linalg.norm(SL), np.linalg.norm(SR), np.linalg.norm(sR[e]))
        for got, ref, fl in ((outs["R"].diag, rd, 0.0), (outs["R"].upper, ru, 0.0), (outs["R"].lower, rl, 0.0),
                             (outs["L"].diag, ld, lg), (outs["L"].upper, lu, lg)):
            assert block_errors(got.cpu().numpy()[e], ref, abs_floor=fl).max() < TOL_FP64


def test_unsymmetrized_output_is_anti_hermitian_and_symmetrized_matches():
    """The unsymmetrised run (every product computed in full) is anti-Hermitian to rounding, and
    its symmetrisation equals the symmetrised run (whose lesser sandwiches are computed as exactly
    anti-Hermitian products) to rounding, measured against the eta-level floor of R12."""
    from gpu_util import lesser_floor
    s = synthetic.random_device(31, 5, 24, 4)
    raw = run_g(s, symmetrize=False)
    sym = run_g(s, symmetrize=True)
    for e in range(4):
        fl = 0.01 * lesser_floor(oracle.solve_g(s, e))
        for i in range(s.nb):
            X = raw["L_diag"][e, i]
            assert np.abs(X + X.conj().T).max() <= 1e-9 * np.abs(X).max()
        X = raw["L_diag"][e]
        want = 0.5 * (X - np.conj(np.swapaxes(X, 1, 2)))
        assert block_errors(sym["L_diag"][e], want, abs_floor=fl).max() <= 1e-11
        _, bad = compare_g(raw, s, e, e, symmetrize=False)
        assert not bad


def test_antihermitian_sandwiches_match_full_products():
    """With symmetrised outputs the lesser/greater sandwiches x B x^H are computed as
    anti-Hermitian products (upper tiles, mirrored); b = 70 spans three 32-wide tiles and a ragged
    tail.  The result equals the unsymmetrised run (every tile computed) after symmetrisation, to
    rounding, and the oracle."""
    s = synthetic.random_device(57, 4, 70, 3)
    raw = run_g(s, symmetrize=False)
    sym = run_g(s, symmetrize=True)
    from gpu_util import lesser_floor
    for e in range(3):
        fl = 0.01 * lesser_floor(oracle.solve_g(s, e))  # rounding scale of eta-level blocks (R12)
        for key in ("L", "G"):
            X = raw[key + "_diag"][e]
            want = 0.5 * (X - np.conj(np.swapaxes(X, 1, 2)))
            assert block_errors(sym[key + "_diag"][e], want, abs_floor=fl).max() <= 1e-11
            assert block_errors(sym[key + "_upper"][e], raw[key + "_upper"][e], abs_floor=fl).max() <= 1e-11
        _, bad = compare_g(sym, s, e, e)
        assert not bad, (e, bad)


def test_gpu_invariants_identity_and_psd():
    """On the GPU output: the spectral functions A_ii = i(G^R - G^A), -iG^<_ii, iG^>_ii are PSD,
    and G^>_ii - G^<_ii - (G^R_ii - G^A_ii) equals the eta term 2 i eta (G^R G^A)_ii of the
    dense oracle (the identity with the eta correction)."""
    s = synthetic.random_device(41, 6, 16, 6)
    res = run_g(s)
    for e in range(6):
        ref = oracle.solve_g(s, e)
        XR = ref["XR"]
        eta_term = 2j * s.eta * XR @ XR.conj().T
        for i in range(s.nb):
            R = res["R_diag"][e, i]
            A = 1j * (R - R.conj().T)
            for Mx in (A, -1j * res["L_diag"][e, i], 1j * res["G_diag"][e, i]):
                w = np.linalg.eigvalsh((Mx + Mx.conj().T) / 2)
                assert w.min() >= -1e-9 * max(1.0, np.abs(w).max())
            lhs = res["G_diag"][e, i] - res["L_diag"][e, i] - (R - R.conj().T)
            blk = eta_term[i * s.bs:(i + 1) * s.bs, i * s.bs:(i + 1) * s.bs]
            scale = max(np.abs(res["G_diag"][e, i]).max(), np.abs(R).max(), 1e-300)
            assert np.abs(lhs - blk).max() <= 1e-10 * scale


def test_status_singular_energy():
    """No contacts, eta = 0, E = 0 and H = 0 in one block: M~ singular -> BT_ERR_SINGULAR for that
    energy only."""
    s = synthetic.random_device(5, 3, 8, 3)
    s.obc = False
    s.eta = 0.0
    s.H_diag[0] = 0.0
    s.H_upper[:] = 0.0
    s.energies = np.array([0.0, 0.5, 1.0])
    res = run_g(s)
    import paper_2508_19138_gb300 as pkg
    assert res["status"].tolist() == [pkg.BT_ERR_SINGULAR, 0, 0]


def test_status_decimation_not_converged():
    s = synthetic.random_device(6, 3, 8, 2)
    res = run_g(s, decim_maxit=2)
    import paper_2508_19138_gb300 as pkg
    assert (res["status"] == pkg.BT_ERR_NOT_CONVERGED).all()


@pytest.mark.parametrize("graph", [False, True])
def test_host_entry_point_matches_device(graph):
    """Host buffers, 5 energies in chunks of 2: the output copies of one chunk overlap the next
    chunk (double-buffered staging, second stream); twice in a row (graph mode: capture, then
    replays).  Bitwise equal to the device entry point."""
    from paper_2508_19138_gb300 import highlevel
    s = synthetic.nanoribbon(nb=4, n_puc=2, puc=10, n_energies=5)
    dev = run_g(s, max_energies=2)
    solver = highlevel.GSolver(s.nb, s.bs, 2, s.eta, s.kT, s.mu_left, s.mu_right, graph=graph)
    for _ in range(2):
        outs, status = highlevel.g_solve_host(solver.ctx, s.H_diag, s.H_upper, s.energies, s.sigR_diag,
                                              s.sigL_diag, s.sigG_diag)
        assert (status.numpy() == 0).all()
        for w in "RLG":
            assert np.array_equal(outs[w].diag.numpy(), dev[w + "_diag"])
            assert np.array_equal(outs[w].upper.numpy(), dev[w + "_upper"])
    solver.close()


@pytest.mark.parametrize("maker", ["random8x32", "ribbon"])
def test_split_precision_path(maker):
    """BT_SPLIT: sweep products as sliced bf16 tensor-core GEMMs, inverses / decimation FP64;
    per-block error <= 1e-8 (or 10x the FP64 route discrepancy where that is larger)."""
    if maker == "random8x32":
        s = synthetic.random_device_8x32().subset(np.arange(0, 64, 8))
    else:
        s = synthetic.nanoribbon(nb=5, n_puc=2, puc=52, n_energies=4)
    res = run_g(s, precision=1)
    assert (res["status"] == 0).all()
    for e in range(len(s.energies)):
        _, bad = compare_g(res, s, e, e, tol=TOL_SPLIT)
        assert not bad, f"e={e}: {bad}"


def test_split_scope_all_products():
    """split_scope = 1: also the block-inversion updates and the decimation products run as
    sliced tensor-core products (the default keeps them FP64)."""
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.nanoribbon(nb=5, n_puc=4, puc=26, n_energies=6)  # bs = 104 > 96: blocked inverse
    solver = GSolver(s.nb, s.bs, 3, s.eta, s.kT, s.mu_left, s.mu_right, precision=1, split_scope=1)
    solver.set_inputs(s.H_diag, s.H_upper, s.sigR_diag, s.sigL_diag, s.sigG_diag)
    outs, status = solver.solve(s.energies)
    torch.cuda.synchronize()
    res = {"status": status.cpu().numpy()}
    for w, o in outs.items():
        res[w + "_diag"] = o.diag.cpu().numpy()
        res[w + "_upper"] = o.upper.cpu().numpy()
        if o.lower is not None:
            res[w + "_lower"] = o.lower.cpu().numpy()
    solver.close()
    assert (res["status"] == 0).all()
    for e in range(len(s.energies)):
        _, bad = compare_g(res, s, e, e, tol=TOL_SPLIT)
        assert not bad, f"e={e}: {bad}"


def test_packed_upper_storage_of_lesser_greater():
    """Sec. 5.2 storage: lesser/greater diagonal blocks written as packed upper triangles match
    the oracle's symmetrised blocks at the FP64 tolerance (and the full-layout run exactly); the
    packed layout is refused for G^R and unsymmetrised runs."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from gpu_util import unpack_upper
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.random_device(61, 4, 70, 3)
    solver = GSolver(s.nb, s.bs, 3, s.eta, s.kT, s.mu_left, s.mu_right, obc=True)
    solver.set_inputs(s.H_diag, s.H_upper)
    full, st1 = solver.allocate_outputs(3)
    packed, st2 = solver.allocate_outputs(3, packed_lg=True)
    solver.solve(s.energies, full, st1)
    solver.solve(s.energies, packed, st2)
    torch.cuda.synchronize()
    assert packed["L"].diag.shape == (3, s.nb, s.bs * (s.bs + 1) // 2)
    res = {"R_diag": packed["R"].diag.cpu().numpy(), "R_upper": packed["R"].upper.cpu().numpy()}
    for w in ("L", "G"):
        got = unpack_upper(packed[w].diag.cpu().numpy(), s.bs)
        assert np.array_equal(got, full[w].diag.cpu().numpy())
        assert np.array_equal(packed[w].upper.cpu().numpy(), full[w].upper.cpu().numpy())
        res[w + "_diag"], res[w + "_upper"] = got, packed[w].upper.cpu().numpy()
    for e in range(3):
        _, bad = compare_g(res, s, e, e)
        assert not bad, (e, bad)
    bad = {"R": pkg.BTOut(packed["L"].diag, None, None, pkg.BT_LAYOUT_PACKED_UPPER)}
    with pytest.raises(pkg.BTError):
        solver.solve(s.energies, bad, st1)
    solver.close()


def test_packed_lesser_greater_inputs():
    """Sec. 5.2 storage of the inputs: Sigma^<> diagonal blocks given by their upper triangles
    (BT_LAYOUT_PACKED_UPPER, anti-Hermitian), off-diagonal blocks in full.  The solve equals the
    one with the full blocks bitwise (the blocks are exactly anti-Hermitian) and the oracle."""
    import torch
    from paper_2508_19138_gb300 import highlevel, BT, BT_LAYOUT_BLOCKS, BT_LAYOUT_PACKED_UPPER, BT_SYM_ANTIHERMITIAN
    rng = np.random.default_rng(23)
    s = synthetic.random_device(23, 4, 20, 3)
    nb, bs, E = s.nb, s.bs, 3

    def antiherm(shape, scale):
        X = synthetic.cn(rng, shape) * scale
        return X - np.conj(np.swapaxes(X, -1, -2))

    Ld, Lu = antiherm((E, nb, bs, bs), 0.01), synthetic.cn(rng, (E, nb - 1, bs, bs)) * 0.01
    Gd, Gu = antiherm((E, nb, bs, bs), 0.01), synthetic.cn(rng, (E, nb - 1, bs, bs)) * 0.01
    iu = np.triu_indices(bs)
    pack = lambda A: np.ascontiguousarray(A[..., iu[0], iu[1]])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    runs = {}
    for packed in (False, True):
        solver = highlevel.GSolver(nb, bs, E, s.eta, s.kT, s.mu_left, s.mu_right, obc=True)
        solver.set_inputs(s.H_diag, s.H_upper)
        lay = BT_LAYOUT_PACKED_UPPER if packed else BT_LAYOUT_BLOCKS
        solver.sigL = BT(t(pack(Ld) if packed else Ld), t(Lu), None, lay, BT_SYM_ANTIHERMITIAN, True)
        solver.sigG = BT(t(pack(Gd) if packed else Gd), t(Gu), None, lay, BT_SYM_ANTIHERMITIAN, True)
        outs, status = solver.allocate_outputs(E)
        solver.solve(s.energies, outs, status)
        torch.cuda.synchronize()
        assert (status.cpu().numpy() == 0).all()
        runs[packed] = {w + "_" + k: getattr(o, k).cpu().numpy() for w, o in outs.items()
                        for k in ("diag", "upper", "lower") if getattr(o, k) is not None}
        solver.close()
    for k in runs[False]:
        assert np.array_equal(runs[False][k], runs[True][k]), k
    for e in range(E):
        z = s.energies[e] + 1j * s.eta
        M, BL, BG, info = oracle.assemble_g(s, e, surface="eig")
        BL = BL + oracle.bt_dense(Ld[e], Lu[e], lower_sign=-1.0)
        BG = BG + oracle.bt_dense(Gd[e], Gu[e], lower_sign=-1.0)
        XR = np.linalg.inv(M)
        for key, B in (("L", BL), ("G", BG)):
            X = oracle.symmetrize_lesser(XR @ B @ XR.conj().T)
            d, u, _ = oracle.selected_blocks(X, nb, bs)
            from gpu_util import compare_blocks, lesser_floor
            fl = 0.01 * lesser_floor(dict(R_diag=oracle.selected_blocks(XR, nb, bs)[0], info=info))
            assert compare_blocks(runs[True][key + "_diag"][e], d, key + "_diag", e, TOL_FP64, fl) <= TOL_FP64
            assert compare_blocks(runs[True][key + "_upper"][e], u, key + "_upper", e, TOL_FP64, fl) <= TOL_FP64
