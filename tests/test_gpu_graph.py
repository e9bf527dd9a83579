"""Graph mode (one captured CUDA graph per chunk, decimation loop as a device-side conditional
while node): replays must give exactly the results of direct launches (same kernels in the same
order), across repeated solves, new energies, chunking, the iteration cap, the split path and
the W system; and the statistics folded in from the device must match the direct mode's."""
import numpy as np
import pytest

import synthetic
from gpu_util import compare_g

pytestmark = pytest.mark.gpu

OUT_KEYS = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")


def solve_both(s, energies_list, max_energies=None, **kw):
    """Runs the same sequence of solves in direct and graph mode; returns per-solve results."""
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    res = {}
    for graph in (False, True):
        stream = torch.cuda.Stream()
        solver = GSolver(s.nb, s.bs, max_energies or len(energies_list[0]), s.eta, s.kT, s.mu_left, s.mu_right,
                         obc=s.obc, stream=stream, graph=graph, **kw)
        with torch.cuda.stream(stream):
            solver.set_inputs(s.H_diag, s.H_upper)
            outs, status = solver.allocate_outputs(len(energies_list[0]))
        torch.cuda.synchronize()
        runs = []
        for E in energies_list:
            with torch.cuda.stream(stream):
                solver.solve(E, outs, status)
            torch.cuda.synchronize()
            r = {}
            for w, o in outs.items():
                r[w + "_diag"] = o.diag.cpu().numpy()
                if o.upper is not None:
                    r[w + "_upper"] = o.upper.cpu().numpy()
                if o.lower is not None:
                    r[w + "_lower"] = o.lower.cpu().numpy()
            r["status"] = status.cpu().numpy()
            r["stats"] = solver.stats()
            runs.append(r)
        solver.close()
        res[graph] = runs
    return res


def assert_identical(a, b):
    for k in OUT_KEYS + ("status",):
        assert np.array_equal(a[k], b[k]), k


def test_graph_replay_equals_direct_random_8x32():
    """The 8 x 32 device: capture on the first solve, replays on new energies and on the first
    energies again; bitwise equal to direct launches, decimation statistics equal."""
    s = synthetic.random_device_8x32()
    E0 = s.energies
    E1 = E0 + 0.0137
    res = solve_both(s, [E0, E1, E0])
    for d, g in zip(res[False], res[True]):
        assert_identical(d, g)
        assert d["stats"]["decim_iterations"] == g["stats"]["decim_iterations"]
        assert d["stats"]["lead_iterations"] == g["stats"]["lead_iterations"]
        # the Newton step after decimation (near-band-edge leads), captured as a second loop
        assert d["stats"]["newton_leads"] == g["stats"]["newton_leads"] > 0
        assert d["stats"]["newton_iterations"] == g["stats"]["newton_iterations"]
        assert d["stats"]["flops_model"] == pytest.approx(g["stats"]["flops_model"], rel=1e-12)
    # the replayed results are also right (not just repeatable)
    r = res[True][1]
    s1 = synthetic.random_device(synthetic.BASE_SEED, 8, 32, 64)
    s1.energies = E1
    for e in (0, 17, 40, 63):
        _, bad = compare_g(r, s1, e, e)
        assert not bad, (e, bad)


def test_graph_chunks_and_ragged_tail():
    """11 energies in chunks of 4 (4 + 4 + 3): one graph per chunk, each replayed."""
    s = synthetic.random_device(31, 4, 16, 11)
    res = solve_both(s, [s.energies, s.energies[::-1].copy()], max_energies=4)
    for d, g in zip(res[False], res[True]):
        assert_identical(d, g)


def test_graph_iteration_cap_reports_not_converged():
    """decim_maxit = 2: the device loop stops at the cap and the energies report
    BT_ERR_NOT_CONVERGED exactly as in direct mode."""
    import paper_2508_19138_gb300 as pkg
    s = synthetic.random_device(5, 3, 8, 6)
    res = solve_both(s, [s.energies, s.energies], decim_maxit=2)
    for d, g in zip(res[False], res[True]):
        assert_identical(d, g)
        assert (g["status"] == pkg.BT_ERR_NOT_CONVERGED).any()
        assert g["stats"]["decim_iterations"] == d["stats"]["decim_iterations"]


def test_graph_split_precision():
    import paper_2508_19138_gb300 as pkg
    s = synthetic.random_device(9, 3, 64, 5)
    res = solve_both(s, [s.energies, s.energies + 0.01], precision=pkg.BT_SPLIT, split_scope=1)
    for d, g in zip(res[False], res[True]):
        assert_identical(d, g)


@pytest.mark.parametrize("obc", [False, True])
def test_graph_w_system(obc):
    """W system: graph replay equals direct launches, without contacts and with them (the
    decimation loop and the Stein doubling loops of the lesser / greater boundary captured as
    conditional while nodes)."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import BT, BTOut
    ws = synthetic.w_system(spacing=2.2, n_energies=4, nb=4, ny=2, nz=2, nx=8, r_cut=5.0)
    nb, bs, E = ws.nb, ws.bs, 4
    parts = [ws.P_blocks(e) for e in range(E)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    P = [t(np.stack([p[j] for p in parts])) for j in range(7)]
    V = BT(t(ws.V_diag), t(ws.V_upper), None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_HERMITIAN, False)
    PR = BT(P[0], P[1], P[2], pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_GENERAL, True)
    PL = BT(P[3], P[4], None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_ANTIHERMITIAN, True)
    PG = BT(P[5], P[6], None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_ANTIHERMITIAN, True)
    got = {}
    for graph in (False, True):
        stream = torch.cuda.Stream()
        desc = pkg.make_desc(nb, bs, E, system=pkg.BT_SYS_W, obc=obc, eta=0.0, graph=graph)
        ctx = pkg.bt_selinv_create(desc, stream)
        mk = lambda *sh: torch.empty(sh, dtype=torch.complex128, device="cuda")
        oR = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), mk(E, nb - 1, bs, bs))
        oL = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
        oG = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), None)
        status = torch.zeros(E, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        outs = []
        for _ in range(2):
            pkg.bt_selinv_solve(ctx, V, None, PR, PL, PG, ws.energies[:E], oR, oL, oG, status)
            torch.cuda.synchronize()
            outs.append([x.cpu().numpy() for x in (oR.diag, oR.upper, oR.lower, oL.diag, oL.upper, oG.diag,
                                                    oG.upper, status)])
        ctx.close()
        got[graph] = outs
    for a, b in zip(got[False], got[True]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("precision,scope", [(0, 0), (1, 1)])
def test_graph_wide_blocks_staged_sigma(precision, scope):
    """b = 200: cluster-parallel inversion panels inside the captured decimation loop; scattering
    self-energies given per energy and passed as energy slices, which graph mode stages into
    fixed buffers so that every batch replays the same graph.  Bitwise equal to direct launches."""
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    s = synthetic.nanoribbon(nb=3, n_puc=2, puc=100, n_energies=6)
    got = {}
    for graph in (False, True):
        stream = torch.cuda.Stream()
        solver = GSolver(s.nb, s.bs, 3, s.eta, s.kT, s.mu_left, s.mu_right, obc=True, precision=precision,
                         split_scope=scope, stream=stream, graph=graph)
        with torch.cuda.stream(stream):
            solver.set_inputs(s.H_diag, s.H_upper, s.sigR_diag, s.sigL_diag, s.sigG_diag)
            outs, status = solver.allocate_outputs(3)
        torch.cuda.synchronize()
        runs = []
        for e0 in (0, 3, 0):
            with torch.cuda.stream(stream):
                solver.solve(s.energies[e0:e0 + 3], outs, status, sig_range=(e0, e0 + 3))
            torch.cuda.synchronize()
            runs.append([o.cpu().numpy() for w in ("R", "L", "G") for o in (outs[w].diag, outs[w].upper)
                         if o is not None] + [status.cpu().numpy()])
        st = solver.stats()
        solver.close()
        got[graph] = (runs, st)
    for a, b in zip(got[False][0], got[True][0]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert got[False][1]["decim_iterations"] == got[True][1]["decim_iterations"]


def test_graph_input_staging_grows_and_replays():
    """Graph mode copies each chunk's per-energy inputs to the context's staging memory: a solve
    with a larger input layout (block self-energies after diagonal-vector ones) grows it, which
    drops the graphs captured on the old staging; solves with new energy batches of the same
    layout then replay.  Every result is bitwise equal to direct launches."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from paper_2508_19138_gb300 import BT, BTOut
    s = synthetic.random_device(23, 4, 48, 9)
    nb, bs, E = s.nb, s.bs, 3
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    rng = np.random.default_rng(5)
    # per-energy scattering self-energies: diagonal vectors, and full diagonal blocks
    gam = 0.02 * (1.0 + rng.random((9, nb, bs)))
    sig_vec = t(-0.5j * gam)
    blk = np.zeros((9, nb, bs, bs), dtype=np.complex128)
    for e in range(9):
        for i in range(nb):
            a = 0.01 * (rng.standard_normal((bs, bs)) + 1j * rng.standard_normal((bs, bs)))
            blk[e, i] = -0.5j * (a @ a.conj().T + np.diag(gam[e, i]))  # anti-Hermitian part: -i/2 Gamma
    sig_blk = t(blk)
    H = BT(t(s.H_diag), t(s.H_upper), None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_HERMITIAN, False)

    def sigma(kind, e0):
        if kind == "vec":
            return BT(sig_vec[e0:e0 + E], None, None, pkg.BT_LAYOUT_DIAGVEC, pkg.BT_SYM_GENERAL, True)
        return BT(sig_blk[e0:e0 + E], None, None, pkg.BT_LAYOUT_BLOCKS, pkg.BT_SYM_GENERAL, True)

    calls = [("vec", 0), ("vec", 3), ("blk", 0), ("blk", 6), ("blk", 3)]
    got = {}
    for graph in (False, True):
        stream = torch.cuda.Stream()
        desc = pkg.make_desc(nb, bs, E, obc=True, eta=s.eta, kT=s.kT, mu_left=s.mu_left, mu_right=s.mu_right,
                             graph=graph)
        ctx = pkg.bt_selinv_create(desc, stream)
        mk = lambda *sh: torch.empty(sh, dtype=torch.complex128, device="cuda")
        oR = BTOut(mk(E, nb, bs, bs), mk(E, nb - 1, bs, bs), mk(E, nb - 1, bs, bs))
        status = torch.zeros(E, dtype=torch.int32, device="cuda")
        outs = []
        for kind, e0 in calls:
            sg = sigma(kind, e0)
            pkg.bt_selinv_solve(ctx, H, None, sg, None, None, s.energies[e0:e0 + E], oR, None, None, status)
            torch.cuda.synchronize()
            outs.append([x.cpu().numpy() for x in (oR.diag, oR.upper, oR.lower, status)])
        ctx.close()
        got[graph] = outs
    for a, b in zip(got[False], got[True]):
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    assert all((o[3] == 0).all() for o in got[True])
