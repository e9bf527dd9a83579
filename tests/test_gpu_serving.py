"""Serving (bt_server_*): requests of different device sizes submitted while others run; each
result equals the same request solved alone (same kernels, same chunking), admission respects
the arena budget, and latency statistics are reported."""
import numpy as np
import pytest

import synthetic
from gpu_util import compare_g

pytestmark = pytest.mark.gpu

SHAPES = [(4, 24, 5), (3, 40, 3), (6, 16, 8), (5, 64, 4), (3, 24, 6), (4, 40, 2)]  # (nb, bs, energies)
CHUNK = 4


def _request_inputs(k, nb, bs, nE):
    s = synthetic.random_device(1000 + k, nb, bs, nE)
    return s


def _tensors(s):
    import torch
    from paper_2508_19138_gb300 import BT, BTOut, BT_LAYOUT_BLOCKS, BT_SYM_HERMITIAN
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    H = BT(t(s.H_diag), t(s.H_upper), None, BT_LAYOUT_BLOCKS, BT_SYM_HERMITIAN, False)
    nE, nb, bs = len(s.energies), s.nb, s.bs
    mk = lambda *sh: torch.full(sh, float("nan"), dtype=torch.complex128, device="cuda")
    outs = {"R": BTOut(mk(nE, nb, bs, bs), mk(nE, nb - 1, bs, bs), mk(nE, nb - 1, bs, bs)),
            "L": BTOut(mk(nE, nb, bs, bs), mk(nE, nb - 1, bs, bs)),
            "G": BTOut(mk(nE, nb, bs, bs), mk(nE, nb - 1, bs, bs))}
    status = torch.full((nE,), -1, dtype=torch.int32, device="cuda")
    return H, outs, status


def _alone(s):
    """The same request through a plain context with the server's chunking."""
    import torch
    from paper_2508_19138_gb300.highlevel import GSolver
    solver = GSolver(s.nb, s.bs, min(CHUNK, len(s.energies)), s.eta, s.kT, s.mu_left, s.mu_right)
    solver.set_inputs(s.H_diag, s.H_upper)
    outs, status = solver.solve(s.energies)
    torch.cuda.synchronize()
    res = {w: (o.diag.cpu().numpy(), o.upper.cpu().numpy()) for w, o in outs.items()}
    solver.close()
    return res


def test_mixed_stream_equals_alone():
    import torch
    import paper_2508_19138_gb300 as pkg
    systems = [_request_inputs(k, *sh) for k, sh in enumerate(SHAPES)]
    srv = pkg.bt_server_create(hbm_budget_bytes=2 << 30, max_active=3, max_energies_per_chunk=CHUNK)
    tickets, held = [], []
    for s in systems:
        H, outs, status = _tensors(s)
        held.append((outs, status))
        tickets.append(pkg.bt_server_submit(srv, s.nb, s.bs, H, s.energies, status, outs["R"], outs["L"], outs["G"],
                                            eta=s.eta, kT=s.kT, mu_left=s.mu_left, mu_right=s.mu_right))
    for t in tickets:
        assert pkg.bt_server_wait(srv, t, 300.0) == 2
    stats = pkg.bt_server_get_stats(srv)
    assert stats["completed"] == len(SHAPES) and stats["failed"] == 0
    assert 0 < stats["p50_latency_s"] <= stats["p99_latency_s"]
    assert stats["peak_active"] >= 2  # requests overlapped
    assert stats["peak_bytes"] <= 2 << 30
    pkg.bt_server_destroy(srv)
    torch.cuda.synchronize()
    for s, (outs, status) in zip(systems, held):
        assert (status.cpu().numpy() == 0).all()
        alone = _alone(s)
        for w in "RLG":
            assert np.array_equal(outs[w].diag.cpu().numpy(), alone[w][0])
            assert np.array_equal(outs[w].upper.cpu().numpy(), alone[w][1])
    # and every block of every request against the oracle
    for s, (outs, _) in zip(systems, held):
        res = {}
        for w in "RLG":
            res[w + "_diag"] = outs[w].diag.cpu().numpy()
            res[w + "_upper"] = outs[w].upper.cpu().numpy()
        res["R_lower"] = outs["R"].lower.cpu().numpy()
        for e in range(len(s.energies)):
            _, bad = compare_g(res, s, e, e)
            assert not bad, (s.nb, s.bs, e, bad)


def test_failed_request_is_reported_and_others_complete():
    """A request that fails inside the server (here: its Hamiltonian lacks the off-diagonal
    blocks, which the solve rejects after admission) ends in state 3 with its error code;
    requests around it complete."""
    import paper_2508_19138_gb300 as pkg
    good = [_request_inputs(60 + k, 3, 16, 3) for k in range(2)]
    bad = _request_inputs(70, 3, 16, 3)
    srv = pkg.bt_server_create(hbm_budget_bytes=1 << 30, max_active=2, max_energies_per_chunk=CHUNK)
    held, tickets = [], []
    for k, s in enumerate([good[0], bad, good[1]]):
        H, outs, status = _tensors(s)
        if s is bad:
            H.upper = None  # injected fault: missing coupling blocks
        held.append((H, status))
        tickets.append(pkg.bt_server_submit(srv, s.nb, s.bs, H, s.energies, status, outs["R"], None, None,
                                            eta=s.eta, kT=s.kT))
    assert pkg.bt_server_wait(srv, tickets[0], 300.0) == 2
    assert pkg.bt_server_wait(srv, tickets[2], 300.0) == 2
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_server_wait(srv, tickets[1], 300.0)
    assert ei.value.status == pkg.BT_ERR_INVALID_ARG
    st = pkg.bt_server_get_stats(srv)
    assert st["completed"] == 2 and st["failed"] == 1
    pkg.bt_server_destroy(srv)


def test_budget_admission_and_rejection():
    import paper_2508_19138_gb300 as pkg
    s_big = _request_inputs(50, 6, 64, 4)
    s_small = _request_inputs(51, 3, 16, 4)
    need = pkg.bt_selinv_workspace_bytes(pkg.make_desc(s_big.nb, s_big.bs, CHUNK))
    # an arena that holds exactly one large request at a time
    srv = pkg.bt_server_create(hbm_budget_bytes=need + 4096, max_active=4, max_energies_per_chunk=CHUNK)
    H, outs, status = _tensors(s_big)
    tickets = [pkg.bt_server_submit(srv, s_big.nb, s_big.bs, H, s_big.energies, status, outs["R"], None, None,
                                    eta=s_big.eta, kT=s_big.kT)]
    H2, outs2, status2 = _tensors(s_big)
    tickets.append(pkg.bt_server_submit(srv, s_big.nb, s_big.bs, H2, s_big.energies, status2, outs2["R"], None,
                                        None, eta=s_big.eta, kT=s_big.kT))
    for t in tickets:
        assert pkg.bt_server_wait(srv, t, 300.0) == 2
    st = pkg.bt_server_get_stats(srv)
    assert st["peak_active"] == 1 and st["peak_bytes"] <= need + 4096
    # a request that can never fit is rejected at submit
    s_huge = _request_inputs(52, 8, 200, 64)
    H3, outs3, status3 = _tensors(s_small)
    with pytest.raises(pkg.BTError) as ei:
        pkg.bt_server_submit(srv, s_huge.nb, s_huge.bs, H3, s_huge.energies, status3, None, None, None)
    assert ei.value.status == pkg.BT_ERR_BUDGET
    assert pkg.bt_server_get_stats(srv)["rejected"] == 1
    pkg.bt_server_destroy(srv)


def test_timed_out_unit_is_started_again():
    """Host watchdog of the work units: the first tensor-core GEMM launch of the server stalls on a
    barrier nothing completes (test hook, 20 ms), so its unit's solve reports BT_ERR_TIMEOUT; the
    server starts that unit again and the request completes, every block against the oracle at the
    split tolerance.  With no retries allowed the same stall fails the request."""
    import torch
    import paper_2508_19138_gb300 as pkg
    from gpu_util import TOL_SPLIT
    s = _request_inputs(80, 3, 32, 6)
    for retries, want_state in ((1, 2), (0, 3)):
        srv = pkg.bt_server_create(hbm_budget_bytes=1 << 30, max_active=1, max_energies_per_chunk=CHUNK,
                                   precision=pkg.BT_SPLIT, max_retries=retries)
        H, outs, status = _tensors(s)
        try:
            pkg.bt_debug_split_stall(20_000_000, 1)
            t = pkg.bt_server_submit(srv, s.nb, s.bs, H, s.energies, status, outs["R"], outs["L"], outs["G"],
                                     eta=s.eta, kT=s.kT, mu_left=s.mu_left, mu_right=s.mu_right)
            if want_state == 2:
                assert pkg.bt_server_wait(srv, t, 300.0) == 2
            else:
                with pytest.raises(pkg.BTError) as ei:
                    pkg.bt_server_wait(srv, t, 300.0)
                assert ei.value.status == pkg.BT_ERR_TIMEOUT
        finally:
            pkg.bt_debug_split_stall(0, 0)
        st = pkg.bt_server_get_stats(srv)
        assert st["retries"] == retries
        pkg.bt_server_destroy(srv)
        torch.cuda.synchronize()
        if want_state == 2:
            assert (status.cpu().numpy() == 0).all()
            res = {w + "_diag": outs[w].diag.cpu().numpy() for w in "RLG"}
            res.update({w + "_upper": outs[w].upper.cpu().numpy() for w in "RLG"})
            res["R_lower"] = outs["R"].lower.cpu().numpy()
            for e in range(len(s.energies)):
                _, bad = compare_g(res, s, e, e, tol=TOL_SPLIT)
                assert not bad, (e, bad)


def test_units_of_a_request_run_concurrently_and_match_alone():
    """One request of 5 chunks on 3 workers: its units run side by side (peak_active 3) and the
    result equals the request solved alone with the same chunking, bitwise."""
    import torch
    import paper_2508_19138_gb300 as pkg
    s = _request_inputs(90, 4, 48, 5 * CHUNK)
    srv = pkg.bt_server_create(hbm_budget_bytes=2 << 30, max_active=3, max_energies_per_chunk=CHUNK)
    H, outs, status = _tensors(s)
    t = pkg.bt_server_submit(srv, s.nb, s.bs, H, s.energies, status, outs["R"], outs["L"], outs["G"],
                             eta=s.eta, kT=s.kT, mu_left=s.mu_left, mu_right=s.mu_right)
    assert pkg.bt_server_wait(srv, t, 300.0) == 2
    st = pkg.bt_server_get_stats(srv)
    assert st["units_done"] == 5 and st["peak_active"] >= 2
    pkg.bt_server_destroy(srv)
    torch.cuda.synchronize()
    alone = _alone(s)
    for w in "RLG":
        assert np.array_equal(outs[w].diag.cpu().numpy(), alone[w][0])
        assert np.array_equal(outs[w].upper.cpu().numpy(), alone[w][1])
