"""Pins of the W-contact route of the oracle (groundwork for the W contacts, Sec. 4.2: Eq. 4 for
the retarded boundary, the Lyapunov / Stein equation of Eq. 7 for the lesser / greater one).

* w_lead_fold on a generic lead whose transfer a = x^R n is far from zero: x^R and w^<> equal the
  surface blocks of X^R and X^R B X^R^H of a long finite lead (dense inverse), the Stein term
  and the y term of a block-tridiagonal right-hand side included; dropping either fails.
* Eq. 7 as printed (w = q - a w a^H) misses the long-lead surface block; w = q + a w a^H matches.
* solve_w_contacts on a small W system equals a dense solve of the device with long explicit
  leads; dropping the lesser boundary fails."""
import numpy as np
import pytest

import oracle
import synthetic
from gpu_util import block_errors


def _lead(seed, bs, eta):
    rng = np.random.default_rng(seed)
    h = synthetic.cn(rng, (bs, bs))
    h = (h + h.conj().T) / 2
    t = 0.6 * synthetic.cn(rng, (bs, bs)) / np.sqrt(bs)
    z = 0.3 + 1j * eta
    m = z * np.eye(bs) - h
    n = -t                       # M_{k,k-1}: coupling to the next cell away from the device
    n_prime = -t.conj().T        # M_{k-1,k}
    g = synthetic.cn(rng, (bs, bs))
    b = -1j * (g @ g.conj().T) / bs                          # anti-Hermitian on-site block
    c = 0.5 * synthetic.cn(rng, (bs, bs)) / np.sqrt(bs)      # B_{k-1,k} (far -> near)
    return m, n, n_prime, b, c


def _chain_surface(m, n, n_prime, b, c, L):
    """Dense solve of L lead cells (cell L-1 next to the device): surface blocks of X^R and X^<>."""
    bs = m.shape[0]
    d = np.repeat(m[None], L, 0)
    up = np.repeat(n_prime[None], L - 1, 0)   # M_{k-1,k}
    lo = np.repeat(n[None], L - 1, 0)         # M_{k,k-1}
    M = oracle.bt_dense(d, up, lo)
    B = oracle.bt_dense(np.repeat(b[None], L, 0), np.repeat(c[None], L - 1, 0), lower_sign=-1.0)
    X = np.linalg.inv(M)
    XL = X @ B @ X.conj().T
    s = slice((L - 1) * bs, L * bs)
    return X[s, s], XL[s, s]


@pytest.mark.parametrize("seed", [0, 1])
def test_lead_fold_matches_long_finite_lead(seed):
    m, n, n_prime, b, c = _lead(seed, 4, 0.05)
    _, _, x, w = oracle.w_lead_fold(m, n, n_prime, b, c)
    a = x @ n
    assert max(abs(np.linalg.eigvals(a))) > 0.3   # the Stein term is not negligible here
    xs, ws = _chain_surface(m, n, n_prime, b, c, 400)
    assert block_errors(x[None], xs[None]).max() < 1e-10
    assert block_errors(w[None], ws[None]).max() < 1e-10
    # the pieces of the reading are all needed
    y = n @ x @ c
    q = x @ (b - y + y.conj().T) @ x.conj().T
    assert block_errors(q[None], ws[None]).max() > 1e-3                      # without the Stein term
    q0 = x @ b @ x.conj().T
    import scipy.linalg as sla
    w0 = sla.solve_discrete_lyapunov(a, q0)
    assert block_errors(w0[None], ws[None]).max() > 1e-3                     # without the y term


@pytest.mark.parametrize("seed", [0, 1])
def test_stein_sign_as_printed_fails(seed):
    """Eq. 7 is printed as w = q - a w a^H.  No scalar factor in a changes the sign of a w a^H
    (c a w (c a)^H = |c|^2 a w a^H), and the printed sign, solved exactly, misses the surface block
    of a long explicit lead by far; w = q + a w a^H matches it (the reading of the oracle)."""
    m, n, n_prime, b, c = _lead(seed, 4, 0.05)
    _, ws = _chain_surface(m, n, n_prime, b, c, 400)
    _, _, x, w = oracle.w_lead_fold(m, n, n_prime, b, c)
    y = n @ x @ c
    a = x @ n
    q = x @ (b - y + y.conj().T) @ x.conj().T
    k = q.shape[0]
    # w = q - a w a^H  <=>  (I + conj(a) (x) a) vec(w) = vec(q), vec stacking columns
    w_printed = np.linalg.solve(np.eye(k * k) + np.kron(a.conj(), a), q.reshape(-1, order="F")).reshape(k, k, order="F")
    assert np.abs(w_printed - (q - a @ w_printed @ a.conj().T)).max() < 1e-12
    assert block_errors(w_printed[None], ws[None]).max() > 0.1
    assert block_errors(w[None], ws[None]).max() < 1e-10


def test_w_contacts_match_long_explicit_leads():
    ws = synthetic.w_system(nb=3, ny=2, nz=2, nx=8, spacing=2.2, r_cut=5.0, n_energies=3)
    keys = ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper")
    for e in range(3):
        got = oracle.solve_w_contacts(ws, e)
        ref = oracle.solve_w_long_leads(ws, e, 16)
        for k in keys:
            assert block_errors(got[k], ref[k]).max() < 1e-12, (e, k)
    # without the lesser boundary blocks the edge cells' W^< is visibly wrong
    orig = oracle.negf.w_lead_fold

    def no_lesser(*args, **kw):
        r, lg, x, w = orig(*args, **kw)
        return r, 0.0 * lg, x, w

    oracle.negf.w_lead_fold = no_lesser
    try:
        bad = oracle.solve_w_contacts(ws, 1)
    finally:
        oracle.negf.w_lead_fold = orig
    ref = oracle.solve_w_long_leads(ws, 1, 16)
    assert block_errors(bad["L_diag"], ref["L_diag"]).max() > 1e-4
