"""Which FP64 route to the lead surface function is right (Sec. 4.2, Eq. 4 and 6)?

Near band edges at eta = 1e-6 the oracle's two FP64 routes, Sancho-Rubio decimation and the
direct eigen route of Eq. 6, disagree by up to ~1e-8.  An extended-precision decimation
(oracle.sancho_rubio_mp, 40 digits) decides: the eigen route is right to ~1e-14, FP64 decimation
is not.  One Newton step on e_s = x^{-1} after FP64 decimation (the step the CUDA path takes,
restated here in numpy) restores FP64 accuracy.  The GPU parity tests therefore compare against
the oracle with eigen-route contacts at the fixed tolerances, without any widening.

The extended-precision route is itself pinned against the closed form of the 1D chain, evaluated
in the same extended precision."""
import numpy as np
import pytest

import oracle
import synthetic

mp = pytest.importorskip("mpmath")


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def chain_surface_mp(z, eps, t, dps=50):
    """1D tight-binding chain (on-site eps, hopping t): g = (w - sqrt(w - 2t) sqrt(w + 2t)) / (2 t^2),
    w = z - eps, on the branch |t g| < 1, in mpmath arithmetic."""
    with mp.workdps(dps):
        w = mp.mpc(z.real, z.imag) - eps
        s = mp.sqrt(w - 2 * t) * mp.sqrt(w + 2 * t)
        g = (w - s) / (2 * t * t)
        if abs(t * g) >= 1:
            g = (w + s) / (2 * t * t)
        return complex(g)


@pytest.mark.parametrize("E", [1.9999999, -1.99999, 0.3, 2.0000001])
def test_extended_route_matches_chain_closed_form_at_band_edges(E):
    """The extended-precision decimation reproduces the chain's closed form to full FP64 accuracy,
    at and next to the band edges +-2t where FP64 decimation needs ~25 iterations."""
    t, eta = 1.0, 1e-6
    z = E + 1j * eta
    m = np.array([[z]])
    n = np.array([[-t + 0j]])
    x, it, ok = oracle.sancho_rubio_mp(m, n, n)
    assert ok
    want = chain_surface_mp(z, 0.0, t)
    assert abs(x[0, 0] - want) <= 1e-15 * abs(want)


def newton_polish(m, n, n_prime, tol=1e-14, maxit=100):
    """FP64 Sancho-Rubio followed by one Newton step on e_s = x^{-1}: the residual
    r = m - n x n' - e_s, the correction d of d - (n x) d (x n') = r by doubling, then
    x = (e_s + d)^{-1} (the CUDA path's polish, written out in numpy)."""
    a, b = n.astype(np.complex128), n_prime.astype(np.complex128)
    e = m.astype(np.complex128)
    es = e.copy()
    ref = max(np.abs(a).max(), np.abs(b).max())
    for _ in range(maxit):
        g = np.linalg.inv(e)
        agb, bga = a @ g @ b, b @ g @ a
        es, e = es - agb, e - agb - bga
        a, b = -(a @ g @ a), -(b @ g @ b)
        if max(np.abs(a).max(), np.abs(b).max()) <= tol * ref:
            break
    x = np.linalg.inv(es)
    A, B = n @ x, x @ n_prime
    X = m - n @ x @ n_prime - es
    for _ in range(64):
        X = X + A @ X @ B
        A, B = A @ A, B @ B
        if np.abs(A).max() * np.abs(B).max() * m.shape[0] ** 2 <= 1e-12:
            break
    return np.linalg.inv(es + X)


@pytest.fixture(scope="module")
def band_edge_leads():
    """A random 4 x 8 device (the 8 x 32 recipe at b = 8) on 400 energies: the three energies
    where the two FP64 routes disagree most, with both leads' blocks."""
    s = synthetic.random_device(77, 4, 8, 400)
    disc = []
    for e in range(len(s.energies)):
        d = 0.0
        for (m, n, np_) in oracle.lead_blocks(s, e):
            d = max(d, rel(oracle.sancho_rubio(m, n, np_)[0], oracle.surface_gf_eig(m, n, np_)))
        disc.append(d)
    worst = np.argsort(disc)[::-1][:3]
    return s, [int(e) for e in worst], [disc[e] for e in worst]


def test_eigen_route_is_right_and_fp64_decimation_is_not(band_edge_leads):
    s, energies, disc = band_edge_leads
    assert disc[0] > 1e-9  # the disagreement to decide
    worst_sr = 0.0
    for e in energies:
        for (m, n, np_) in oracle.lead_blocks(s, e):
            exact, _, ok = oracle.sancho_rubio_mp(m, n, np_)
            assert ok
            assert rel(oracle.surface_gf_eig(m, n, np_), exact) < 1e-13
            assert rel(newton_polish(m, n, np_), exact) < 1e-13
            worst_sr = max(worst_sr, rel(oracle.sancho_rubio(m, n, np_)[0], exact))
    assert worst_sr > 1e-9  # FP64 decimation alone is the inaccurate route


def test_selected_blocks_with_eigen_contacts_match_exact_contacts(band_edge_leads):
    """At the worst energy the oracle's selected blocks with eigen-route contacts equal those with
    extended-precision contacts to ~1e-11 per block; with FP64-decimation contacts they do not
    meet the 1e-10 FP64 tolerance."""
    s, energies, _ = band_edge_leads
    e = energies[0]
    exact = oracle.solve_g(s, e, surface="exact")
    eig = oracle.solve_g(s, e, surface="eig")
    dec = oracle.solve_g(s, e, surface="decimation")
    worst_eig = worst_dec = 0.0
    for k in ("R_diag", "R_upper", "R_lower", "L_diag", "L_upper", "G_diag", "G_upper"):
        for i in range(exact[k].shape[0]):
            worst_eig = max(worst_eig, rel(eig[k][i], exact[k][i]))
            worst_dec = max(worst_dec, rel(dec[k][i], exact[k][i]))
    assert worst_eig < 1e-11
    assert worst_dec > 1e-10
