"""Pins of the CPU oracle against results fixed by mathematics and physics, not by the oracle
itself: closed-form surface Green's functions of the 1D chain, integer Landauer transmission,
the eigen-route (direct) surface function, block-inverse closed forms, continued fractions,
anti-Hermiticity, the G^> - G^< identity, PSD spectral functions, current conservation and the
equilibrium relation.  A dropped term, a flipped sign, a transposed operand or a wrong lead
orientation in the oracle fails at least one of these (see the mutation tests at the end)."""
import numpy as np
import pytest

import oracle
import synthetic
from conftest import rel_fro


def chain_surface_closed_form(z, eps, t):
    """Surface GF of a semi-infinite chain: g = (w - sqrt(w^2 - 4 t^2)) / (2 t^2), w = z - eps,
    with the root chosen so that |t g| < 1 (retarded, decaying)."""
    w = z - eps
    r = np.sqrt(w * w - 4 * t * t + 0j)
    g1 = (w - r) / (2 * t * t)
    g2 = (w + r) / (2 * t * t)
    return g1 if abs(t * g1) < 1 else g2


def bulk_chain_closed_form(z, eps, t):
    """Diagonal GF of the infinite chain: 1 / sqrt((z-eps)^2 - 4t^2), branch with Im < 0."""
    w = z - eps
    r = np.sqrt(w * w - 4 * t * t + 0j)
    g = 1.0 / r
    return g if g.imag <= 0 else -g


@pytest.mark.parametrize("E", [-2.5, -1.0, 0.0, 0.7, 1.9, 2.3, 3.5])
@pytest.mark.parametrize("eta", [1e-3, 1e-6])
def test_sancho_rubio_1d_chain_closed_form(E, eta):
    eps, t = 0.2, -1.0
    z = E + 1j * eta
    m = np.array([[z - eps]])
    n = np.array([[-t]])  # M = z - H: coupling block of M is -t
    x, it, ok = oracle.sancho_rubio(m, n, n)
    assert ok and it < 60
    g = chain_surface_closed_form(z, eps, t)
    assert abs(x[0, 0] - g) <= 1e-12 * abs(g) + 1e-12
    assert x[0, 0].imag < 0  # retarded


def test_sancho_rubio_multichannel_closed_form():
    rng = np.random.default_rng(3)
    bs, t = 6, 0.8
    h00 = synthetic.cn(rng, (bs, bs))
    h00 = (h00 + h00.conj().T) / 2
    lam, U = np.linalg.eigh(h00)
    for E in (-1.3, 0.1, 2.2):
        z = E + 1e-5j
        x, it, ok = oracle.sancho_rubio(z * np.eye(bs) - h00, -t * np.eye(bs), -t * np.eye(bs))
        ref = U @ np.diag([chain_surface_closed_form(z, l, t) for l in lam]) @ U.conj().T
        assert ok
        assert rel_fro(x, ref) < 1e-11


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sancho_rubio_matches_eigen_route(seed):
    """Sancho-Rubio vs the direct polynomial-eigenproblem route (Eq. 6) on random leads."""
    rng = np.random.default_rng(seed)
    bs = 5
    h00 = synthetic.cn(rng, (bs, bs))
    h00 = (h00 + h00.conj().T) / 2 / np.sqrt(bs)
    h01 = 0.5 * synthetic.cn(rng, (bs, bs)) / np.sqrt(bs)
    for E in (-0.8, 0.0, 0.9):
        z = E + 1e-3j
        m = z * np.eye(bs) - h00
        x_sr, _, ok = oracle.sancho_rubio(m, -h01, -h01.conj().T)
        x_ev = oracle.surface_gf_eig(m, -h01, -h01.conj().T)
        assert ok
        assert rel_fro(x_sr, x_ev) < 1e-9
        # it is a fixed point of Eq. 4
        fp = np.linalg.inv(m - (-h01) @ x_sr @ (-h01.conj().T))
        assert rel_fro(fp, x_sr) < 1e-12


@pytest.mark.parametrize("E", [-1.5, 0.3, 1.2])
def test_finite_chain_with_contacts_is_infinite_chain(E):
    """A segment of a uniform chain with both contacts attached is the infinite chain:
    every diagonal element of G^R equals 1/sqrt((z-eps)^2 - 4t^2) (pins the lead orientation,
    the boundary blocks and the dense inverse)."""
    eps, t, eta = 0.1, 1.0, 1e-5
    s = synthetic.chain_1d(7, eps, t, [E], eta)
    r = oracle.solve_g(s, 0)
    g = bulk_chain_closed_form(E + 1j * eta, eps, t)
    for i in range(7):
        assert abs(r["R_diag"][i][0, 0] - g) < 1e-10 * abs(g)
    # and off-diagonal G_{i,i+1} = g * lambda with the decaying Bloch factor (same for all i)
    assert np.allclose(r["R_upper"][:, 0, 0], r["R_upper"][0, 0, 0], rtol=1e-10)


@pytest.mark.parametrize("E,T_expected", [(-2.5, 0.0), (-1.0, 1.0), (0.0, 1.0), (1.7, 1.0), (2.4, 0.0)])
def test_chain_transmission_integer(E, T_expected):
    s = synthetic.chain_1d(5, 0.0, 1.0, [E], 1e-9)
    assert abs(oracle.transmission(s, 0) - T_expected) < 1e-6


def test_multichannel_transmission_counts_open_modes():
    rng = np.random.default_rng(11)
    bs, t, nb = 5, 1.0, 4
    h00 = synthetic.cn(rng, (bs, bs))
    h00 = (h00 + h00.conj().T)
    lam = np.linalg.eigvalsh(h00)
    s = synthetic.GSystem(H_diag=np.broadcast_to(h00, (nb, bs, bs)).copy(),
                          H_upper=np.broadcast_to(t * np.eye(bs), (nb - 1, bs, bs)).astype(np.complex128),
                          energies=np.array([-1.0, 0.2, 1.4]), eta=1e-9, mu_left=0, mu_right=0, kT=0.025)
    for e, E in enumerate(s.energies):
        expected = int(np.sum(np.abs(E - lam) < 2 * abs(t)))
        assert abs(oracle.transmission(s, e) - expected) < 1e-5


def test_bond_current_conserved_and_equals_transmission():
    """Periodic device, f_L = 1, f_R = 0, eta -> 0: 2 Re Tr[H_{i,i+1} G^<_{i+1,i}] is the same at
    every interface and equals T(E) (f_L - f_R).  Pins the off-diagonal lesser blocks."""
    rng = np.random.default_rng(5)
    bs, nb = 4, 6
    h00 = synthetic.cn(rng, (bs, bs))
    h00 = (h00 + h00.conj().T) / 2
    h01 = synthetic.cn(rng, (bs, bs))
    s = synthetic.GSystem(H_diag=np.broadcast_to(h00, (nb, bs, bs)).copy(),
                          H_upper=np.broadcast_to(h01, (nb - 1, bs, bs)).copy(),
                          energies=np.array([-0.7, 0.4]), eta=1e-10, mu_left=50.0, mu_right=-50.0,
                          kT=0.025)
    for e in range(2):
        r = oracle.solve_g(s, e)
        I = oracle.bond_currents(s.H_upper, r["L_upper"])
        T = oracle.transmission(s, e)
        assert T > 0.5
        assert np.allclose(I, T, rtol=1e-6, atol=1e-8)


def test_contact_currents_meir_wingreen():
    """Coherent transport (no scattering, eta -> 0) with f_L = 1, f_R = 0 on a random, non-periodic
    device: the current into the device at each contact, Tr[B^<_c G^>_cc - B^>_c G^<_cc] over that
    contact's edge block, is +T(E) at the left and -T(E) at the right, and the bond current inside
    the device is T(E) at every interface.  T comes from retarded quantities only, so this pins the
    lesser/greater edge blocks and the contacts' Fermi weights and orientation."""
    s = synthetic.random_device(12, 5, 6, 8, e_lo=-1.0, e_hi=1.0, coupling=1.5, eta=1e-10, mu_left=50.0,
                                mu_right=-50.0)
    open_channels = 0
    for e in range(s.energies.size):
        r = oracle.solve_g(s, e)
        o = oracle.obc_self_energies(s, e)
        I_left = np.trace(o["L_L"] @ r["G_diag"][0] - o["G_L"] @ r["L_diag"][0])
        I_right = np.trace(o["L_R"] @ r["G_diag"][-1] - o["G_R"] @ r["L_diag"][-1])
        T = oracle.transmission(s, e)
        tol = 1e-6 * max(1.0, T)
        assert abs(I_left - T) <= tol and abs(I_right + T) <= tol, (e, I_left, I_right, T)
        assert np.allclose(oracle.bond_currents(s.H_upper, r["L_upper"]), T, rtol=1e-6, atol=1e-8)
        open_channels += T > 0.5
    assert open_channels >= 2


def test_two_block_inverse_closed_form():
    """N = 2, no contacts: blocks of the 2x2 block inverse via the Schur complement."""
    rng = np.random.default_rng(2)
    bs = 3
    A = synthetic.cn(rng, (2, bs, bs)) + 3 * np.eye(bs)
    Bu = synthetic.cn(rng, (1, bs, bs))
    s = synthetic.GSystem(H_diag=-A, H_upper=-Bu, energies=np.array([0.0]), eta=0.0, mu_left=0,
                          mu_right=0, kT=0.025, obc=False)
    # M = 0*I - H = A on the diagonal, Bu above, Bu^H below
    r = oracle.solve_g(s, 0)
    A11, A22, A12, A21 = A[0], A[1], Bu[0], Bu[0].conj().T
    inv = np.linalg.inv
    X11 = inv(A11 - A12 @ inv(A22) @ A21)
    X22 = inv(A22 - A21 @ inv(A11) @ A12)
    X12 = -inv(A11) @ A12 @ X22
    X21 = -inv(A22) @ A21 @ X11
    assert rel_fro(r["R_diag"][0], X11) < 1e-13
    assert rel_fro(r["R_diag"][1], X22) < 1e-13
    assert rel_fro(r["R_upper"][0], X12) < 1e-13
    assert rel_fro(r["R_lower"][0], X21) < 1e-13


def test_scalar_continued_fraction():
    """b = 1, no contacts: X_11 = 1/(a1 - u1 l1/(a2 - u2 l2/(...)))."""
    rng = np.random.default_rng(4)
    nb = 6
    a = rng.standard_normal(nb) + 1j * rng.standard_normal(nb) + 4
    u = rng.standard_normal(nb - 1)
    s = synthetic.GSystem(H_diag=(-a).reshape(nb, 1, 1).astype(np.complex128),
                          H_upper=(-u).reshape(nb - 1, 1, 1).astype(np.complex128),
                          energies=np.array([0.0]), eta=0.0, mu_left=0, mu_right=0, kT=0.025, obc=False)
    r = oracle.solve_g(s, 0)
    acc = a[-1]
    for i in range(nb - 2, -1, -1):
        acc = a[i] - u[i] * u[i] / acc
    assert abs(r["R_diag"][0][0, 0] - 1 / acc) < 1e-14


@pytest.fixture(scope="module")
def dev():
    return synthetic.random_device(21, 6, 8, 12)


def test_lesser_greater_anti_hermitian(dev):
    for e in (0, 5, 11):
        r = oracle.solve_g(dev, e, symmetrize=False)
        for X in (r["XL"], r["XG"]):
            assert np.abs(X + X.conj().T).max() <= 1e-12 * np.abs(X).max()


def test_greater_minus_lesser_identity(dev):
    """G^> - G^< = G^R - G^A + 2 i eta G^R G^A (S = I; eta enters only M~)."""
    for e in (1, 6, 10):
        r = oracle.solve_g(dev, e, symmetrize=False)
        XR = r["XR"]
        rhs = XR - XR.conj().T + 2j * dev.eta * XR @ XR.conj().T
        scale = max(np.abs(r["XG"]).max(), np.abs(r["XL"]).max(), np.abs(XR).max())
        assert np.abs(r["XG"] - r["XL"] - rhs).max() <= 1e-12 * scale


def test_spectral_functions_psd(dev):
    for e in (2, 7):
        r = oracle.solve_g(dev, e)
        for i in range(dev.nb):
            A = 1j * (r["R_diag"][i] - r["R_diag"][i].conj().T)
            for Mx in (A, -1j * r["L_diag"][i], 1j * r["G_diag"][i]):
                w = np.linalg.eigvalsh((Mx + Mx.conj().T) / 2)
                assert w.min() >= -1e-10 * max(1.0, np.abs(w).max())


def test_equilibrium_relation():
    s = synthetic.random_device(8, 5, 4, 6)
    s.mu_left = s.mu_right = 0.05
    for e in range(6):
        r = oracle.solve_g(s, e, symmetrize=False)
        XR = r["XR"]
        f = float(oracle.fermi(s.energies[e], 0.05, s.kT))
        ref = -f * (XR - XR.conj().T + 2j * s.eta * XR @ XR.conj().T)
        assert np.abs(r["XL"] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_fermi_limits_and_symmetry():
    assert oracle.fermi(1e6, 0.0, 0.025) == 0.0
    assert oracle.fermi(-1e6, 0.0, 0.025) == 1.0
    x = np.linspace(-1, 1, 11)
    assert np.allclose(oracle.fermi(x, 0.0, 0.1) + oracle.fermi(-x, 0.0, 0.1), 1.0, atol=1e-15)
    assert abs(oracle.fermi(0.0, 0.0, 0.1) - 0.5) < 1e-16


def test_scattering_inputs_fluctuation_dissipation():
    """The nanoribbon inputs satisfy Sigma^> - Sigma^< = Sigma^R - Sigma^A."""
    s = synthetic.nanoribbon(nb=3, n_puc=2, puc=8, n_energies=4)
    assert np.allclose(s.sigG_diag - s.sigL_diag, s.sigR_diag - np.conj(s.sigR_diag), atol=1e-18)


def test_sampled_banded_matches_dense():
    s = synthetic.nanoribbon(nb=5, n_puc=2, puc=6, n_energies=3)
    for e in (0, 2):
        d = oracle.solve_g(s, e)
        smp = oracle.solve_g_sampled(s, e, [0, 2, 4])
        for i, r in smp.items():
            assert rel_fro(r["R_diag"], d["R_diag"][i]) < 1e-12
            assert rel_fro(r["L_diag"], d["L_diag"][i]) < 1e-11
            assert rel_fro(r["G_diag"], d["G_diag"][i]) < 1e-11
            if i + 1 < s.nb:
                assert rel_fro(r["R_upper"], d["R_upper"][i]) < 1e-12
                assert rel_fro(r["R_lower"], d["R_lower"][i]) < 1e-12
                assert rel_fro(r["L_upper"], d["L_upper"][i]) < 1e-11
                assert rel_fro(r["G_upper"], d["G_upper"][i]) < 1e-11


# ---------------------------------------------------------------- W system pins

@pytest.fixture(scope="module")
def wsmall():
    return synthetic.w_system(nb=4, ny=2, nz=2, nx=8, spacing=2.2, r_cut=5.0, n_energies=3)


def test_w_system_inputs_block_tridiagonal(wsmall):
    """With cell length > 3 r_cut, V P^R and V P^<> V^H have no blocks beyond the first
    off-diagonal (the BT exactness the W solve relies on)."""
    bs, nb = wsmall.bs, wsmall.nb
    M, BL, BG, V = oracle.assemble_w(wsmall, 0)
    for A in (M, BL, BG):
        for i in range(nb):
            for j in range(nb):
                if abs(i - j) > 1:
                    assert np.abs(A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]).max() == 0.0


def test_w_greater_minus_lesser_identity(wsmall):
    """W^> - W^< = W^R - W^A exactly when P^> - P^< = P^R - P^A and V = V^H."""
    for e in range(3):
        M, BL, BG, V = oracle.assemble_w(wsmall, e)
        XR = np.linalg.inv(M)
        WR = XR @ V
        WL = XR @ BL @ XR.conj().T
        WG = XR @ BG @ XR.conj().T
        assert np.abs((WG - WL) - (WR - WR.conj().T)).max() <= 1e-12 * np.abs(WR).max()


def test_w_solution_satisfies_system(wsmall):
    """(I - V P^R) W^R = V and W^< = W^R P^< W^A (Table 2)."""
    r = oracle.solve_w(wsmall, 1, symmetrize=False)
    nb, bs = wsmall.nb, wsmall.bs
    V = oracle.bt_dense(wsmall.V_diag, wsmall.V_upper)
    PRd, PRu, PRl, PLd, PLu, _, _ = wsmall.P_blocks(1)
    PR = oracle.bt_dense(PRd, PRu, PRl)
    PL = oracle.bt_dense(PLd, PLu, lower_sign=-1.0)
    assert np.abs((np.eye(nb * bs) - V @ PR) @ r["WR"] - V).max() < 1e-12
    WL = r["WR"] @ PL @ r["WR"].conj().T
    d, u, _ = oracle.selected_blocks(WL, nb, bs)
    assert rel_fro(d, r["L_diag"]) < 1e-12 and rel_fro(u, r["L_upper"]) < 1e-12


# ---------------------------------------------------------------- mutation tests
# A plausible mistake planted in the oracle (on the CPU) must fail a pin above.

def _periodic_device(seed, bs, nb, energies, eta):
    rng = np.random.default_rng(seed)
    h00 = synthetic.cn(rng, (bs, bs))
    h00 = (h00 + h00.conj().T) / 2
    h01 = synthetic.cn(rng, (bs, bs))
    return synthetic.GSystem(H_diag=np.broadcast_to(h00, (nb, bs, bs)).copy(),
                             H_upper=np.broadcast_to(h01, (nb - 1, bs, bs)).copy(),
                             energies=np.asarray(energies, dtype=np.float64), eta=eta, mu_left=0.0,
                             mu_right=0.0, kT=0.025), h00, h01


def bloch_integral(z, h00, h01, nk=4096):
    """Diagonal cell block of the infinite periodic chain's G^R by the Bloch sum
    G_00 = (1/2pi) int dk (z - h00 - h01 e^{ik} - h01^H e^{-ik})^{-1} (trapezoid rule, which
    converges exponentially for the periodic integrand)."""
    bs = h00.shape[0]
    acc = np.zeros((bs, bs), dtype=np.complex128)
    for k in 2 * np.pi * np.arange(nk) / nk:
        acc += np.linalg.inv(z * np.eye(bs) - h00 - h01 * np.exp(1j * k) - h01.conj().T * np.exp(-1j * k))
    return acc / nk


def test_periodic_device_equals_bloch_integral():
    """A segment of a periodic chain with both contacts attached is the infinite chain: every
    diagonal block of G^R equals the Bloch-sum G_00.  With a non-symmetric coupling this pins
    the direction of n and n' in both leads."""
    s, h00, h01 = _periodic_device(5, 3, 5, [-0.6, 0.5], 0.05)
    for e, E in enumerate(s.energies):
        r = oracle.solve_g(s, e)
        ref = bloch_integral(E + 1j * s.eta, h00, h01)
        for i in range(s.nb):
            assert rel_fro(r["R_diag"][i], ref) < 1e-10


def test_mutation_wrong_lead_orientation_is_caught(monkeypatch):
    orig = oracle.negf.lead_blocks

    def swapped(sysg, e):
        (mL, nL, npL), (mR, nR, npR) = orig(sysg, e)
        return (mL, npL, nL), (mR, npR, nR)  # transposed couplings

    monkeypatch.setattr(oracle.negf, "lead_blocks", swapped)
    s, h00, h01 = _periodic_device(5, 3, 5, [-0.6], 0.05)
    r = oracle.solve_g(s, 0)
    ref = bloch_integral(-0.6 + 1j * s.eta, h00, h01)
    assert rel_fro(r["R_diag"][0], ref) > 1e-3


def test_mutation_dropped_decimation_term_is_caught(monkeypatch):
    def bad(m, n, n_prime, tol=1e-14, maxit=100):
        a, b, e = n.copy(), n_prime.copy(), m.copy()
        es = e.copy()
        for _ in range(maxit):
            g = np.linalg.inv(e)
            es = es - a @ g @ b
            e = e - a @ g @ b  # dropped the b g a term
            a = -(a @ g @ a)
            b = -(b @ g @ b)
            if max(np.abs(a).max(), np.abs(b).max()) < tol:
                break
        return np.linalg.inv(es), maxit, True

    eps, t, E = 0.2, -1.0, 0.7
    z = E + 1e-3j
    try:
        x, _, _ = bad(np.array([[z - eps]]), np.array([[-t]]), np.array([[-t]]))
    except np.linalg.LinAlgError:
        return  # the mutated iteration breaks down: caught
    assert abs(x[0, 0] - chain_surface_closed_form(z, eps, t)) > 1e-6


def test_mutation_wrong_fluctuation_dissipation_sign_is_caught(dev):
    r = oracle.solve_g(dev, 3)
    for i in range(dev.nb):
        bad = 1j * r["L_diag"][i]  # would be -i G^< if the sign of B^< were flipped
        w = np.linalg.eigvalsh((bad + bad.conj().T) / 2)
        if np.abs(w).max() > 1e-12:
            assert w.min() < 0
            return
    pytest.fail("no block had a nonzero lesser function")


def test_mutation_w_product_order_is_caught(wsmall, monkeypatch):
    """M = I - P^R V instead of I - V P^R: the solution no longer satisfies (I - V P^R) W^R = V."""
    orig = oracle.negf.assemble_w

    def swapped(wsys, e):
        M, BL, BG, V = orig(wsys, e)
        PRd, PRu, PRl, *_ = wsys.P_blocks(e)
        PR = oracle.bt_dense(PRd, PRu, PRl)
        return np.eye(M.shape[0]) - PR @ V, BL, BG, V

    monkeypatch.setattr(oracle.negf, "assemble_w", swapped)
    r = oracle.solve_w(wsmall, 1, symmetrize=False)
    V = oracle.bt_dense(wsmall.V_diag, wsmall.V_upper)
    PRd, PRu, PRl, *_ = wsmall.P_blocks(1)
    PR = oracle.bt_dense(PRd, PRu, PRl)
    resid = np.abs((np.eye(V.shape[0]) - V @ PR) @ r["WR"] - V).max()
    assert resid > 1e-6 * np.abs(V).max()


def test_mutation_hermitian_instead_of_antihermitian_symmetrisation_is_caught(dev, monkeypatch):
    """(X + X^H)/2 in place of (X - X^H)/2 (Sec. 5.2) keeps only the rounding noise of the lesser
    and greater functions: the G^> - G^< identity of Table 2, which the symmetrised blocks satisfy,
    no longer holds."""
    bs = dev.bs

    def identity_error():
        r = oracle.solve_g(dev, 3)
        XR = r["XR"]
        lhs = r["G_diag"][0] - r["L_diag"][0]
        rhs = (XR - XR.conj().T + 2j * dev.eta * XR @ XR.conj().T)[:bs, :bs]
        return np.abs(lhs - rhs).max() / np.abs(rhs).max()

    assert identity_error() < 1e-8
    monkeypatch.setattr(oracle.negf, "symmetrize_lesser", lambda X: 0.5 * (X + X.conj().T))
    bad = identity_error()
    assert bad > 1e-3, bad
