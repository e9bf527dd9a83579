"""Dense CPU oracle (test infrastructure only; see the package docstring).

Notation follows the paper: M(E) = E S - H (Table 2), B^R_scatt = Sigma^R, B^<> = Sigma^<>,
M~ = M - B^R_scatt - B^R_OBC (Table 2), x^R the lead surface function of Eq. 4 with blocks
m, n, n' of M - B^R_scatt.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

__all__ = [
    "fermi", "bt_dense", "sancho_rubio", "sancho_rubio_mp", "surface_gf_eig", "surface_function",
    "lead_blocks", "obc_self_energies",
    "assemble_g", "selected_blocks", "symmetrize_lesser", "solve_g", "assemble_w", "solve_w",
    "transmission", "bond_currents", "block_rows_banded", "solve_g_sampled", "w_bt_blocks", "solve_w_sampled",
    "w_extended_chain",
    "w_lead_fold", "solve_w_contacts", "solve_w_long_leads",
]


def fermi(E, mu, kT):
    """Fermi-Dirac occupation 1 / (1 + exp((E - mu)/kT)) of a contact (Sec. 4.2: the lesser/greater
    boundary blocks carry the contacts' occupations), evaluated without overflow."""
    x = (np.asarray(E, dtype=np.float64) - mu) / kT
    ex = np.exp(-np.abs(x))
    return np.where(x > 0, ex / (1.0 + ex), 1.0 / (1.0 + ex))


def bt_dense(diag, upper, lower=None, lower_sign=1.0):
    """Dense n x n matrix from BT blocks (the block-tridiagonal operands of Eq. 1 and Table 2).
    lower=None means block (i+1,i) = lower_sign * upper[i]^H
    (lower_sign = +1 Hermitian pattern, -1 anti-Hermitian pattern)."""
    nb, bs = diag.shape[0], diag.shape[1]
    A = np.zeros((nb * bs, nb * bs), dtype=np.complex128)
    for i in range(nb):
        A[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] = diag[i]
    for i in range(nb - 1):
        A[i * bs:(i + 1) * bs, (i + 1) * bs:(i + 2) * bs] = upper[i]
        lo = lower[i] if lower is not None else lower_sign * np.conj(upper[i].T)
        A[(i + 1) * bs:(i + 2) * bs, i * bs:(i + 1) * bs] = lo
    return A


def sancho_rubio(m, n, n_prime, tol=1e-14, maxit=100):
    """Surface function x solving x = (m - n x n')^{-1} (Eq. 4) by Sancho-Rubio decimation.

    Decimation of every second cell of the semi-infinite chain with diagonal blocks m,
    coupling n (cell j -> j+1, away from the device) and n' (j+1 -> j).  With g = e^{-1}:
        e_s <- e_s - a g b,   e <- e - a g b - b g a,   a <- -a g a,   b <- -b g b
    starting from a = n, b = n', e = e_s = m; stop when max|a|, max|b| <= tol * max|n|.
    Returns (x = e_s^{-1}, iterations, converged).
    """
    a = np.array(n, dtype=np.complex128)
    b = np.array(n_prime, dtype=np.complex128)
    e = np.array(m, dtype=np.complex128)
    es = e.copy()
    ref = max(np.abs(a).max(), np.abs(b).max())
    if ref == 0.0:
        return np.linalg.inv(es), 0, True
    it = 0
    converged = False
    while it < maxit:
        it += 1
        g = np.linalg.inv(e)
        agb = a @ g @ b
        bga = b @ g @ a
        es = es - agb
        e = e - agb - bga
        a = -(a @ g @ a)
        b = -(b @ g @ b)
        if max(np.abs(a).max(), np.abs(b).max()) <= tol * ref:
            converged = True
            break
    return np.linalg.inv(es), it, converged


def surface_gf_eig(m, n, n_prime):
    """Surface function of Eq. 4 by the direct route (Eq. 6 with N_U = 1): solve the
    linearised quadratic eigenproblem (n' lam^{-1} + m + n lam) phi = 0, keep the bs modes
    with |lam| < 1 (decaying away from the device), T = Phi Lam Phi^{-1}, x = (m + n T)^{-1}."""
    bs = m.shape[0]
    I = np.eye(bs)
    Z = np.zeros((bs, bs))
    A = np.block([[Z, I], [-n_prime, -m]])
    B = np.block([[I, Z], [Z, n]])
    lam, vec = sla.eig(A, B)
    order = np.argsort(np.abs(lam))
    keep = order[:bs]
    if not np.all(np.abs(lam[keep]) < 1.0):
        raise ValueError("fewer than bs decaying modes")
    Phi = vec[:bs, keep]
    T = Phi @ np.diag(lam[keep]) @ np.linalg.inv(Phi)
    return np.linalg.inv(m + n @ T)


def sancho_rubio_mp(m, n, n_prime, dps=40, tol=1e-30, maxit=400):
    """The decimation of sancho_rubio (Sec. 4.2, Eq. 4) carried out in mpmath arithmetic with `dps`
    significant decimal digits, for small blocks.  The inputs are exact binary numbers, so the
    result, rounded to complex128, is the surface function of the given FP64 blocks to full
    FP64 accuracy wherever the decimation converges.  It decides which FP64 route is right where
    the two disagree (near band edges, at small eta).  Returns (x as complex128, iterations,
    converged)."""
    import mpmath as mp

    def to_mp(A):
        A = np.asarray(A, dtype=np.complex128)
        M = mp.matrix(A.shape[0], A.shape[1])
        for i in range(A.shape[0]):
            for j in range(A.shape[1]):
                M[i, j] = mp.mpc(float(A[i, j].real), float(A[i, j].imag))
        return M

    def maxabs(M):
        return max(abs(M[i, j]) for i in range(M.rows) for j in range(M.cols))

    with mp.workdps(dps):
        a, b, e = to_mp(n), to_mp(n_prime), to_mp(m)
        es = e.copy()
        ref = max(maxabs(a), maxabs(b))
        it, converged = 0, ref == 0
        while not converged and it < maxit:
            it += 1
            g = e ** -1
            agb = a * g * b
            bga = b * g * a
            es = es - agb
            e = e - agb - bga
            a = -(a * g * a)
            b = -(b * g * b)
            converged = max(maxabs(a), maxabs(b)) <= tol * ref
        x = es ** -1
        out = np.array([[complex(x[i, j]) for j in range(x.cols)] for i in range(x.rows)], dtype=np.complex128)
    return out, it, converged


def surface_function(m, n, n_prime, route="decimation", tol=1e-14, maxit=100):
    """Surface function x = (m - n x n')^{-1} of Eq. 4 by one of three routes:
      "decimation"  Sancho-Rubio in FP64 (sancho_rubio), the solver the paper cites;
      "eig"         the direct route through the decaying modes of the lead (Eq. 6,
                    surface_gf_eig): the definition of the retarded surface function written out;
      "exact"       Sancho-Rubio in extended precision (sancho_rubio_mp), small blocks only.
    FP64 decimation loses accuracy where a lead mode decays slowly (energies near a band edge at
    small eta: up to ~1e-8 relative); the eigen route keeps FP64 accuracy there (the tests check
    both against the extended-precision route).  Returns (x, iterations, converged)."""
    if route == "decimation":
        return sancho_rubio(m, n, n_prime, tol, maxit)
    if route == "eig":
        return surface_gf_eig(m, n, n_prime), 0, True
    if route == "exact":
        return sancho_rubio_mp(m, n, n_prime)
    raise ValueError(f"unknown surface-function route {route!r}")


def _M_blocks(sysg, e):
    """Blocks of M - B^R_scatt at energy index e (Table 2, left column: M = E S - H):
    (diag [N,b,b], upper, lower)."""
    z = sysg.energies[e] + 1j * sysg.eta
    nb, bs = sysg.nb, sysg.bs
    I = np.eye(bs)
    diag = z * I[None] - sysg.H_diag
    upper = -sysg.H_upper
    lower = -np.conj(np.swapaxes(sysg.H_upper, 1, 2))
    if sysg.sigR_diag is not None:
        diag = diag - np.stack([np.diag(sysg.sigR_diag[e, i]) for i in range(nb)])
    return diag, upper, lower


def lead_blocks(sysg, e):
    """(m, n, n') of Eq. 4 for the left and right leads (Sec. 4.2): the edge cells of M - B^R_scatt repeated
    periodically.  Left lead: m = M_11, n = M_21, n' = M_12.  Right: m = M_NN,
    n = M_{N-1,N}, n' = M_{N,N-1}."""
    d, u, l = _M_blocks(sysg, e)
    left = (d[0], l[0], u[0])
    right = (d[-1], u[-1], l[-1])
    return left, right


def obc_self_energies(sysg, e, tol=1e-14, maxit=100, surface="decimation"):
    """Boundary blocks B_OBC at energy index e.  Retarded: n x n' with x from Eq. 4 (by the route
    `surface` of surface_function).  Lesser/greater by fluctuation-dissipation:
        B^<_c = -f_c (B^R_c - B^R_c^H),  B^>_c = (1 - f_c)(B^R_c - B^R_c^H).
    Returns dict with keys R_L, R_R, L_L, L_R, G_L, G_R, it_L, it_R, ok."""
    if sysg.nb < 2:
        raise ValueError("contacts from the edge blocks need at least two blocks")
    (mL, nL, npL), (mR, nR, npR) = lead_blocks(sysg, e)
    xL, itL, okL = surface_function(mL, nL, npL, surface, tol, maxit)
    xR, itR, okR = surface_function(mR, nR, npR, surface, tol, maxit)
    SL = nL @ xL @ npL
    SR = nR @ xR @ npR
    E = sysg.energies[e]
    fL = float(fermi(E, sysg.mu_left, sysg.kT))
    fR = float(fermi(E, sysg.mu_right, sysg.kT))
    gL = SL - SL.conj().T
    gR = SR - SR.conj().T
    return dict(R_L=SL, R_R=SR, L_L=-fL * gL, L_R=-fR * gR, G_L=(1 - fL) * gL, G_R=(1 - fR) * gR,
                it_L=itL, it_R=itR, ok=okL and okR)


def assemble_g(sysg, e, tol=1e-14, maxit=100, surface="decimation"):
    """Dense M~ = E S - H - Sigma^R_scatt - Sigma^R_OBC and B^<> = Sigma^<>_scatt + Sigma^<>_OBC
    (Table 2; the element-wise G assembly of Sec. 4.3.1); `surface` picks the route of the lead
    surface functions (surface_function)."""
    d, u, l = _M_blocks(sysg, e)
    nb, bs = sysg.nb, sysg.bs
    M = bt_dense(d, u, l)
    n = nb * bs
    BL = np.zeros((n, n), dtype=np.complex128)
    BG = np.zeros((n, n), dtype=np.complex128)
    if sysg.sigL_diag is not None:
        BL += np.diag(sysg.sigL_diag[e].reshape(-1))
    if sysg.sigG_diag is not None:
        BG += np.diag(sysg.sigG_diag[e].reshape(-1))
    info = {}
    if sysg.obc:
        o = obc_self_energies(sysg, e, tol, maxit, surface)
        M[:bs, :bs] -= o["R_L"]
        M[-bs:, -bs:] -= o["R_R"]
        BL[:bs, :bs] += o["L_L"]
        BL[-bs:, -bs:] += o["L_R"]
        BG[:bs, :bs] += o["G_L"]
        BG[-bs:, -bs:] += o["G_R"]
        info = o
    return M, BL, BG, info


def selected_blocks(X, nb, bs):
    """Diagonal, upper (i,i+1) and lower (i+1,i) blocks of a dense matrix: the selected blocks of
    X that Sec. 3 asks for."""
    diag = np.stack([X[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] for i in range(nb)])
    if nb > 1:
        upper = np.stack([X[i * bs:(i + 1) * bs, (i + 1) * bs:(i + 2) * bs] for i in range(nb - 1)])
        lower = np.stack([X[(i + 1) * bs:(i + 2) * bs, i * bs:(i + 1) * bs] for i in range(nb - 1)])
    else:
        upper = np.zeros((0, bs, bs), dtype=X.dtype)
        lower = np.zeros((0, bs, bs), dtype=X.dtype)
    return diag, upper, lower


def symmetrize_lesser(X):
    """Sec. 5.2: X_ij <- (X_ij - X_ji^*)/2 on the whole matrix."""
    return 0.5 * (X - X.conj().T)


def solve_g(sysg, e, symmetrize=True, tol=1e-14, maxit=100, surface="decimation"):
    """Selected blocks of X^R = M~^{-1} and X^<> = X^R B^<> X^R^H at energy index e, by dense
    inversion (Eq. 1), with the lead surface functions by the route `surface`.  Returns dict:
    R_diag, R_upper, R_lower, L_diag, L_upper, G_diag,
    G_upper (lesser/greater lower blocks are -upper^H), plus 'info' from the OBC."""
    M, BL, BG, info = assemble_g(sysg, e, tol, maxit, surface)
    XR = np.linalg.inv(M)
    XL = XR @ BL @ XR.conj().T
    XG = XR @ BG @ XR.conj().T
    if symmetrize:
        XL = symmetrize_lesser(XL)
        XG = symmetrize_lesser(XG)
    nb, bs = sysg.nb, sysg.bs
    Rd, Ru, Rl = selected_blocks(XR, nb, bs)
    Ld, Lu, _ = selected_blocks(XL, nb, bs)
    Gd, Gu, _ = selected_blocks(XG, nb, bs)
    return dict(R_diag=Rd, R_upper=Ru, R_lower=Rl, L_diag=Ld, L_upper=Lu, G_diag=Gd, G_upper=Gu,
                info=info, XR=XR, XL=XL, XG=XG, M=M, BL=BL, BG=BG)


# ----------------------------------------------------------------------------------------------
# W system (Table 2, right column)
# ----------------------------------------------------------------------------------------------

def assemble_w(wsys, e):
    """Dense M~ = I - V P^R and B^<> = V P^<> V^H (Sec. 4.3.1, W assembly)."""
    nb, bs = wsys.nb, wsys.bs
    V = bt_dense(wsys.V_diag, wsys.V_upper)
    PRd, PRu, PRl, PLd, PLu, PGd, PGu = wsys.P_blocks(e)
    PR = bt_dense(PRd, PRu, PRl)
    PL = bt_dense(PLd, PLu, lower_sign=-1.0)
    PG = bt_dense(PGd, PGu, lower_sign=-1.0)
    n = nb * bs
    M = np.eye(n) - V @ PR
    BL = V @ PL @ V.conj().T
    BG = V @ PG @ V.conj().T
    return M, BL, BG, V


def solve_w(wsys, e, symmetrize=True):
    """W^R = (I - V P^R)^{-1} V and W^<> = X^R (V P^<> V^H) X^R^H, selected blocks (Table 2, right
    column; no contacts)."""
    M, BL, BG, V = assemble_w(wsys, e)
    XR = np.linalg.inv(M)
    WR = XR @ V
    WL = XR @ BL @ XR.conj().T
    WG = XR @ BG @ XR.conj().T
    if symmetrize:
        WL = symmetrize_lesser(WL)
        WG = symmetrize_lesser(WG)
    nb, bs = wsys.nb, wsys.bs
    Rd, Ru, Rl = selected_blocks(WR, nb, bs)
    Ld, Lu, _ = selected_blocks(WL, nb, bs)
    Gd, Gu, _ = selected_blocks(WG, nb, bs)
    XRd, XRu, XRl = selected_blocks(XR, nb, bs)
    return dict(R_diag=Rd, R_upper=Ru, R_lower=Rl, L_diag=Ld, L_upper=Lu, G_diag=Gd, G_upper=Gu,
                XR_diag=XRd, XR_upper=XRu, XR_lower=XRl, M=M, BL=BL, BG=BG, XR=XR, WR=WR)


# ----------------------------------------------------------------------------------------------
# Observables (Sec. 4.5) used as invariants
# ----------------------------------------------------------------------------------------------

def transmission(sysg, e):
    """Landauer transmission T = Tr[Gam_L G^R_1N Gam_R G^A_N1] with Gam_c = i(B^R_c - B^R_c^H).
    Not a step of the method: a physical observable of the G system (Table 2) that the pins
    compare with closed forms and with the currents."""
    M, _, _, o = assemble_g(sysg, e)
    bs = sysg.bs
    XR = np.linalg.inv(M)
    GamL = 1j * (o["R_L"] - o["R_L"].conj().T)
    GamR = 1j * (o["R_R"] - o["R_R"].conj().T)
    G1N = XR[:bs, -bs:]
    return float(np.real(np.trace(GamL @ G1N @ GamR @ G1N.conj().T)))


def bond_currents(H_upper, L_upper):
    """Bond current between cells i and i+1: I_i = 2 Re Tr[H_{i,i+1} G^<_{i+1,i}] with
    G^<_{i+1,i} = -(G^<_{i,i+1})^H (anti-Hermiticity, Sec. 5.2).  Not a step of the method: an
    observable the pins use to check the off-diagonal lesser blocks."""
    out = []
    for i in range(H_upper.shape[0]):
        Glow = -np.conj(L_upper[i].T)
        out.append(2.0 * np.real(np.trace(H_upper[i] @ Glow)))
    return np.array(out)


# ----------------------------------------------------------------------------------------------
# Sampled blocks for devices too large for a dense inverse: rows of M~^{-1} by banded LU
# ----------------------------------------------------------------------------------------------

def _band_storage(A_diag, A_upper, A_lower, transpose):
    """LAPACK band storage of a BT matrix (or its transpose) with l = u = 2 bs - 1 (the BT
    structure of Eq. 1 as a band matrix)."""
    nb, bs = A_diag.shape[0], A_diag.shape[1]
    n = nb * bs
    kl = ku = 2 * bs - 1
    ab = np.zeros((kl + ku + 1, n), dtype=np.complex128)

    def put(block, r0, c0):
        if transpose:
            block = block.T
            r0, c0 = c0, r0
        rr, cc = np.meshgrid(np.arange(bs) + r0, np.arange(bs) + c0, indexing="ij")
        ab[ku + rr - cc, cc] = block

    for i in range(nb):
        put(A_diag[i], i * bs, i * bs)
    for i in range(nb - 1):
        put(A_upper[i], i * bs, (i + 1) * bs)
        put(A_lower[i], (i + 1) * bs, i * bs)
    return ab, kl, ku


def block_rows_banded(A_diag, A_upper, A_lower, rows):
    """Full block rows `rows` of A^{-1} for a BT matrix A (Eq. 1), by banded LU of A^T (LAPACK gbsv):
    row block i of A^{-1} is (A^{-T} E_i)^T.  Returns {i: [bs, n] array}."""
    nb, bs = A_diag.shape[0], A_diag.shape[1]
    n = nb * bs
    ab, kl, ku = _band_storage(A_diag, A_upper, A_lower, transpose=True)
    rhs = np.zeros((n, bs * len(rows)), dtype=np.complex128)
    for k, i in enumerate(rows):
        rhs[i * bs:(i + 1) * bs, k * bs:(k + 1) * bs] = np.eye(bs)
    Z = sla.solve_banded((kl, ku), ab, rhs, check_finite=False)
    return {i: Z[:, k * bs:(k + 1) * bs].T.copy() for k, i in enumerate(rows)}


def solve_g_sampled(sysg, e, blocks, symmetrize=True, tol=1e-14, maxit=100, surface="decimation"):
    """Selected blocks (Sec. 3, Eq. 1 and Table 2) at energy index e for block indices `blocks`
    without a dense inverse:
    rows i and i+1 of X^R by banded LU, then X^<>_{ij} = X^R[i,:] B^<> X^R[j,:]^H with the
    (block-diagonal) B^<> of the G system.  Returns {i: dict(R_diag, R_upper, R_lower, L_diag,
    L_upper, G_diag, G_upper)} (upper/lower entries only when i+1 < N)."""
    nb, bs = sysg.nb, sysg.bs
    d, u, l = _M_blocks(sysg, e)
    d = d.copy()
    bl = [np.zeros((bs, bs), np.complex128) for _ in range(nb)]
    bg = [np.zeros((bs, bs), np.complex128) for _ in range(nb)]
    for i in range(nb):
        if sysg.sigL_diag is not None:
            bl[i] += np.diag(sysg.sigL_diag[e, i])
        if sysg.sigG_diag is not None:
            bg[i] += np.diag(sysg.sigG_diag[e, i])
    if sysg.obc:
        o = obc_self_energies(sysg, e, tol, maxit, surface)
        d[0] -= o["R_L"]
        d[-1] -= o["R_R"]
        bl[0] += o["L_L"]
        bl[-1] += o["L_R"]
        bg[0] += o["G_L"]
        bg[-1] += o["G_R"]
    need = sorted(set(list(blocks) + [i + 1 for i in blocks if i + 1 < nb]))
    rows = block_rows_banded(d, u, l, need)

    def quad(ri, rj, bb):
        acc = np.zeros((bs, bs), np.complex128)
        for k in range(nb):
            acc += ri[:, k * bs:(k + 1) * bs] @ bb[k] @ rj[:, k * bs:(k + 1) * bs].conj().T
        return acc

    out = {}
    for i in blocks:
        ri = rows[i]
        r = dict(R_diag=ri[:, i * bs:(i + 1) * bs])
        Ld = quad(ri, ri, bl)
        Gd = quad(ri, ri, bg)
        if symmetrize:
            Ld = 0.5 * (Ld - Ld.conj().T)
            Gd = 0.5 * (Gd - Gd.conj().T)
        r["L_diag"], r["G_diag"] = Ld, Gd
        if i + 1 < nb:
            rj = rows[i + 1]
            r["R_upper"] = ri[:, (i + 1) * bs:(i + 2) * bs]
            r["R_lower"] = rj[:, i * bs:(i + 1) * bs]
            Lu = quad(ri, rj, bl)
            Gu = quad(ri, rj, bg)
            if symmetrize:
                Lu = 0.5 * (Lu - quad(rj, ri, bl).conj().T)
                Gu = 0.5 * (Gu - quad(rj, ri, bg).conj().T)
            r["L_upper"], r["G_upper"] = Lu, Gu
        out[i] = r
    return out


def w_bt_blocks(wsys, e):
    """Block-tridiagonal blocks of M = I - V P^R and B^<> = V P^<> V^H (Table 2, right column) at
    energy index e, each block summed from the products of the V and P blocks it contains:
    M_ij = delta_ij I - sum_k V_ik P_kj and B_ij = sum_{k,l} V_ik P_kl (V_jl)^H for |i - j| <= 1.
    Exact when the cells are longer than three cut-off radii (the blocks two or more cells apart
    then vanish).  Returns (M_d, M_u, M_l, BL_d, BL_u, BG_d, BG_u, V block accessor)."""
    nb, bs = wsys.nb, wsys.bs
    PRd, PRu, PRl, PLd, PLu, PGd, PGu = wsys.P_blocks(e)

    def Vb(i, j):
        if i == j:
            return wsys.V_diag[i]
        return wsys.V_upper[i] if j == i + 1 else wsys.V_upper[j].conj().T

    def Pb(d, u, l, i, j):
        if i == j:
            return d[i]
        if j == i + 1:
            return u[i]
        return l[j] if l is not None else -u[j].conj().T

    near = lambda i: [k for k in (i - 1, i, i + 1) if 0 <= k < nb]
    I = np.eye(bs)
    Md = np.stack([I - sum(Vb(i, k) @ Pb(PRd, PRu, PRl, k, i) for k in near(i)) for i in range(nb)])
    Mu = np.stack([-sum(Vb(i, k) @ Pb(PRd, PRu, PRl, k, i + 1) for k in near(i) if abs(k - i - 1) <= 1)
                   for i in range(nb - 1)]) if nb > 1 else np.zeros((0, bs, bs), np.complex128)
    Ml = np.stack([-sum(Vb(i + 1, k) @ Pb(PRd, PRu, PRl, k, i) for k in near(i + 1) if abs(k - i) <= 1)
                   for i in range(nb - 1)]) if nb > 1 else np.zeros((0, bs, bs), np.complex128)

    def B(d, u, i, j):
        acc = np.zeros((bs, bs), np.complex128)
        for k in near(i):
            for l_ in near(j):
                if abs(k - l_) <= 1:
                    acc += Vb(i, k) @ Pb(d, u, None, k, l_) @ Vb(j, l_).conj().T
        return acc

    BLd = np.stack([B(PLd, PLu, i, i) for i in range(nb)])
    BGd = np.stack([B(PGd, PGu, i, i) for i in range(nb)])
    BLu = np.stack([B(PLd, PLu, i, i + 1) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, bs, bs), np.complex128)
    BGu = np.stack([B(PGd, PGu, i, i + 1) for i in range(nb - 1)]) if nb > 1 else np.zeros((0, bs, bs), np.complex128)
    return Md, Mu, Ml, BLd, BLu, BGd, BGu, Vb


def solve_w_sampled(wsys, e, blocks, symmetrize=True):
    """Selected blocks of W^R = X^R V and W^<> = X^R B^<> X^R^H (Table 2, right column; no
    contacts) for block indices `blocks` without a dense inverse: rows of X^R = M^{-1} by banded LU
    (block_rows_banded), then the products with the block-tridiagonal V and B^<> of w_bt_blocks.
    Returns {i: dict(R_diag, R_upper, R_lower, L_diag, L_upper, G_diag, G_upper)} (upper / lower
    entries only when i + 1 < N)."""
    nb, bs = wsys.nb, wsys.bs
    Md, Mu, Ml, BLd, BLu, BGd, BGu, Vb = w_bt_blocks(wsys, e)
    need = sorted(set(list(blocks) + [i + 1 for i in blocks if i + 1 < nb]))
    rows = block_rows_banded(Md, Mu, Ml, need)
    cols = lambda r, k: r[:, k * bs:(k + 1) * bs]

    def wr(r, j):  # (X^R V)_{., j} from a block row of X^R
        return sum(cols(r, k) @ Vb(k, j) for k in (j - 1, j, j + 1) if 0 <= k < nb)

    def Bb(d, u, k, l_):
        if k == l_:
            return d[k]
        return u[k] if l_ == k + 1 else -u[l_].conj().T

    def row_times_b(ri, d, u):  # the block row X^R[i, :] B^<> (B block-tridiagonal)
        return [sum(cols(ri, k) @ Bb(d, u, k, l_) for k in (l_ - 1, l_, l_ + 1) if 0 <= k < nb) for l_ in range(nb)]

    def quad(tb, rj):  # (X^R[i, :] B^<>) X^R[j, :]^H
        return sum(tb[l_] @ cols(rj, l_).conj().T for l_ in range(nb))

    tbs = {}
    for j in need:
        tbs[j] = (row_times_b(rows[j], BLd, BLu), row_times_b(rows[j], BGd, BGu))
    out = {}
    for i in blocks:
        ri = rows[i]
        r = dict(R_diag=wr(ri, i))
        Ld, Gd = quad(tbs[i][0], ri), quad(tbs[i][1], ri)
        if symmetrize:
            Ld, Gd = 0.5 * (Ld - Ld.conj().T), 0.5 * (Gd - Gd.conj().T)
        r["L_diag"], r["G_diag"] = Ld, Gd
        if i + 1 < nb:
            rj = rows[i + 1]
            r["R_upper"], r["R_lower"] = wr(ri, i + 1), wr(rj, i)
            Lu, Gu = quad(tbs[i][0], rj), quad(tbs[i][1], rj)
            if symmetrize:
                Lu = 0.5 * (Lu - quad(tbs[i + 1][0], ri).conj().T)
                Gu = 0.5 * (Gu - quad(tbs[i + 1][1], ri).conj().T)
            r["L_upper"], r["G_upper"] = Lu, Gu
        out[i] = r
    return out


# ----------------------------------------------------------------------------------------------
# W system with contacts (Sec. 4.2: retarded OBC by Eq. 4, lesser/greater OBC by the discrete
# Lyapunov equation of Eq. 7).  Groundwork for the W contacts: the CUDA path does not solve W
# with contacts.
#
# Reading.  Each lead is the periodic continuation of the device's edge cell (its diagonal
# blocks and its coupling to the next cell inward), for V and for P.  M = I - V P^R and
# B^<> = V P^<> V^H are then block-tridiagonal over the whole chain (cells longer than 3 r_cut).
# A lead with bulk blocks m, n (coupling from a cell to the next one away from the device),
# n', and right-hand-side blocks b, c (c = B_{far, near}) folds into the device's edge cell as
#     x^R = (m - n x^R n')^{-1}                         (Eq. 4)
#     y = n x^R c,   a = x^R n,   q = x^R (b - y + y^H) x^R^H
#     w^<> = q + a w^<> a^H                              (Eq. 7; a Stein equation)
#     B^R_OBC = n x^R n',   B^<>_OBC = n w^<> n^H - (y - y^H)
# — the fixed point of the forward recursion of Eq. 9-10 run along the lead from infinity.  The
# edge cells' own blocks of M and B include the products with the first lead cell.  Eq. 7 is
# printed with a minus sign before a w a^H; the fixed point has a plus sign (a scalar factor in a
# cannot change that sign), and the long-lead pin decides between the two.
# ----------------------------------------------------------------------------------------------

def w_extended_chain(wsys, e, n_lead):
    """BT blocks of V, P^R, P^<, P^> (Table 2, right column) over n_lead lead cells, the device,
    n_lead lead cells (Sec. 4.2: periodic leads): each
    lead repeats the device's edge cell and its coupling to the next cell inward.  Returns
    (V_d, V_u, PR_d, PR_u, PR_l, PL_d, PL_u, PG_d, PG_u) for the whole chain."""
    nb = wsys.nb
    PRd, PRu, PRl, PLd, PLu, PGd, PGu = wsys.P_blocks(e)
    ops_d = [wsys.V_diag, PRd, PLd, PGd]
    ops_u = [wsys.V_upper, PRu, PLu, PGu]

    def extend_d(d):
        return np.concatenate([np.repeat(d[:1], n_lead, 0), d, np.repeat(d[-1:], n_lead, 0)])

    def extend_u(u):
        return np.concatenate([np.repeat(u[:1], n_lead, 0), u, np.repeat(u[-1:], n_lead, 0)])

    Vd, PRd_x, PLd_x, PGd_x = (extend_d(d) for d in ops_d)
    Vu, PRu_x, PLu_x, PGu_x = (extend_u(u) for u in ops_u)
    PRl_x = extend_u(PRl)
    return Vd, Vu, PRd_x, PRu_x, PRl_x, PLd_x, PLu_x, PGd_x, PGu_x


def _w_chain_dense(wsys, e, n_lead):
    """Dense M = I - V P^R, B^<> = V P^<> V^H and V (Table 2, right column) of the chain of
    w_extended_chain."""
    Vd, Vu, PRd, PRu, PRl, PLd, PLu, PGd, PGu = w_extended_chain(wsys, e, n_lead)
    V = bt_dense(Vd, Vu)
    PR = bt_dense(PRd, PRu, PRl)
    PL = bt_dense(PLd, PLu, lower_sign=-1.0)
    PG = bt_dense(PGd, PGu, lower_sign=-1.0)
    n = V.shape[0]
    return np.eye(n) - V @ PR, V @ PL @ V.conj().T, V @ PG @ V.conj().T, V


def w_lead_fold(m, n, n_prime, b, c, tol=1e-14, maxit=200):
    """Retarded and lesser/greater boundary blocks of one lead (Sec. 4.2: Eq. 4 for x^R, the Stein
    equation of Eq. 7 for w^<>; see the reading above).
    Returns (B^R_OBC, B^<>_OBC, x^R, w^<>)."""
    x, _, ok = sancho_rubio(m, n, n_prime, tol, maxit)
    if not ok:
        raise ValueError("decimation did not converge")
    y = n @ x @ c
    a = x @ n
    q = x @ (b - y + y.conj().T) @ x.conj().T
    w = sla.solve_discrete_lyapunov(a, q)   # w = a w a^H + q
    return n @ x @ n_prime, n @ w @ n.conj().T - (y - y.conj().T), x, w


def solve_w_contacts(wsys, e, symmetrize=True):
    """Selected blocks of W^R = X^R V and W^<> = X^<> (Table 2, right column) for the W system with
    both leads attached (Sec. 4.2, Eq. 4 and 7; the reading above), by folding the leads into the
    edge cells and a dense solve of the device.  W^R's edge blocks include V's coupling to the
    first lead cells through X^R_{0,-1} = -X^R_{00} M_{0,-1} x^R_L (and the mirror on the right)."""
    nb, bs = wsys.nb, wsys.bs
    K = 4   # lead cells in the assembly window: cell 1 and cell (K + nb + 2) are bulk lead cells
    M, BL, BG, V = _w_chain_dense(wsys, e, K)
    blk = lambda A, i, j: A[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs]
    d0, d1 = K, K + nb          # device cells [d0, d1)
    sl = slice(d0 * bs, d1 * bs)
    Md = M[sl, sl].copy()
    Bs = {"L": BL[sl, sl].copy(), "G": BG[sl, sl].copy()}
    # left lead: bulk cell 1, away = toward cell 0
    kL = 1
    mL, nL, npL = blk(M, kL, kL), blk(M, kL, kL - 1), blk(M, kL - 1, kL)
    # right lead: bulk cell d1 + 2, away = toward d1 + 3
    kR = d1 + 2
    mR, nR, npR = blk(M, kR, kR), blk(M, kR, kR + 1), blk(M, kR + 1, kR)
    outs = {}
    xs = {}
    for w, B in (("L", BL), ("G", BG)):
        bLb, cL = blk(B, kL, kL), blk(B, kL - 1, kL)
        bRb, cR = blk(B, kR, kR), blk(B, kR + 1, kR)
        rL, lgL, xL, _ = w_lead_fold(mL, nL, npL, bLb, cL)
        rR, lgR, xR, _ = w_lead_fold(mR, nR, npR, bRb, cR)
        Bs[w][:bs, :bs] += lgL
        Bs[w][-bs:, -bs:] += lgR
        xs = {"L": xL, "R": xR, "RL": rL, "RR": rR}
    Md[:bs, :bs] -= xs["RL"]
    Md[-bs:, -bs:] -= xs["RR"]
    XR = np.linalg.inv(Md)
    # W^R = X^R V over the whole chain restricted to device rows: device columns from the
    # device X^R, plus the first lead cell on each side
    Vx = V
    XRfull = np.zeros((nb * bs, (nb + 2) * bs), dtype=np.complex128)   # columns: lead cell, device, lead cell
    XRfull[:, bs:-bs] = XR
    XRfull[:, :bs] = -XR[:, :bs] @ blk(M, d0, d0 - 1) @ xs["L"]        # X^R_{i,-1}
    XRfull[:, -bs:] = -XR[:, -bs:] @ blk(M, d1 - 1, d1) @ xs["R"]      # X^R_{i,N}
    Vrows = Vx[(d0 - 1) * bs:(d1 + 1) * bs, sl]                           # V_{k, device} for k in [d0-1, d1]
    WR = XRfull @ Vrows
    res = {}
    for w in ("L", "G"):
        X = XR @ Bs[w] @ XR.conj().T
        if symmetrize:
            X = symmetrize_lesser(X)
        d, u, _ = selected_blocks(X, nb, bs)
        res[w + "_diag"], res[w + "_upper"] = d, u
    d, u, l = selected_blocks(WR, nb, bs)
    res.update(R_diag=d, R_upper=u, R_lower=l, WR=WR, XR=XR, M=Md, BL=Bs["L"], BG=Bs["G"])
    return res


def solve_w_long_leads(wsys, e, n_lead, symmetrize=True):
    """The same selected blocks from a finite chain with n_lead lead cells on each side, solved
    densely without any boundary condition: converges to solve_w_contacts as n_lead grows (the
    absorbing part of P^R damps the leads).  The pin of the folding (Sec. 4.2: the boundary
    blocks stand for semi-infinite leads)."""
    nb, bs = wsys.nb, wsys.bs
    M, BL, BG, V = _w_chain_dense(wsys, e, n_lead)
    XR = np.linalg.inv(M)
    sl = slice(n_lead * bs, (n_lead + nb) * bs)
    res = {}
    for w, B in (("L", BL), ("G", BG)):
        X = (XR @ B @ XR.conj().T)[sl, sl]
        if symmetrize:
            X = symmetrize_lesser(X)
        d, u, _ = selected_blocks(X, nb, bs)
        res[w + "_diag"], res[w + "_upper"] = d, u
    WR = (XR @ V)[sl, sl]
    d, u, l = selected_blocks(WR, nb, bs)
    res.update(R_diag=d, R_upper=u, R_lower=l)
    return res
