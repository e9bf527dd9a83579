"""Seeded synthetic inputs for block-tridiagonal (BT) NEGF systems.

This module builds *inputs only*: Hamiltonian / Coulomb blocks, scattering
self-energies and energy grids shaped after the devices of the paper's Table 3
(silicon nanowire / nanoribbon transport cells, N_BS = 416 = 4 primitive cells
x 104 orbitals) and after the problem statement of Sec. 3 (Eqs. 1-3, Table 2).
It contains none of the method's arithmetic (no assembly, no decimation, no
inversion). Both the CPU oracle and the GPU path consume these arrays, so a
mismatch between them can never come from a shared helper.

Every array is complex128 (interleaved re/im) laid out as row-major blocks:
diagonal blocks [N][b][b], upper blocks (i, i+1) [N-1][b][b].
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

BASE_SEED = 20250826


def cn(rng: np.random.Generator, shape) -> np.ndarray:
    """Circular complex normal CN(0, 1): E|x|^2 = 1."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


@dataclasses.dataclass
class GSystem:
    """Inputs of the electron (G) system of Table 2.

    H_diag [N,b,b], H_upper [N-1,b,b]; H is Hermitian so block (i+1,i) is
    H_upper[i]^H.  S is the identity (orthogonal MLWF basis, Sec. 4.1).
    Scattering self-energies are either None or diagonal vectors
    sig*_diag [E,N,b] (retarded / lesser / greater).
    """
    H_diag: np.ndarray
    H_upper: np.ndarray
    energies: np.ndarray
    eta: float
    mu_left: float
    mu_right: float
    kT: float
    obc: bool = True
    sigR_diag: Optional[np.ndarray] = None
    sigL_diag: Optional[np.ndarray] = None
    sigG_diag: Optional[np.ndarray] = None

    @property
    def nb(self) -> int:
        return self.H_diag.shape[0]

    @property
    def bs(self) -> int:
        return self.H_diag.shape[1]

    def subset(self, idx) -> "GSystem":
        """Same device on a subset of the energy grid."""
        idx = np.asarray(idx)
        pick = lambda a: None if a is None else np.ascontiguousarray(a[idx])
        return dataclasses.replace(self, energies=np.ascontiguousarray(self.energies[idx]),
                                   sigR_diag=pick(self.sigR_diag), sigL_diag=pick(self.sigL_diag),
                                   sigG_diag=pick(self.sigG_diag))


def random_device(seed: int, nb: int, bs: int, n_energies: int, e_lo: float = -3.0, e_hi: float = 3.0,
                  coupling: float = 0.3, eta: float = 1e-6, mu_left: float = 0.1, mu_right: float = -0.1,
                  kT: float = 0.025) -> GSystem:
    """Random BT device: Hermitian on-site blocks (X + X^H)/sqrt(2)/sqrt(bs), X ~ CN(0,1),
    coupling blocks coupling * X / sqrt(bs); contacts are the edge blocks repeated.
    With nb=8, bs=32, 64 energies on [-3, 3] this is the 8x32 random-device workload."""
    rng = np.random.default_rng(seed)
    X = cn(rng, (nb, bs, bs))
    H_diag = (X + np.conj(np.swapaxes(X, 1, 2))) / np.sqrt(2.0) / np.sqrt(bs)
    H_upper = coupling * cn(rng, (max(nb - 1, 0), bs, bs)) / np.sqrt(bs)
    energies = np.linspace(e_lo, e_hi, n_energies)
    return GSystem(H_diag=np.ascontiguousarray(H_diag), H_upper=np.ascontiguousarray(H_upper),
                   energies=energies, eta=eta, mu_left=mu_left, mu_right=mu_right, kT=kT, obc=True)


def random_device_8x32(seed: int = BASE_SEED) -> GSystem:
    """8 blocks of 32, 64 energies on [-3, 3], eta = 1e-6, Fermi levels +/-0.1, kT = 0.025."""
    return random_device(seed, 8, 32, 64)


def _fermi_occupation(E: np.ndarray, mu: np.ndarray, kT: float) -> np.ndarray:
    # occupation used only to *build* scattering self-energy inputs (Sec. 3: Sigma^<> consistent
    # with Fermi occupations); overflow-safe logistic
    x = (E - mu) / kT
    out = np.empty(np.broadcast(E, mu).shape)
    pos = x > 0
    ex = np.exp(-np.abs(x))
    out[...] = np.where(pos, ex / (1.0 + ex), 1.0 / (1.0 + ex))
    return out


def nanoribbon(seed: int = BASE_SEED + 1, nb: int = 40, n_puc: int = 4, puc: int = 104,
               n_energies: int = 512, e_lo: float = -4.0, e_hi: float = 4.0, eta: float = 1e-6,
               mu_left: float = 0.1, mu_right: float = -0.1, kT: float = 0.025,
               h_density: float = 0.08, c_density: float = 0.10, gamma_max: float = 1e-3) -> GSystem:
    """Nanoribbon-shaped G system (Table 3 shapes: transport cell = n_puc primitive cells of
    `puc` orbitals; defaults give N_B = 40, N_BS = 416, 512 energies on [-4, 4]).

    * H is periodic along transport (every H_ii equal, every H_{i,i+1} equal), as the paper's
      devices built by repeating one primitive cell (Sec. 4.1).
    * H_ii: sparse Hermitian, ~h_density nonzero, values CN(0,1)/sqrt(h_density*bs).
    * H_{i,i+1}: fixed ~c_density nonzero pattern inside the primitive-cell blocks (p, q) with
      q <= p (a cell couples to the next n_puc cells along +x), values
      0.3*CN(0,1)/sqrt(c_density*bs).
    * Sigma^R_scatt = -i*gamma on the diagonal, gamma ~ U(0, gamma_max] per energy and orbital.
    * Sigma^<_scatt = -f_i (Sigma^R - Sigma^A), Sigma^>_scatt = (1 - f_i)(Sigma^R - Sigma^A), with
      the block's chemical potential mu_i interpolated linearly from mu_left to mu_right.
    """
    rng = np.random.default_rng(seed)
    bs = n_puc * puc
    mask = rng.random((bs, bs)) < h_density / 2.0
    mask = mask | mask.T
    vals = cn(rng, (bs, bs)) / np.sqrt(h_density * bs)
    h = np.where(mask, vals, 0.0)
    h = (h + h.conj().T) / np.sqrt(2.0)
    allowed = np.zeros((bs, bs), dtype=bool)
    for p in range(n_puc):
        for q in range(p + 1):
            allowed[p * puc:(p + 1) * puc, q * puc:(q + 1) * puc] = True
    frac_allowed = allowed.mean()
    cmask = allowed & (rng.random((bs, bs)) < min(1.0, c_density / frac_allowed))
    c = np.where(cmask, 0.3 * cn(rng, (bs, bs)) / np.sqrt(c_density * bs), 0.0)
    H_diag = np.ascontiguousarray(np.broadcast_to(h, (nb, bs, bs)))
    H_upper = np.ascontiguousarray(np.broadcast_to(c, (max(nb - 1, 0), bs, bs)))
    energies = np.linspace(e_lo, e_hi, n_energies)
    gamma = gamma_max * (1.0 - rng.random((n_energies, nb, bs)))  # U(0, gamma_max]
    sigR = -1j * gamma
    mu_i = mu_left + (mu_right - mu_left) * (np.arange(nb) / max(nb - 1, 1))
    f = _fermi_occupation(energies[:, None, None], mu_i[None, :, None], kT)
    spectral = sigR - np.conj(sigR)  # Sigma^R - Sigma^A of the input
    sigL = -f * spectral
    sigG = (1.0 - f) * spectral
    return GSystem(H_diag=H_diag, H_upper=H_upper, energies=energies, eta=eta, mu_left=mu_left,
                   mu_right=mu_right, kT=kT, obc=True, sigR_diag=np.ascontiguousarray(sigR),
                   sigL_diag=np.ascontiguousarray(sigL), sigG_diag=np.ascontiguousarray(sigG))


def nanoribbon_40x416(seed: int = BASE_SEED + 1) -> GSystem:
    """The 40 x 416, 512-energy nanoribbon workload."""
    return nanoribbon(seed)


def chain_1d(nb: int, eps: float, t: float, energies, eta: float, mu_left: float = 0.0,
             mu_right: float = 0.0, kT: float = 0.025, bs: int = 1) -> GSystem:
    """Uniform tight-binding chain (on-site eps, hopping t) with bs independent copies
    (h00 = eps*I, h01 = t*I): the textbook case with closed-form surface Green's function."""
    I = np.eye(bs, dtype=np.complex128)
    H_diag = np.ascontiguousarray(np.broadcast_to(eps * I, (nb, bs, bs)))
    H_upper = np.ascontiguousarray(np.broadcast_to(t * I, (max(nb - 1, 0), bs, bs)))
    return GSystem(H_diag=H_diag, H_upper=H_upper, energies=np.asarray(energies, dtype=np.float64),
                   eta=eta, mu_left=mu_left, mu_right=mu_right, kT=kT, obc=True)


# ----------------------------------------------------------------------------------------------
# Screened-interaction (W) system, Table 2 right column.
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class WSystem:
    """Inputs of the W system: bare Coulomb V (real symmetric BT) and polarisation P^{R,<,>}(E).

    P(E) is stored compactly as energy-independent BT bases plus per-energy weights:
      P^R(E) = R0 + r1[e] * R1 - (i/2) * (1 + g1[e]) * Gam
      P^<(E) = -i * a[e] * (1 + g1[e]) * Gam,  P^>(E) = -i * (1 + a[e]) * (1 + g1[e]) * Gam
    with R0, R1 real symmetric and Gam Hermitian positive semidefinite (diagonally dominant),
    so P^> - P^< = P^R - P^A and P^<> are anti-Hermitian.  `P_blocks(e)` expands one energy.
    """
    V_diag: np.ndarray
    V_upper: np.ndarray
    R0_diag: np.ndarray
    R0_upper: np.ndarray
    R1_diag: np.ndarray
    R1_upper: np.ndarray
    Gam_diag: np.ndarray
    Gam_upper: np.ndarray
    r1: np.ndarray
    g1: np.ndarray
    a: np.ndarray
    energies: np.ndarray

    @property
    def nb(self) -> int:
        return self.V_diag.shape[0]

    @property
    def bs(self) -> int:
        return self.V_diag.shape[1]

    def P_blocks(self, e: int):
        """(PR_diag, PR_upper, PR_lower, PL_diag, PL_upper, PG_diag, PG_upper) for energy e;
        P^<> lower blocks are -upper^H."""
        s = 1.0 + self.g1[e]
        PR_d = self.R0_diag + self.r1[e] * self.R1_diag - 0.5j * s * self.Gam_diag
        PR_u = self.R0_upper + self.r1[e] * self.R1_upper - 0.5j * s * self.Gam_upper
        PR_l = (np.conj(np.swapaxes(self.R0_upper, 1, 2)) + self.r1[e] * np.conj(np.swapaxes(self.R1_upper, 1, 2))
                - 0.5j * s * np.conj(np.swapaxes(self.Gam_upper, 1, 2)))
        PL_d = -1j * self.a[e] * s * self.Gam_diag
        PL_u = -1j * self.a[e] * s * self.Gam_upper
        PG_d = -1j * (1.0 + self.a[e]) * s * self.Gam_diag
        PG_u = -1j * (1.0 + self.a[e]) * s * self.Gam_upper
        return PR_d, PR_u, PR_l, PL_d, PL_u, PG_d, PG_u

    def subset(self, idx) -> "WSystem":
        idx = np.asarray(idx)
        return dataclasses.replace(self, r1=self.r1[idx], g1=self.g1[idx], a=self.a[idx],
                                   energies=self.energies[idx])


def _grid_positions(nb: int, ny: int, nz: int, nx: int, spacing: float) -> np.ndarray:
    """Atom positions (Angstrom): block i holds nx slabs of an ny x nz cross-section."""
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cell = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * spacing
    out = []
    for i in range(nb):
        p = cell.copy()
        p[:, 0] += i * nx * spacing
        out.append(p)
    return np.stack(out)  # [nb, bs, 3]


def _banded_from_positions(pos: np.ndarray, r_cut: float, fn):
    """BT blocks of the matrix fn(r_ij) restricted to r_ij <= r_cut (diag + upper)."""
    nb = pos.shape[0]
    diag, upper = [], []
    for i in range(nb):
        d = np.linalg.norm(pos[i][:, None, :] - pos[i][None, :, :], axis=-1)
        diag.append(np.where(d <= r_cut, fn(d), 0.0))
        if i + 1 < nb:
            d = np.linalg.norm(pos[i][:, None, :] - pos[i + 1][None, :, :], axis=-1)
            upper.append(np.where(d <= r_cut, fn(d), 0.0))
    return np.stack(diag), (np.stack(upper) if upper else np.zeros((0,) + diag[0].shape))


def w_system(seed: int = BASE_SEED + 2, nb: int = 16, ny: int = 8, nz: int = 8, nx: int = 16,
             spacing: float = 2.2, r_cut: float = 7.5, n_energies: int = 256,
             target_norm: float = 0.5) -> WSystem:
    """W-type system: nb cells of ny x nz x nx atoms on a `spacing` grid (defaults: 16 cells of
    8x8x16 = 1024 atoms, 2.2 A grid, block length 35.2 A), one orbital per atom.
    V_ij = 1/(1 + r_ij) for r_ij <= r_cut (the r_cut truncation of Sec. 4.1), P banded with the
    same r_cut.  With nx*spacing > 3*r_cut, V, P, V P^R and V P^<> V^H are exactly
    block-tridiagonal."""
    assert nx * spacing > 3.0 * r_cut, "cell too short: V P V^H would not be block-tridiagonal"
    rng = np.random.default_rng(seed)
    pos = _grid_positions(nb, ny, nz, nx, spacing)
    V_d, V_u = _banded_from_positions(pos, r_cut, lambda r: 1.0 / (1.0 + r))
    mask_d, mask_u = _banded_from_positions(pos, r_cut, lambda r: np.ones_like(r))
    bs = V_d.shape[1]

    def rand_sym(scale):
        d = rng.standard_normal(mask_d.shape) * mask_d
        d = (d + np.swapaxes(d, 1, 2)) / 2.0
        u = rng.standard_normal(mask_u.shape) * mask_u
        return d * scale, u * scale

    R0_d, R0_u = rand_sym(1.0)
    R1_d, R1_u = rand_sym(0.3)
    # Gamma: Hermitian, off-diagonal random, diagonal = row sum of |offdiag| + 0.1 -> PSD
    Gd = rng.standard_normal(mask_d.shape) * mask_d
    Gd = (Gd + np.swapaxes(Gd, 1, 2)) / 2.0
    for i in range(nb):
        np.fill_diagonal(Gd[i], 0.0)
    Gu = np.abs(rng.standard_normal(mask_u.shape)) * mask_u * 0.5
    rows = np.abs(Gd).sum(axis=2)
    rows[:-1] += np.abs(Gu).sum(axis=2)
    rows[1:] += np.abs(Gu).sum(axis=1)
    for i in range(nb):
        Gd[i] += np.diag(rows[i] + 0.1)
    # scale P so that ||V P^R||_2 ~ target_norm (estimate with a row-sum bound on each factor)
    def inf_norm(d, u):
        r = np.abs(d).sum(axis=2)
        r[:-1] += np.abs(u).sum(axis=2)
        r[1:] += np.abs(u).sum(axis=1)
        return r.max()
    nV = inf_norm(V_d, V_u)
    nP = inf_norm(R0_d, R0_u) + inf_norm(R1_d, R1_u) + inf_norm(Gd, Gu)
    s = target_norm / (nV * nP)
    c = lambda x: np.ascontiguousarray(x.astype(np.complex128))
    return WSystem(V_diag=c(V_d), V_upper=c(V_u), R0_diag=c(R0_d * s), R0_upper=c(R0_u * s),
                   R1_diag=c(R1_d * s), R1_upper=c(R1_u * s), Gam_diag=c(Gd * s), Gam_upper=c(Gu * s),
                   r1=rng.uniform(-1.0, 1.0, n_energies), g1=rng.uniform(0.0, 0.5, n_energies),
                   a=rng.uniform(0.0, 1.0, n_energies), energies=np.linspace(0.0, 1.0, n_energies))


def w_system_16x1024(seed: int = BASE_SEED + 2) -> WSystem:
    return w_system(seed)


# ----------------------------------------------------------------------------------------------
# Serving stream
# ----------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    nb: int
    bs: int
    n_energies: int
    seed: int


def serving_stream(n_requests: int = 2000, rate_per_s: float = 1.0, seed: int = BASE_SEED + 4,
                   block_sizes=(64, 128, 256, 416, 832), nb_range=(8, 64),
                   energy_counts=(32, 128, 512)):
    """Poisson arrivals; each request is a random device (as the 8x32 workload) of random shape,
    generated from seed + rid."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, n_requests))
    out = []
    for rid in range(n_requests):
        out.append(Request(rid=rid, arrival_s=float(t[rid]), nb=int(rng.integers(nb_range[0], nb_range[1] + 1)),
                           bs=int(rng.choice(block_sizes)), n_energies=int(rng.choice(energy_counts)),
                           seed=seed + rid))
    return out
