"""FP64 ro-vibrational wavepackets on two coupled surfaces (Eqs. 3-8).

Test infrastructure only (see the package header): the library never calls it.

Each molecule carries xi^{(s)}_{jm}(R), s in {g, e}, j <= Jmax, |m| <= j,
on a uniform radial grid (Eq. 3: expansion of chi_{g,e} in rotational
functions).  One step of length dtau advances Eq. 4 with the effective
Hamiltonians of Eq. 5 by the split-operator method (the paper's FFT
split-operator propagator), literally:

    psi <- T(1/2) Mask V(1/2) K(E') V(1/2) T(1/2) psi

* T(tau)  = exp(-i tau p^2/2mu) on the periodic radial box, written as the
            dense circulant matrix
            K_prop[a,b] = (1/Nr) sum_p exp(i k_p (r_a-r_b)) exp(-i k_p^2 tau/2mu),
            k_p = 2 pi p/(Nr dR), p in [-Nr/2, Nr/2).
* V(tau)  = exp(-i tau (U_s(R) + j(j+1)/(2 mu R^2))) per surface and j
            (Eq. 5; U_g Eq. 6, U_e of the form A + B exp(-beta (R - rc)),
            which is Eq. 7 for A=0, B=2 D_e).
* K(E')   = exp(+i d dtau sigma_x (x) (E'_x X + E'_y Y + E'_z Z)), the
            transition-dipole coupling of Eq. 4 with the field E' in the
            molecule frame.  Reading of the "*" on the second line of Eq. 4:
            the coupling operator must be Hermitian, H_eg = H_ge^dagger, and
            E.R^hat is Hermitian in the Y_jm basis, so both lines carry the
            same matrix.  Evaluated by its Taylor series.
* Mask    = cos(pi/2 (R - ra)/(Rmax - ra))**power for R > ra, else 1.

Observables after the step: populations P_s = sum |xi_s|^2 dR, the norm
removed by the mask in this step, the induced dipole
mu' = d <psi| sigma_x (x) R^hat |psi> (mean-field source of Eq. 1's
polarization current) rotated to the lab frame, and Eq. 8's numerator
<chi_e|R|chi_e> and denominator <chi_e|chi_e>.
"""
from __future__ import annotations

import numpy as np

from .constants import F_AU, T_AU


# -----------------------------------------------------------------------------
# rotational basis and angular matrices (Eq. 3/4)
# -----------------------------------------------------------------------------

def channels(jmax):
    """Channel list (j, m) in the order ch = j^2 + j + m."""
    return [(j, m) for j in range(jmax + 1) for m in range(-j, j + 1)]


def angular_matrices(jmax):
    """X, Y, Z: matrices of sin(t)cos(p), sin(t)sin(p), cos(t) between complex
    spherical harmonics Y_jm (Condon-Shortley) -- the lab-to-molecule field
    projections of Eq. 4.  Built from the textbook recursions
      cos(t) Y_jm  couples (j+-1, m)   with sqrt(((j+1)^2-m^2)/((2j+1)(2j+3)))
      sin(t)e^{ip} Y_jm -> -sqrt((j+m+1)(j+m+2)/((2j+1)(2j+3))) Y_{j+1,m+1}
                           +sqrt((j-m)(j-m-1)/((2j-1)(2j+1)))  Y_{j-1,m+1}
    and X = (S+ + S-)/2, Y = (S+ - S-)/(2i), S- = S+^dagger."""
    ch = channels(jmax)
    idx = {c: i for i, c in enumerate(ch)}
    n = len(ch)
    Z = np.zeros((n, n), np.complex128)
    Sp = np.zeros((n, n), np.complex128)
    for (j, m), col in idx.items():
        if (j + 1, m) in idx:
            v = np.sqrt(((j + 1) ** 2 - m ** 2) / ((2 * j + 1) * (2 * j + 3)))
            Z[idx[(j + 1, m)], col] = v
            Z[col, idx[(j + 1, m)]] = v
        if (j + 1, m + 1) in idx:
            Sp[idx[(j + 1, m + 1)], col] = -np.sqrt((j + m + 1) * (j + m + 2) /
                                                    ((2 * j + 1) * (2 * j + 3)))
        if j >= 1 and (j - 1, m + 1) in idx:
            Sp[idx[(j - 1, m + 1)], col] = np.sqrt((j - m) * (j - m - 1) /
                                                   ((2 * j - 1) * (2 * j + 1)))
    Sm = Sp.conj().T
    X = 0.5 * (Sp + Sm)
    Y = (Sp - Sm) / 2j
    return X, Y, Z


def rotation_matrix(q):
    """Rotation matrices [n,3,3] (molecule frame -> lab) from quaternions
    (w, x, y, z), normalised here."""
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((q.shape[0], 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - w * z)
    R[:, 0, 2] = 2 * (x * z + w * y)
    R[:, 1, 0] = 2 * (x * y + w * z)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - w * x)
    R[:, 2, 0] = 2 * (x * z - w * y)
    R[:, 2, 1] = 2 * (y * z + w * x)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


# -----------------------------------------------------------------------------
# radial grid, potentials, kinetic propagator, ground state (Eqs. 5-7)
# -----------------------------------------------------------------------------

def radial_grid(sp):
    if sp.nr == 1:
        return np.array([sp.rmin]), 1.0
    dR = (sp.rmax - sp.rmin) / (sp.nr - 1)
    return sp.rmin + dR * np.arange(sp.nr), dR


def potentials(sp, r):
    """U_g (Eq. 6) and U_e (Eq. 7 family) in E_h."""
    Ug = sp.De * (1.0 - np.exp(-sp.a * (r - sp.re))) ** 2 - sp.De
    Ue = sp.A + sp.B * np.exp(-sp.beta * (r - sp.rc))
    return Ug, Ue


def wave_numbers(nr, dR):
    p = np.arange(nr) - nr // 2
    return 2.0 * np.pi * p / (nr * dR)


def kinetic_propagator(sp, tau):
    """Dense circulant exp(-i tau p^2/2mu) on the periodic radial box."""
    r, dR = radial_grid(sp)
    k = wave_numbers(sp.nr, dR)
    diff = r[:, None] - r[None, :]
    ph = np.exp(-1j * k ** 2 * tau / (2.0 * sp.mass))
    return (np.exp(1j * k[None, None, :] * diff[:, :, None]) * ph).sum(axis=2) / sp.nr


def kinetic_matrix(sp):
    """Fourier-grid kinetic energy matrix T[a,b] = (1/Nr) sum_p k_p^2/(2mu)
    exp(i k_p (r_a - r_b)) (real symmetric)."""
    r, dR = radial_grid(sp)
    k = wave_numbers(sp.nr, dR)
    diff = r[:, None] - r[None, :]
    T = (np.exp(1j * k[None, None, :] * diff[:, :, None]) * (k ** 2 / (2 * sp.mass))).sum(axis=2)
    return (T / sp.nr).real


def fgh_spectrum(sp):
    """Eigenvalues/vectors of the Fourier-grid Hamiltonian T + diag(U_g)."""
    r, _ = radial_grid(sp)
    Ug, _ = potentials(sp, r)
    H = kinetic_matrix(sp) + np.diag(Ug)
    return np.linalg.eigh(H)


def ground_state(sp):
    """v=0, j=0 ground-surface radial function (initial condition of the
    paper's runs), normalised as sum |xi|^2 dR = 1, sign fixed so that the
    largest-magnitude sample is positive."""
    _, dR = radial_grid(sp)
    w, v = fgh_spectrum(sp)
    g = v[:, 0].copy()
    if g[np.argmax(np.abs(g))] < 0:
        g = -g
    return g / np.sqrt((g * g).sum() * dR)


def mask(sp):
    r, _ = radial_grid(sp)
    m = np.ones_like(r)
    sel = r > sp.absorber_r
    if sp.absorber_r < sp.rmax:
        x = (r[sel] - sp.absorber_r) / (sp.rmax - sp.absorber_r)
        m[sel] = np.clip(np.cos(0.5 * np.pi * x), 0.0, None) ** sp.absorber_power
    return m


# -----------------------------------------------------------------------------
# an ensemble of molecules of one species
# -----------------------------------------------------------------------------

class SpeciesEnsemble:
    """FP64 state psi[n, 2, Nrot, Nr] of the molecules of one species."""

    def __init__(self, sp, quat, dtau, taylor_tol=1e-18):
        self.sp = sp
        self.n = quat.shape[0]
        self.dtau = dtau
        self.r, self.dR = radial_grid(sp)
        self.ch = channels(sp.jmax)
        self.nrot = len(self.ch)
        self.X, self.Y, self.Z = angular_matrices(sp.jmax)
        self.O = rotation_matrix(quat)                         # molecule -> lab
        Ug, Ue = potentials(sp, self.r)
        jj = np.array([j * (j + 1) for j, _ in self.ch], np.float64)
        cent = jj[:, None] / (2.0 * sp.mass * self.r[None, :] ** 2)
        self.V = np.stack([Ug[None, :] + cent, Ue[None, :] + cent])   # [2, nrot, nr]
        self.Vhalf = np.exp(-0.5j * dtau * self.V)
        self.Thalf = kinetic_propagator(sp, 0.5 * dtau)
        self.mask = mask(sp)
        self.taylor_tol = taylor_tol
        # transition dipole at each radial point (e a0): the constant d, or an
        # R-dependent d(R) given at the grid points
        dR_tab = getattr(sp, "dipole_R", None)
        self.d_r = (np.full(sp.nr, float(sp.dipole)) if dR_tab is None
                    else np.asarray(dR_tab, np.float64).reshape(sp.nr))
        self.psi = np.zeros((self.n, 2, self.nrot, sp.nr), np.complex128)
        self.psi[:, 0, 0, :] = ground_state(sp)[None, :]
        self.absorbed = np.zeros((self.n, 2))
        self.mu_lab = np.zeros((self.n, 3))

    # -- pieces of the step ---------------------------------------------------
    def apply_T(self, psi, Kp):
        """out[..., a] = sum_b Kp[a, b] psi[..., b] (per channel, along R)."""
        return psi @ Kp.T

    def coupling(self, psi, E_mol_au):
        """exp(+i dtau d(R) sigma_x (x) M) psi by its Taylor series, with
        M = E'_x X + E'_y Y + E'_z Z per molecule (Eq. 4 coupling terms) and
        the transition dipole d(R) acting point-wise along R (constant d:
        the paper's case)."""
        M = (E_mol_au[:, 0, None, None] * self.X + E_mol_au[:, 1, None, None] * self.Y
             + E_mol_au[:, 2, None, None] * self.Z)
        out = psi.copy()
        term = psi.copy()
        for n in range(1, 200):
            # sigma_x (x) M (x) d(R): swap the surfaces, apply M along the
            # channel index and d(R) along R
            sw = term[:, ::-1] * self.d_r
            term = (1j * self.dtau / n) * (M[:, None] @ sw)
            out += term
            if np.sqrt((np.abs(term) ** 2).sum()) < self.taylor_tol:
                break
        return out

    def dipole_mol(self, psi):
        """mu' = 2 Re sum_R d(R) xi_g^dagger A xi_e dR for A = X, Y, Z (a.u.)."""
        g, e = psi[:, 0], psi[:, 1]
        out = np.empty((psi.shape[0], 3))
        for c, A in enumerate((self.X, self.Y, self.Z)):
            Ae = A @ e                                           # [k, a, r]
            out[:, c] = 2.0 * self.dR * (g.conj() * Ae * self.d_r).sum(axis=(1, 2)).real
        return out

    # -- one split-operator step ------------------------------------------------
    def step(self, E_lab_si):
        """Advance every molecule by dtau under the lab field E_lab_si [n,3]
        (V/m, the field at time n); return the lab dipole at n+1 (a.u.)."""
        E_mol = np.einsum("kji,kj->ki", self.O, E_lab_si) / F_AU      # O^T E
        psi = self.apply_T(self.psi, self.Thalf)
        psi = self.Vhalf[None] * psi
        psi = self.coupling(psi, E_mol)
        psi = self.Vhalf[None] * psi
        w = 1.0 - self.mask ** 2
        self.absorbed += (np.abs(psi) ** 2 * w).sum(axis=(2, 3)) * self.dR
        psi = psi * self.mask
        psi = self.apply_T(psi, self.Thalf)
        self.psi = psi
        self.mu_lab = np.einsum("kij,kj->ki", self.O, self.dipole_mol(psi))
        return self.mu_lab

    # -- observables ------------------------------------------------------------
    def populations(self):
        return (np.abs(self.psi) ** 2).sum(axis=(2, 3)) * self.dR       # [n, 2]

    def excited_R(self):
        """Eq. 8 numerator <chi_e|R|chi_e> and denominator <chi_e|chi_e>."""
        pe = np.abs(self.psi[:, 1]) ** 2
        return (pe * self.r).sum(axis=(1, 2)) * self.dR, pe.sum(axis=(1, 2)) * self.dR


def dtau_au(dt_s, substeps=1):
    """Molecular time step in atomic units (one molecular step every
    `substeps` field steps)."""
    return dt_s * substeps / T_AU
