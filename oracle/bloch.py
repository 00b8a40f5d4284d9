"""Frozen two-level molecules: Bloch equations integrated by classical RK4.

Test infrastructure: imported only by tests/, __graft_entry__.smoke() and
bench.py's CPU legs; the library never calls it.

Scaling-experiments section (Fig. 5d): with their ro-vibrational degrees of
freedom frozen, the molecules become two-level emitters with no internal
structure, whose equations of motion are the Bloch equations, integrated
with the fourth-order Runge-Kutta scheme.

Readings (the paper gives no equations for this model):
  * Hamiltonian (atomic units) H = w0 |e><e| - d E_par (|g><e| + |e><g|):
    transition energy w0, transition dipole d along the molecular axis n
    (the molecule frame's z axis in the lab, fixed: rotation is frozen too),
    E_par = n . E the local lab field projected on it.
  * Bloch vector u = 2 Re rho_eg, v = 2 Im rho_eg, w = rho_ee - rho_gg;
    from d rho/dt = -i [H, rho] with Omega = 2 d E_par:
        du/dt =  w0 v                - g2 u
        dv/dt = -w0 u - Omega w      - g2 v
        dw/dt =  Omega v             - g1 (w + 1)
    with optional population relaxation g1 = 1/T1 and dephasing g2 = 1/T2
    (0 = none).  Start in the ground state (0, 0, -1).
  * The field is held at E^n over the step t_n -> t_n + dtau (the coupled
    step's order: the molecules advance under E^n), one RK4 step per
    molecular step.
  * Dipole <d sigma_x> = d u along n; populations P_g = (1 - w)/2,
    P_e = (1 + w)/2; no absorbed norm; Eq. 8's <R>_e with the bond frozen at
    r_e is r_e (numerator r_e P_e, denominator P_e).
"""
from __future__ import annotations

import numpy as np

from .constants import F_AU, HARTREE_EV, T_AU
from .molecule import rotation_matrix


def bloch_rhs(y, w0, omega, g1, g2):
    """Right-hand side of the Bloch equations for Bloch vectors y [n, 3]."""
    u, v, w = y[:, 0], y[:, 1], y[:, 2]
    return np.stack([w0 * v - g2 * u,
                     -w0 * u - omega * w - g2 * v,
                     omega * v - g1 * (w + 1.0)], axis=1)


def rk4_step(y, h, w0, omega, g1, g2):
    """One classical fourth-order Runge-Kutta step of size h (field held)."""
    k1 = bloch_rhs(y, w0, omega, g1, g2)
    k2 = bloch_rhs(y + 0.5 * h * k1, w0, omega, g1, g2)
    k3 = bloch_rhs(y + 0.5 * h * k2, w0, omega, g1, g2)
    k4 = bloch_rhs(y + h * k3, w0, omega, g1, g2)
    return y + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)


class BlochEnsemble:
    """n frozen two-level molecules of one species, stepped together."""

    def __init__(self, sp, quat, dtau):
        self.sp = sp
        self.n = quat.shape[0]
        self.dtau = dtau
        self.w0 = sp.w0_ev / HARTREE_EV
        self.g1 = T_AU / sp.T1 if sp.T1 > 0 else 0.0
        self.g2 = T_AU / sp.T2 if sp.T2 > 0 else 0.0
        self.d = sp.dipole
        self.axis = rotation_matrix(quat)[:, :, 2]      # molecule z axis in the lab
        self.y = np.zeros((self.n, 3))
        self.y[:, 2] = -1.0
        self.absorbed = np.zeros((self.n, 2))
        self.mu_lab = np.zeros((self.n, 3))

    def step(self, E_lab_si):
        """Advance by dtau under the lab field E (V/m, [n, 3]); returns the lab
        dipoles (a.u.)."""
        e_par = np.einsum("ni,ni->n", self.axis, np.asarray(E_lab_si, np.float64)) / F_AU
        omega = 2.0 * self.d * e_par
        self.y = rk4_step(self.y, self.dtau, self.w0, omega, self.g1, self.g2)
        self.mu_lab = (self.d * self.y[:, 0])[:, None] * self.axis
        return self.mu_lab

    def populations(self):
        w = self.y[:, 2]
        return np.stack([0.5 * (1.0 - w), 0.5 * (1.0 + w)], axis=1)

    def excited_R(self):
        pe = 0.5 * (1.0 + self.y[:, 2])
        return self.sp.re * pe, pe
