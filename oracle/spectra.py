"""Spectral detection: running Fourier transforms of the tangential fields on
z-planes and the Poynting flux spectrum through them (the transmission and
reflection spectra of Figs. 2, 4 and 6a).  FP64, test infrastructure only.

Definitions (the Yee stagger fixes the sampling):
  F^(omega) = dt sum_n F(t_n) e^{i omega t_n}, per cell of plane k, with
  - Ex, Ey of plane k after step n (time t_{n+1} = (n+1) dt);
  - Hx, Hy averaged over the planes z = (k - 1/2) dx and (k + 1/2) dx
    (array indices k - 1 and k) after the same step (time t_{n+1/2});
  so Ex pairs with Hy at (i+1/2, j) and Ey with Hx at (i, j+1/2).
  flux(omega) = Re sum_cells (Ex^ conj(Hy^) - Ey^ conj(Hx^)) dx^2   [J s],
  whose integral (1/pi) int_0^inf flux d omega is the energy through the plane.
"""
from __future__ import annotations

import numpy as np


class FluxDFT:
    def __init__(self, yee, planes, omega):
        self.f = yee
        self.k = [int(k) for k in planes]
        self.w = np.asarray(omega, np.float64)
        self.acc = np.zeros((yee.S, len(self.k), self.w.size, 4, yee.ny, yee.nx), np.complex128)

    def accumulate(self):
        """Add the current fields; call right after the E half step."""
        f = self.f
        pE = np.exp(1j * self.w * f.n * f.dt) * f.dt            # t_{n+1}: f.n counts the steps taken
        pH = np.exp(1j * self.w * (f.n - 0.5) * f.dt) * f.dt    # t_{n+1/2}
        for d, k in enumerate(self.k):
            comps = (f.Ex[:, k], f.Ey[:, k], 0.5 * (f.Hx[:, k - 1] + f.Hx[:, k]),
                     0.5 * (f.Hy[:, k - 1] + f.Hy[:, k]))
            for c, v in enumerate(comps):
                ph = pE if c < 2 else pH
                self.acc[:, d, :, c] += ph[None, :, None, None] * v[:, None]

    def flux(self, d):
        """[nsim][nfreq] Poynting flux spectrum through plane d (+z)."""
        a = self.acc[:, d]
        s = a[:, :, 0] * np.conj(a[:, :, 3]) - a[:, :, 1] * np.conj(a[:, :, 2])
        return np.real(s.sum(axis=(-2, -1))) * self.f.dx ** 2


def pulse_spectrum(omega, E0, carrier_ev, fwhm, t0):
    """|int E(t) e^{i omega t} dt|^2 of E(t) = E0 exp(-4 ln2 ((t - t0)/fwhm)^2)
    cos(w0 (t - t0)), w0 = carrier / hbar: the closed form of the Gaussian's
    transform, both sidebands."""
    from .constants import HBAR_EVS
    a = 4.0 * np.log(2.0) / fwhm ** 2
    w0 = carrier_ev / HBAR_EVS
    omega = np.asarray(omega, np.float64)
    amp = 0.5 * E0 * np.sqrt(np.pi / a) * (np.exp(-(omega - w0) ** 2 / (4 * a)) + np.exp(-(omega + w0) ** 2 / (4 * a)))
    return amp ** 2
