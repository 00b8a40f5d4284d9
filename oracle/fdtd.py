"""FP64 Yee FDTD with Drude metal, CPML in z, periodic x/y and a TF/SF source.

Test infrastructure only (see the package header): the library never calls it.

Follows the paper's field model: Maxwell's curl equations (Eq. 1) marched by
the leap-frog Yee scheme with central differences (section "The domain
decomposition methodology for FDTD"), a Drude current in metal cells
(Eq. 2), periodic boundaries along X and Y and convolutional PML along Z,
and plane-wave excitation from the molecule side.

Grid (x fastest, arrays [nsim, nz, ny, nx]); cell (i,j,k) owns
  Ex(i+1/2, j, k)   Ey(i, j+1/2, k)   Ez(i, j, k+1/2)
  Hx(i, j+1/2, k+1/2)  Hy(i+1/2, j, k+1/2)  Hz(i+1/2, j+1/2, k)
E is stored at integer time steps n, H at n+1/2.  In "pml" mode the box is
closed by perfect conductors at z=0 (Ex=Ey=0 on plane k=0, never updated)
and at z=nz*dx (the implicit plane k=nz); in "periodic" mode z wraps too.

Readings where the paper is silent (the paper cites CPML [73] and the
Drude model [74] without stating the discretisation):
* Drude ADE, central difference at time n:
    J^{n+1/2} = alpha J^{n-1/2} + beta E^n,
    alpha = (1 - g dt/2)/(1 + g dt/2),  beta = eps0 wp^2 dt/(1 + g dt/2);
  then E^{n+1} = E^n + dt/(eps0 eps_inf) (curl H^{n+1/2} - J^{n+1/2})
                 - (P^{n+1} - P^n)/(eps0 eps_inf).
* CPML (Roden-Gedney), kappa = 1, grading order m = 3,
  sigma(rho) = sigma_max (rho/L)^3, sigma_max = 0.8 (m+1)/(eta0 dx),
  alpha(rho) = alpha_max (1 - rho/L), alpha_max = 0.05 S/m, rho the depth
  into the layer measured from its inner face, L = pml*dx;
  b = exp(-(sigma + alpha) dt/eps0),  a = sigma/(sigma + alpha) (b - 1);
  psi^{new} = b psi + a dF/dz, and dF/dz -> dF/dz + psi in the curl.
* TF/SF: total field for k >= src_k.  The incident field comes from a 1D
  vacuum Yee line with the same dz and dt, whose node m sits at
  z = (src_k - 2 + m) dz (H node m at +dz/2).  Its node 0 is hard-driven by
  f(t) = E0 exp(-4 ln2 ((t-t0)/fwhm)^2) cos(w (t-t0)), its far end is a
  perfect conductor placed beyond any return within the run.
"""
from __future__ import annotations

import numpy as np

from .constants import C0, EPS0, HBAR_EVS, MU0

AUX_OFFSET = 2          # aux node index that coincides with the TF/SF plane
CPML_ORDER = 3
CPML_ALPHA_MAX = 0.05   # S/m


def pulse(t, E0, carrier_ev, fwhm, t0):
    """Incident waveform: Gaussian field envelope (FWHM of the field) times a
    cosine carrier, peak E0 at t0 (plane-wave short-pulse excitation)."""
    w = carrier_ev / HBAR_EVS
    return E0 * np.exp(-4.0 * np.log(2.0) * ((t - t0) / fwhm) ** 2) * np.cos(w * (t - t0))


def cw(t, E0, carrier_ev, t_on, t0):
    """Continuous-wave drive switched on smoothly over t_on (Sec. 3 ramps its
    CW runs up over the first few fs; the sin^2 envelope is our reading):
    E0 sin^2(pi t / (2 t_on)) cos(w (t - t0)) for t < t_on, then
    E0 cos(w (t - t0))."""
    w = carrier_ev / HBAR_EVS
    ramp = np.where(t < t_on, np.sin(0.5 * np.pi * np.clip(t, 0.0, None) / t_on) ** 2, 1.0)
    return E0 * ramp * np.cos(w * (t - t0))


def drude_coefficients(wp_ev, gamma_ev, dt):
    """alpha, beta of the central-difference discretisation of Eq. 2."""
    wp = wp_ev / HBAR_EVS
    g = gamma_ev / HBAR_EVS
    den = 1.0 + 0.5 * g * dt
    return (1.0 - 0.5 * g * dt) / den, EPS0 * wp * wp * dt / den


def cpml_profile(z, nz, pml, dx, dt):
    """CPML b, a at height z (metres; array) for a box [0, nz*dx] with `pml`
    cells of absorber at each end.  Outside the layers b=1, a=0."""
    L = pml * dx
    eta0 = np.sqrt(MU0 / EPS0)
    smax = 0.8 * (CPML_ORDER + 1) / (eta0 * dx)
    rho = np.maximum(L - z, 0.0) + np.maximum(z - (nz * dx - L), 0.0)
    inside = rho > 0
    sig = np.where(inside, smax * (rho / L) ** CPML_ORDER, 0.0)
    alp = np.where(inside, CPML_ALPHA_MAX * (1.0 - rho / L), 0.0)
    b = np.where(inside, np.exp(-(sig + alp) * dt / EPS0), 1.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        a = np.where(sig > 0, sig / (sig + alp) * (b - 1.0), 0.0)
    return b, a


class YeeOracle:
    """FP64 field state and the two half-step updates (Eq. 1, Eq. 2)."""

    def __init__(self, nx, ny, nz, nsim, dx, dt, mat_id, materials, *, pml=10,
                 bc_z="pml", src_k=-1, src=None, aux_len=None, src_kind="pulse"):
        self.nx, self.ny, self.nz, self.S = nx, ny, nz, nsim
        self.dx, self.dt = dx, dt
        self.bc_z = bc_z
        self.pml = pml if bc_z == "pml" else 0
        shp = (nsim, nz, ny, nx)
        self.Ex, self.Ey, self.Ez = (np.zeros(shp) for _ in range(3))
        self.Hx, self.Hy, self.Hz = (np.zeros(shp) for _ in range(3))
        self.Jx, self.Jy, self.Jz = (np.zeros(shp) for _ in range(3))
        mat = np.asarray(mat_id).reshape(shp)
        eps = np.array([m[0] for m in materials], np.float64)
        al = np.ones(len(materials))
        be = np.zeros(len(materials))
        for i, (_, wp, g) in enumerate(materials):
            if wp > 0:
                al[i], be[i] = drude_coefficients(wp, g, dt)
        self.metal = np.array([m[1] > 0 for m in materials])[mat]
        self.eps_r = eps[mat]
        self.alpha = al[mat]
        self.beta = be[mat]
        self.ce = dt / (EPS0 * self.eps_r)          # E update scale
        self.ch = dt / MU0                           # H update scale
        # CPML coefficient columns (E nodes at z = k dx, H-type nodes at (k+1/2) dx)
        if self.pml > 0:
            zk = np.arange(nz) * dx
            zh = (np.arange(nz) + 0.5) * dx
            self.bE, self.aE = (v[None, :, None, None] for v in cpml_profile(zk, nz, self.pml, dx, dt))
            self.bH, self.aH = (v[None, :, None, None] for v in cpml_profile(zh, nz, self.pml, dx, dt))
            self.psi_Exz, self.psi_Eyz, self.psi_Hxz, self.psi_Hyz = (np.zeros(shp) for _ in range(4))
        # TF/SF source and its 1D incident-field line
        self.src_k = src_k
        self.src_fn = cw if src_kind == "cw" else pulse
        if src_k >= 0:
            self.src = np.asarray(src, np.float64).reshape(nsim, 4)
            L = aux_len if aux_len is not None else 4096
            self.aux_E = np.zeros((nsim, L + 1))
            self.aux_H = np.zeros((nsim, L))
            self.aux_E[:, 0] = self._drive(0)
        self.n = 0

    # -- helpers --------------------------------------------------------------
    def _drive(self, n):
        t = n * self.dt
        return np.array([float(self.src_fn(t, *self.src[s])) for s in range(self.S)])

    def _zplus(self, F):
        """F[k+1] along z (perfect conductor beyond the top, or wrap)."""
        if self.bc_z == "periodic":
            return np.roll(F, -1, axis=1)
        out = np.zeros_like(F)
        out[:, :-1] = F[:, 1:]
        return out

    def _zminus(self, F):
        """F[k-1] along z (zero below the bottom, or wrap)."""
        if self.bc_z == "periodic":
            return np.roll(F, 1, axis=1)
        out = np.zeros_like(F)
        out[:, 1:] = F[:, :-1]
        return out

    # -- H^{n-1/2} -> H^{n+1/2} -----------------------------------------------
    def step_h(self):
        d = self.dx
        Ex, Ey, Ez = self.Ex, self.Ey, self.Ez
        dEz_dy = (np.roll(Ez, -1, axis=2) - Ez) / d
        dEy_dz = (self._zplus(Ey) - Ey) / d
        dEx_dz = (self._zplus(Ex) - Ex) / d
        dEz_dx = (np.roll(Ez, -1, axis=3) - Ez) / d
        dEy_dx = (np.roll(Ey, -1, axis=3) - Ey) / d
        dEx_dy = (np.roll(Ex, -1, axis=2) - Ex) / d
        if self.pml > 0:
            self.psi_Hxz = self.bH * self.psi_Hxz + self.aH * dEy_dz
            self.psi_Hyz = self.bH * self.psi_Hyz + self.aH * dEx_dz
            dEy_dz = dEy_dz + self.psi_Hxz
            dEx_dz = dEx_dz + self.psi_Hyz
        self.Hx -= self.ch * (dEz_dy - dEy_dz)
        self.Hy -= self.ch * (dEx_dz - dEz_dx)
        self.Hz -= self.ch * (dEy_dx - dEx_dy)
        if self.src_k >= 0:
            ks = self.src_k
            # the H_y plane just below the TF/SF plane sees the scattered Ex
            einc = self.aux_E[:, AUX_OFFSET]
            self.Hy[:, ks - 1] += (self.ch / d) * einc[:, None, None]
            # incident line: H^{n+1/2}
            self.aux_H -= (self.dt / (MU0 * d)) * (self.aux_E[:, 1:] - self.aux_E[:, :-1])

    # -- E^n -> E^{n+1} -------------------------------------------------------
    def step_e(self, dP=None):
        """dP: optional (dPx, dPy, dPz), each [nsim, nz, ny, nx], the change of
        the macroscopic polarization P^{n+1} - P^n in C/m^2 (Eq. 1's current
        J = dP/dt integrated over the step)."""
        d = self.dx
        Hx, Hy, Hz = self.Hx, self.Hy, self.Hz
        dHz_dy = (Hz - np.roll(Hz, 1, axis=2)) / d
        dHy_dz = (Hy - self._zminus(Hy)) / d
        dHx_dz = (Hx - self._zminus(Hx)) / d
        dHz_dx = (Hz - np.roll(Hz, 1, axis=3)) / d
        dHy_dx = (Hy - np.roll(Hy, 1, axis=3)) / d
        dHx_dy = (Hx - np.roll(Hx, 1, axis=2)) / d
        if self.pml > 0:
            self.psi_Exz = self.bE * self.psi_Exz + self.aE * dHy_dz
            self.psi_Eyz = self.bE * self.psi_Eyz + self.aE * dHx_dz
            dHy_dz = dHy_dz + self.psi_Exz
            dHx_dz = dHx_dz + self.psi_Eyz
        cx = dHz_dy - dHy_dz
        cy = dHx_dz - dHz_dx
        cz = dHy_dx - dHx_dy
        if self.src_k >= 0:
            ks = self.src_k
            # the E_x plane at the TF/SF plane sees the total H_y below it
            cx[:, ks] += self.aux_H[:, AUX_OFFSET - 1][:, None, None] / d
        # Drude current at n+1/2 from E^n (Eq. 2), only in metal cells
        m = self.metal
        self.Jx = np.where(m, self.alpha * self.Jx + self.beta * self.Ex, 0.0)
        self.Jy = np.where(m, self.alpha * self.Jy + self.beta * self.Ey, 0.0)
        self.Jz = np.where(m, self.alpha * self.Jz + self.beta * self.Ez, 0.0)
        self.Ex += self.ce * (cx - self.Jx)
        self.Ey += self.ce * (cy - self.Jy)
        self.Ez += self.ce * (cz - self.Jz)
        if dP is not None:
            inv = 1.0 / (EPS0 * self.eps_r)
            self.Ex -= dP[0] * inv
            self.Ey -= dP[1] * inv
            self.Ez -= dP[2] * inv
        if self.bc_z == "pml":
            self.Ex[:, 0] = 0.0
            self.Ey[:, 0] = 0.0
        if self.src_k >= 0:
            self.aux_E[:, 1:-1] -= (self.dt / (EPS0 * d)) * (self.aux_H[:, 1:] - self.aux_H[:, :-1])
            self.aux_E[:, 0] = self._drive(self.n + 1)
        self.n += 1

    def step(self, dP=None):
        self.step_h()
        self.step_e(dP)

    def gather(self, sim, ci, cj, ck):
        """E^n owned by cells (sim, ck, cj, ci): [n, 3] in V/m."""
        return np.stack([self.Ex[sim, ck, cj, ci], self.Ey[sim, ck, cj, ci],
                         self.Ez[sim, ck, cj, ci]], axis=1)
