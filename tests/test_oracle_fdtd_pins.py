"""Pins of the FP64 field oracle against what physics and the mathematics fix.

* discrete plane-wave eigenmode of the Yee scheme (numerical dispersion
  relation sin^2(w dt/2)/(c dt)^2 = sum_i sin^2(k_i dx/2)/dx^2);
* TF/SF: the scattered-field region stays empty and the total-field region
  equals the incident line in vacuum;
* CPML: the wave that enters the z absorber does not come back;
* Drude slab: reflectivity against the closed-form thin-film formula with
  eps(w) = eps_inf - wp^2/(w^2 + i g w) (Eq. 2's susceptibility);
* polarization current: a thin sheet of oscillating polarization radiates
  E = -(eta0/2) dz dP/dt to either side (Eq. 1 with J = dP/dt).
"""
import numpy as np
import pytest

from oracle.constants import C0, EPS0, HBAR_EVS, MU0
from oracle.fdtd import AUX_OFFSET, YeeOracle, pulse
import workloads as W

DX = 2e-9
DT = DX / (2 * C0)


def _yee_positions(nx, ny, nz, comp):
    """Staggered positions (in units of dx) of one field component."""
    off = {"Ex": (0.5, 0, 0), "Ey": (0, 0.5, 0), "Ez": (0, 0, 0.5),
           "Hx": (0, 0.5, 0.5), "Hy": (0.5, 0, 0.5), "Hz": (0.5, 0.5, 0)}[comp]
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i + off[0], j + off[1], k + off[2]


def test_yee_vacuum_dispersion_eigenmode():
    nx, ny, nz = 6, 5, 7
    p = np.array([1, 2, 3])
    kvec = 2 * np.pi * p / (np.array([nx, ny, nz]) * DX)
    Kt = 2 / DX * np.sin(kvec * DX / 2)
    # the scheme's wave speed is 1/sqrt(mu0 eps0) (CODATA: c to 2e-14)
    Om = np.linalg.norm(Kt) / np.sqrt(MU0 * EPS0)
    w = 2 / DT * np.arcsin(DT * Om / 2)
    E0 = np.cross(Kt, [1.0, 0.3, 0.2])
    E0 *= 1e9 / np.linalg.norm(E0)
    H0 = np.cross(Kt, E0) / (MU0 * Om)
    mat = np.zeros((1, nz, ny, nx), np.uint8)
    f = YeeOracle(nx, ny, nz, 1, DX, DT, mat, W.configs.MATERIALS, bc_z="periodic")

    def field(comp, t):
        x, y, z = _yee_positions(nx, ny, nz, comp)
        ph = kvec[0] * x * DX + kvec[1] * y * DX + kvec[2] * z * DX - w * t
        amp = {"Ex": E0[0], "Ey": E0[1], "Ez": E0[2], "Hx": H0[0], "Hy": H0[1], "Hz": H0[2]}[comp]
        return (amp * np.cos(ph))[None]

    for c in ("Ex", "Ey", "Ez"):
        setattr(f, c, field(c, 0.0))
    for c in ("Hx", "Hy", "Hz"):
        setattr(f, c, field(c, -0.5 * DT))
    nsteps = 2000
    for _ in range(nsteps):
        f.step()
    num = sum(np.sum((getattr(f, c) - field(c, nsteps * DT)) ** 2) for c in ("Ex", "Ey", "Ez"))
    den = sum(np.sum(field(c, nsteps * DT) ** 2) for c in ("Ex", "Ey", "Ez"))
    assert np.sqrt(num / den) < 1e-12
    # a wrong dispersion (continuum w = c|k|) would be far off after 2000 steps
    assert abs(w - C0 * np.linalg.norm(kvec)) * nsteps * DT > 1e-2


def _column(nz, src_k, mat=None, pulse_row=(1e9, 1.5498, 10e-15, 12e-15), nx=1, ny=1, pml=10):
    m = np.zeros((1, nz, ny, nx), np.uint8) if mat is None else mat
    return YeeOracle(nx, ny, nz, 1, DX, DT, m, W.configs.MATERIALS, pml=pml, bc_z="pml",
                     src_k=src_k, src=np.array([pulse_row]), aux_len=8192)


def test_tfsf_scattered_region_stays_empty_and_total_region_is_incident():
    # the numerical light cone (one cell per step) stays clear of the top PML
    nz, ks = 700, 30
    f = _column(nz, ks, nx=2, ny=3, pulse_row=(1e9, 1.5498, 1e-15, 1e-15))
    peak = 0.0
    for n in range(600):
        f.step()
        peak = max(peak, np.abs(f.Ex).max())
        # scattered-field region: E planes k < ks, H planes k < ks - 1
        sf = max(np.abs(f.Ex[:, :ks]).max(), np.abs(f.Ey[:, :ks]).max(),
                 np.abs(f.Ez[:, :ks]).max(), np.abs(f.Hy[:, :ks - 1]).max() * 376.73)
        assert sf <= 1e-13 * 1e9
    assert peak > 0.5e9           # the pulse is in the box
    # total-field region equals the incident line at the same heights
    m = np.arange(0, nz - 10 - ks)
    inc = f.aux_E[0, AUX_OFFSET + m]
    tot = f.Ex[0, ks + m, 0, 0]
    assert np.max(np.abs(tot - inc)) <= 1e-13 * 1e9
    assert np.abs(f.Ey).max() == 0 and np.abs(f.Ez).max() == 0


def test_cpml_reflection_is_small():
    nz, ks = 260, 30
    f = _column(nz, ks, pulse_row=(1e9, 1.5498, 2e-15, 3e-15))
    refl = 0.0
    inc_peak = 0.0
    for n in range(3000):
        f.step()
        inc_peak = max(inc_peak, abs(f.aux_E[0, AUX_OFFSET]))
        refl = max(refl, np.abs(f.Ex[0, 12:ks - 2]).max())
    assert inc_peak > 0.9e9
    # 10 cells, cubic grading: the return is ~3e-5 of the incident peak; a
    # perfect conductor without the layer would send back all of it
    assert refl < 1e-4 * inc_peak


def _film_reflectance(eps, d, omega):
    """Normal-incidence reflectance of a film of permittivity eps(w) and
    thickness d in vacuum (Airy summation of the two interfaces)."""
    n = np.sqrt(eps)
    r12 = (1 - n) / (1 + n)
    r23 = (n - 1) / (n + 1)
    beta = omega / C0 * n * d
    ph = np.exp(2j * beta)
    return np.abs((r12 + r23 * ph) / (1 + r12 * r23 * ph)) ** 2


@pytest.mark.slow
def test_drude_slab_reflectivity_matches_thin_film_formula():
    nz, ks, k0, thick = 520, 30, 200, 10
    mat = np.zeros((1, nz, 1, 1), np.uint8)
    mat[0, k0:k0 + thick] = W.configs.MAT_SILVER
    f = _column(nz, ks, mat=mat, pulse_row=(1e9, 2.1, 1e-15, 3e-15))
    nsteps = 12000
    kp = ks - 8
    inc = np.zeros(nsteps)
    ref = np.zeros(nsteps)
    for n in range(nsteps):
        f.step()
        inc[n] = f.aux_E[0, AUX_OFFSET]
        ref[n] = f.Ex[0, kp, 0, 0]
    ev = np.linspace(1.2, 3.0, 19)
    w = ev / HBAR_EVS
    t = np.arange(1, nsteps + 1) * DT
    Fi = np.exp(1j * np.outer(w, t)) @ inc
    Fr = np.exp(1j * np.outer(w, t)) @ ref
    R_fdtd = np.abs(Fr / Fi) ** 2
    eps_inf, wp, g = W.configs.MATERIALS[W.configs.MAT_SILVER]
    wp_, g_ = wp / HBAR_EVS, g / HBAR_EVS
    eps = eps_inf - wp_ ** 2 / (w ** 2 + 1j * g_ * w)
    R_exact = _film_reflectance(eps, thick * DX, w)
    # 2 nm cells: the grid gives 4.5e-4; gamma x10 would be off by 8e-2,
    # eps_inf = 1 by 0.19
    assert np.max(np.abs(R_fdtd - R_exact)) < 2e-3
    # the slab reflects strongly below the screened plasma edge
    assert R_exact[0] > 0.5 and R_fdtd[0] > 0.5


def test_polarization_sheet_radiates_minus_half_eta0_dz_dPdt():
    """A sheet of polarization P(t) in one E_x plane is a surface current
    K = dz dP/dt; Ampere's law (Eq. 1) makes it radiate E_x = -eta0 K/2 to
    both sides.  Checked with a slow Gaussian P so the grid error is small."""
    nz, k0, kp = 400, 200, 260
    f = YeeOracle(1, 1, nz, 1, DX, DT, np.zeros((1, nz, 1, 1), np.uint8),
                  W.configs.MATERIALS, pml=10, bc_z="pml")
    tau = 400 * DT
    Pamp = 1e-3
    P = lambda n: Pamp * np.exp(-(((n - 1200) * DT) / tau) ** 2)
    rec = []
    for n in range(2400):
        dP = np.zeros((3, 1, nz, 1, 1))
        dP[0, 0, k0] = P(n + 1) - P(n)
        f.step(dP)
        rec.append(f.Ex[0, kp, 0, 0])
    rec = np.array(rec)
    eta0 = np.sqrt(MU0 / EPS0)
    delay = (kp - k0) * DX / C0
    n = np.arange(2400)
    t = (n + 1) * DT - delay
    dPdt = Pamp * np.exp(-(((t / DT) - 1200) * DT / tau) ** 2) * (-2 * ((t / DT) - 1200) * DT / tau ** 2)
    expect = -0.5 * eta0 * DX * dPdt
    sel = slice(800, 2000)
    assert np.max(np.abs(rec[sel] - expect[sel])) < 2e-2 * np.max(np.abs(expect))
