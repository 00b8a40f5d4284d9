"""Pins of the FP64 molecular oracle (Eqs. 3-8) against closed forms,
library routines and invariants -- never against itself.

* X/Y/Z angular matrices vs brute-force quadrature of spherical harmonics
  (scipy's Y_jm, Gauss-Legendre in cos(theta) x uniform phi), j <= 16;
* Fourier-grid eigenvalues vs the Morse closed form (Eq. 6);
* phase rate of the propagated ground state = its energy, error O(dtau^2);
* dense kinetic circulant vs numpy's FFT;
* Taylor coupling exponential vs scipy.linalg.expm;
* field-free norm conservation; norm + absorbed = 1 with the absorber on;
* two-level (Rabi) limit vs the analytic formula and vs expm products;
* orientation invariance (rotation-closed full j shells);
* Eq. 8 numerator: free motion on a flat excited surface gives
  <R>(t) = <R>(0) + k0 t / mu exactly;
* the merged phi = T^(1/2) psi form used by the GPU equals the literal step.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.special

import workloads as W
from oracle import molecule as M
from oracle.constants import A0, EA0, F_AU, T_AU

DT = 2e-9 / (2 * 299792458.0)
DTAU = DT / T_AU


def _sph(j, m, th, ph):
    return scipy.special.sph_harm_y(j, m, th, ph)


def test_angular_matrices_match_quadrature():
    jmax = 16
    xg, wg = np.polynomial.legendre.leggauss(48)
    nphi = 72
    phi = 2 * np.pi * np.arange(nphi) / nphi
    th = np.arccos(xg)
    TH, PH = np.meshgrid(th, phi, indexing="ij")
    w = (wg[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).ravel()
    TH, PH = TH.ravel(), PH.ravel()
    Ymat = np.stack([_sph(j, m, TH, PH) for j, m in M.channels(jmax)], axis=1)
    X, Y, Z = M.angular_matrices(jmax)
    for f, A in ((np.sin(TH) * np.cos(PH), X), (np.sin(TH) * np.sin(PH), Y), (np.cos(TH), Z)):
        Q = (Ymat.conj() * (w * f)[:, None]).T @ Ymat
        assert np.max(np.abs(Q - A)) < 1e-13
    # Hermitian, and x^2 + y^2 + z^2 = 1 on every fully-coupled block
    for A in (X, Y, Z):
        assert np.allclose(A, A.conj().T, atol=0)


def test_fgh_eigenvalues_match_morse_closed_form():
    sp = W.species_config0()
    w, _ = M.fgh_spectrum(sp)
    we = sp.a * np.sqrt(2 * sp.De / sp.mass)
    v = np.arange(6) + 0.5
    Ev = -sp.De + we * v - (we * v) ** 2 / (4 * sp.De)
    assert np.max(np.abs(w[:6] - Ev)) < 1e-8
    assert abs(w[0] - (-0.0927561)) < 1e-7
    # number of bound states of the Morse well: floor(2 De / we + 1/2) = 14
    assert int(np.floor(2 * sp.De / we + 0.5)) == 14


def _field_free(sp, dtau, nsteps, quat=None):
    q = np.array([[1.0, 0, 0, 0]]) if quat is None else quat
    ens = M.SpeciesEnsemble(sp, q, dtau)
    for _ in range(nsteps):
        ens.step(np.zeros((q.shape[0], 3)))
    return ens


def test_ground_state_phase_rate_is_its_energy_to_second_order():
    sp = W.species_config0()
    E0 = M.fgh_spectrum(sp)[0][0]
    psi0 = M.ground_state(sp)
    _, dR = M.radial_grid(sp)
    errs = []
    for dtau in (4 * DTAU, 2 * DTAU):
        n = int(round(200 * 4 * DTAU / dtau))
        ens = M.SpeciesEnsemble(sp, np.array([[1.0, 0, 0, 0]]), dtau)
        phase = 0.0
        prev = ens.psi[0, 0, 0].copy()
        for _ in range(n):
            ens.step(np.zeros((1, 3)))
            cur = ens.psi[0, 0, 0]
            phase += np.angle((prev.conj() * cur).sum())      # unwrapped
            prev = cur.copy()
        ov = (psi0 * ens.psi[0, 0, 0]).sum() * dR
        rate = -phase / (n * dtau)
        errs.append(abs(rate - E0))
        assert abs(abs(ov) - 1) < 1e-10         # stays the eigenstate
    assert errs[0] < 1e-7
    assert 3.0 < errs[0] / errs[1] < 5.0         # Strang splitting: O(dtau^2)


def test_kinetic_circulant_matches_fft():
    sp = W.Species(nr=64, mass=918.0)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    tau = 3.7
    K = M.kinetic_propagator(sp, tau)
    _, dR = M.radial_grid(sp)
    k = 2 * np.pi * np.fft.fftfreq(64, d=dR)
    ref = np.fft.ifft(np.exp(-1j * k ** 2 * tau / (2 * sp.mass)) * np.fft.fft(x))
    assert np.max(np.abs(K @ x - ref)) < 1e-13
    assert np.allclose(K.conj().T @ K, np.eye(64), atol=1e-13)


def test_taylor_coupling_matches_expm():
    sp = W.Species(nr=4, jmax=3, mass=918.0)
    ens = M.SpeciesEnsemble(sp, np.array([[1.0, 0, 0, 0]]), DTAU)
    rng = np.random.default_rng(1)
    psi = rng.standard_normal((1, 2, 16, 4)) + 1j * rng.standard_normal((1, 2, 16, 4))
    E = np.array([[0.02, -0.015, 0.03]])        # a.u., ~1e10 V/m: many terms
    out = ens.coupling(psi, E)
    Mx = E[0, 0] * ens.X + E[0, 1] * ens.Y + E[0, 2] * ens.Z
    H = -sp.dipole * np.kron(np.array([[0, 1], [1, 0]]), Mx)     # -d sigma_x (x) M
    U = scipy.linalg.expm(-1j * DTAU * H)
    ref = np.einsum("ab,br->ar", U, psi[0].reshape(32, 4)).reshape(2, 16, 4)
    assert np.max(np.abs(out[0] - ref)) < 1e-13


def test_field_free_norm_is_conserved():
    sp = W.Species(nr=64, jmax=2, absorber_r=20.0)
    ens = _field_free(sp, DTAU, 2000)
    P = ens.populations()[0]
    # 4000 applications of a float64 circulant whose unitarity defect is a
    # few ulp: drift ~2e-12 (FP32 arithmetic would give ~1e-7 per step)
    assert abs(P.sum() - 1.0) < 1e-11


def test_norm_plus_absorbed_is_one():
    """Mass 1 (light) so the kinetic kick spreads the packet into the mask."""
    sp = W.Species(nr=64, jmax=1, mass=20.0, De=0.02)
    q = np.array([[1.0, 0, 0, 0], [0.5, 0.5, 0.5, 0.5]])
    ens = M.SpeciesEnsemble(sp, q, DTAU)
    r, dR = M.radial_grid(sp)
    ens.psi[:, 0, 0, :] *= np.exp(3j * r)[None]          # launch outward
    for n in range(600):
        ens.step(np.array([[1e9, 0, 0], [0, 2e9, 1e9]]))
    tot = ens.populations().sum(axis=1) + ens.absorbed.sum(axis=1)
    assert np.max(np.abs(tot - 1.0)) < 1e-12
    assert ens.absorbed.sum(axis=1).min() > 1e-3       # the mask did act


def _two_level_species(delta):
    # one flat radial function: huge mass (T = 1, no centrifugal term), U_g = 0,
    # U_e = delta, absorber off
    return W.Species(nr=4, jmax=1, mass=1e30, De=0.0, a=1.0, A=delta, B=0.0,
                     absorber_r=1e3)


@pytest.mark.parametrize("delta", [0.0, 0.002])
def test_two_level_rabi_limit(delta):
    sp = _two_level_species(delta)
    Ez_si = 5e10
    E = Ez_si / F_AU
    ens = M.SpeciesEnsemble(sp, np.array([[1.0, 0, 0, 0]]), DTAU)
    nsteps = 3000
    Pe = np.zeros(nsteps)
    muz = np.zeros(nsteps)
    for n in range(nsteps):
        mu = ens.step(np.array([[0.0, 0.0, Ez_si]]))
        Pe[n] = ens.populations()[0, 1]
        muz[n] = mu[0, 2]
    t = (np.arange(nsteps) + 1) * DTAU
    Om = 2 * sp.dipole * E / np.sqrt(3)
    W2 = Om ** 2 + delta ** 2
    exact = Om ** 2 / W2 * np.sin(np.sqrt(W2) * t / 2) ** 2
    # the 2x2 Strang product (V/2, K, V/2) by expm
    V = np.diag([0.0, delta])
    K = np.array([[0, -sp.dipole * E / np.sqrt(3)], [-sp.dipole * E / np.sqrt(3), 0]])
    S = scipy.linalg.expm(-0.5j * DTAU * V) @ scipy.linalg.expm(-1j * DTAU * K) @ \
        scipy.linalg.expm(-0.5j * DTAU * V)
    c = np.array([1.0, 0.0], complex)
    Pe_s = np.zeros(nsteps)
    mu_s = np.zeros(nsteps)
    for n in range(nsteps):
        c = S @ c
        Pe_s[n] = abs(c[1]) ** 2
        mu_s[n] = 2 * sp.dipole * (c[0].conj() * c[1]).real / np.sqrt(3)
    assert np.max(np.abs(Pe - Pe_s)) < 1e-12
    assert np.max(np.abs(muz - mu_s)) < 1e-12
    if delta == 0.0:
        assert np.max(np.abs(Pe - exact)) < 1e-12
    else:
        err = np.max(np.abs(Pe - exact))
        assert 1e-12 < err < 1e-4 * np.max(exact)      # O(dtau^2) Strang error
    assert Pe.max() > 0.1 * Om ** 2 / W2


def test_orientation_invariance():
    sp = W.Species(nr=32, jmax=2, mass=918.0)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((4, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    qid = np.tile([1.0, 0, 0, 0], (4, 1))
    a = M.SpeciesEnsemble(sp, q, DTAU)
    b = M.SpeciesEnsemble(sp, qid, DTAU)
    Edir = np.array([0.3, -0.5, 0.8])
    for n in range(300):
        E = np.tile(Edir * 3e10 * np.cos(0.05 * n), (4, 1))
        mua = a.step(E)
        mub = b.step(E)
        assert np.max(np.abs(mua - mub)) < 1e-12 * max(1.0, np.abs(mub).max())
    assert np.max(np.abs(a.populations() - b.populations())) < 1e-12
    assert np.abs(mub).max() > 1e-6


def test_free_motion_excited_R_expectation():
    """Flat excited surface (B = 0, A = 0): free motion, for which the
    split-operator step is exact, so Eq. 8's <R>_e moves at k0/mu."""
    sp = W.Species(nr=128, rmin=1.0, rmax=30.0, jmax=0, mass=918.0, A=0.0, B=0.0,
                   absorber_r=1e3)
    ens = M.SpeciesEnsemble(sp, np.array([[1.0, 0, 0, 0]]), DTAU)
    r, dR = M.radial_grid(sp)
    k0 = 8.0
    g = np.exp(-((r - 8.0) / 1.5) ** 2) * np.exp(1j * k0 * r)   # resolved in k
    ens.psi[:] = 0
    ens.psi[0, 1, 0] = g / np.sqrt((np.abs(g) ** 2).sum() * dR)
    num0, den0 = (v[0] for v in ens.excited_R())
    nsteps = 3000
    for _ in range(nsteps):
        ens.step(np.zeros((1, 3)))
    num, den = (v[0] for v in ens.excited_R())
    assert abs(den - 1) < 1e-11
    assert abs(num / den - (num0 / den0 + k0 / sp.mass * nsteps * DTAU)) < 1e-6


def test_merged_phi_form_equals_literal_step():
    """The GPU stores phi = T^(1/2) psi and applies one full T per step,
    taking populations and dipole before the trailing half kinetic."""
    sp = W.Species(nr=64, jmax=2, mass=918.0)
    q = np.array([[0.9, 0.1, -0.3, 0.2]])
    lit = M.SpeciesEnsemble(sp, q, DTAU)
    mer = M.SpeciesEnsemble(sp, q, DTAU)
    Tfull = M.kinetic_propagator(sp, DTAU)
    phi = mer.apply_T(mer.psi, mer.Thalf)
    rng = np.random.default_rng(3)
    for n in range(200):
        E = rng.standard_normal((1, 3)) * 2e10
        mu_lit = lit.step(E)
        Em = np.einsum("kji,kj->ki", mer.O, E) / F_AU
        chi = mer.Vhalf[None] * phi
        chi = mer.coupling(chi, Em)
        chi = mer.Vhalf[None] * chi
        chi = chi * mer.mask
        mu_mer = np.einsum("kij,kj->ki", mer.O, mer.dipole_mol(chi))
        P_mer = (np.abs(chi) ** 2).sum(axis=(2, 3)) * mer.dR
        phi = mer.apply_T(chi, Tfull)
        assert np.max(np.abs(mu_lit - mu_mer)) < 1e-13
        assert np.max(np.abs(lit.populations() - P_mer)) < 1e-12
    psi_back = mer.apply_T(phi, M.kinetic_propagator(sp, -0.5 * DTAU))
    assert np.max(np.abs(psi_back - lit.psi)) < 1e-12


def test_atomic_unit_constants_are_consistent():
    e = 1.602176634e-19
    hbar = 6.62607015e-34 / (2 * np.pi)
    Eh = 4.3597447222071e-18
    assert abs(EA0 / (e * A0) - 1) < 1e-10
    assert abs(F_AU / (Eh / (e * A0)) - 1) < 1e-10
    assert abs(T_AU / (hbar / Eh) - 1) < 1e-10
