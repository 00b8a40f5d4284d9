"""Pins of three molecular oracle terms that the other pins leave free: the
excited surface's exponential (the Eq. 7 family A + B exp(-beta (R - rc))),
the absorbing mask, and the centrifugal term j(j+1)/(2 mu R^2) of Eq. 5.
Each is checked against physics that does not call the oracle's own formula:

* excited surface -- Ehrenfest's theorem: a packet on the excited surface,
  field off, j = 0, absorber off, obeys d^2<R>/dt^2 = -<U_e'(R)>/mu, with
  U_e' taken from the analytic derivative -beta B exp(-beta (R - rc)); the
  split-operator step meets it to O(dtau^2);
* mask -- with the kinetic step the identity (mass 1e30) and the field off,
  a ground-surface packet held on one grid point r_i > r_a loses exactly
  1 - cos^(2p)(pi/2 (r_i - r_a)/(r_max - r_a)) of its norm in one step, and
  that loss is what the absorbed-norm tally records;
* centrifugal term -- the quasi-energy of the v = 0 level in channel j
  (eigenphase of the oracle's one-step propagator restricted to that
  channel) rises over j = 0 by the rotational-constant expansion of a Morse
  oscillator, B_0 j(j+1) - D [j(j+1)]^2, with B_e = 1/(2 mu r_e^2),
  alpha_e = 6 sqrt(w_e x_e B_e^3)/w_e - 6 B_e^2/w_e (Pekeris),
  B_0 = B_e - alpha_e/2 and D = 4 B_e^3/w_e^2.

Each pin is run once more with a plausible mistake planted in the oracle's
tables (a flipped sign, an inverted exponent, cos for cos^p, j^2 for
j(j+1), a dropped factor 2), on the CPU, and must then fail.
"""
import numpy as np
import pytest

import workloads as W
from oracle import molecule as M
from oracle.constants import T_AU

DT = 2e-9 / (2 * 299792458.0)
DTAU = DT / T_AU
IDENT = np.array([[1.0, 0.0, 0.0, 0.0]])


def _replace_potential(ens, surface, U_new):
    """Plant a different radial potential on one surface (mutation tests)."""
    Ug, Ue = M.potentials(ens.sp, ens.r)
    old = Ug if surface == 0 else Ue
    ens.V[surface] += (U_new - old)[None, :]
    ens.Vhalf = np.exp(-0.5j * ens.dtau * ens.V)


# ---- excited surface: Ehrenfest ---------------------------------------------

def _ehrenfest_error(dtau, nsteps, mutate=None):
    """Largest deviation of the second difference of <R>_e from
    -<U_e'>/mu over the run, relative to the largest acceleration."""
    sp = W.Species(nr=256, rmin=1.0, rmax=14.0, jmax=0, absorber_r=1e3)
    ens = M.SpeciesEnsemble(sp, IDENT, dtau)
    if mutate is not None:
        mutate(ens)
    r, dR = M.radial_grid(sp)
    g = np.exp(-((r - 4.0) / 0.4) ** 2)
    ens.psi[:] = 0
    ens.psi[0, 1, 0] = g / np.sqrt((g * g).sum() * dR)
    force = sp.beta * sp.B * np.exp(-sp.beta * (r - sp.rc))   # -U_e'(R), analytic
    R, F = [], []
    for n in range(nsteps + 1):
        pe = np.abs(ens.psi[0, 1, 0]) ** 2 * dR
        R.append((pe * r).sum())
        F.append((pe * force).sum())
        if n < nsteps:
            ens.step(np.zeros((1, 3)))
    R, F = np.array(R), np.array(F)
    acc = (R[2:] - 2.0 * R[1:-1] + R[:-2]) / dtau ** 2
    pred = F[1:-1] / sp.mass
    return np.max(np.abs(acc - pred)) / np.max(np.abs(pred)), R[-1] - R[0]


def test_excited_surface_obeys_ehrenfest():
    e4, moved = _ehrenfest_error(4 * DTAU, 300)
    e2, _ = _ehrenfest_error(2 * DTAU, 600)
    assert moved > 0.1                       # pushed outward by the repulsive wall
    assert e4 < 3e-6 and e2 < 1e-6
    assert 3.0 < e4 / e2 < 5.0               # the Strang error, O(dtau^2)


@pytest.mark.parametrize("mistake", ["sign of beta", "exponent divided by beta", "sign of rc"])
def test_ehrenfest_pin_catches_planted_excited_surface_mistakes(mistake):
    def mutate(ens):
        sp, r = ens.sp, ens.r
        U = {"sign of beta": sp.A + sp.B * np.exp(+sp.beta * (r - sp.rc)),
             "exponent divided by beta": sp.A + sp.B * np.exp(-(r - sp.rc) / sp.beta),
             "sign of rc": sp.A + sp.B * np.exp(-sp.beta * (r + sp.rc))}[mistake]
        _replace_potential(ens, 1, U)
    err, _ = _ehrenfest_error(4 * DTAU, 300, mutate)
    assert err > 0.1


# ---- absorbing mask -----------------------------------------------------------

def _mask_loss(power, ri, mutate=None):
    sp = W.Species(nr=64, jmax=0, mass=1e30, absorber_r=8.5, absorber_power=power)
    ens = M.SpeciesEnsemble(sp, IDENT, DTAU)
    if mutate is not None:
        mutate(ens)
    _, dR = M.radial_grid(sp)
    ens.psi[:] = 0
    ens.psi[0, 0, 0, ri] = 1.0 / np.sqrt(dR)
    ens.step(np.zeros((1, 3)))
    lost = 1.0 - ens.populations()[0].sum()
    return lost, ens.absorbed[0, 0]


def _expected_loss(power, ri):
    r_i = 1.0 + ri * 9.0 / 63.0
    if r_i <= 8.5:
        return 0.0
    return 1.0 - np.cos(0.5 * np.pi * (r_i - 8.5) / (10.0 - 8.5)) ** (2.0 * power)


@pytest.mark.parametrize("power", [0.125, 1.0])
@pytest.mark.parametrize("ri", [50, 58, 60, 62])
def test_mask_removes_the_closed_form_norm(power, ri):
    lost, tally = _mask_loss(power, ri)
    want = _expected_loss(power, ri)
    assert abs(lost - want) < 1e-13
    assert abs(tally - want) < 1e-13          # the absorbed-norm tally is that loss


@pytest.mark.parametrize("mistake", ["cos instead of cos^p", "cos^2p as the mask", "start at rmin"])
def test_mask_pin_catches_planted_mistakes(mistake):
    def mutate(ens):
        sp, r = ens.sp, ens.r
        x = np.clip((r - 8.5) / 1.5, 0.0, None)
        if mistake == "cos instead of cos^p":
            ens.mask = np.where(r > 8.5, np.cos(0.5 * np.pi * x), 1.0)
        elif mistake == "cos^2p as the mask":
            ens.mask = ens.mask ** 2
        else:
            ens.mask = np.where(r > 8.5, np.cos(0.5 * np.pi * (r - 8.5) / (10.0 - 1.0)) ** sp.absorber_power, 1.0)
    worst = max(abs(_mask_loss(0.125, ri, mutate)[0] - _expected_loss(0.125, ri)) for ri in (58, 60, 62))
    assert worst > 1e-3


# ---- centrifugal term ---------------------------------------------------------

def _v0_quasi_energy(sp, j, mutate=None):
    """Quasi-energy of the v = 0 level of channel (j, m = 0): the eigenphase,
    over dtau, of the oracle's field-free one-step propagator on that channel
    (built by stepping the nr unit vectors) whose eigenvector overlaps the
    j = 0 ground state most."""
    nr = sp.nr
    ens = M.SpeciesEnsemble(sp, np.tile(IDENT, (nr, 1)), DTAU)
    if mutate is not None:
        mutate(ens)
    ch = j * j + j
    ens.psi[:] = 0
    ens.psi[np.arange(nr), 0, ch, np.arange(nr)] = 1.0
    ens.step(np.zeros((nr, 3)))
    U = ens.psi[:, 0, ch, :].T                    # column b: the image of e_b
    lam, V = np.linalg.eig(U)
    k = np.argmax(np.abs(M.ground_state(sp) @ V))
    return -np.angle(lam[k]) / DTAU


def _rotational_expansion(sp, j):
    Be = 1.0 / (2.0 * sp.mass * sp.re ** 2)
    we = sp.a * np.sqrt(2.0 * sp.De / sp.mass)
    wexe = we * we / (4.0 * sp.De)
    alpha = 6.0 * np.sqrt(wexe * Be ** 3) / we - 6.0 * Be ** 2 / we
    D = 4.0 * Be ** 3 / we ** 2
    x = j * (j + 1.0)
    return (Be - 0.5 * alpha) * x - D * x * x


def _rotational_errors(mutate=None):
    sp = W.Species(nr=128, jmax=4, absorber_r=1e3)
    e0 = _v0_quasi_energy(sp, 0, mutate)
    return [abs((_v0_quasi_energy(sp, j, mutate) - e0) / _rotational_expansion(sp, j) - 1.0)
            for j in (1, 2, 3, 4)]


def test_centrifugal_term_gives_the_rotational_constants():
    errs = _rotational_errors()
    # the remainder (~1.2e-4) is the expansion's higher orders plus the
    # split-operator error; j^2 for j(j+1) would be off by >= 20 %
    assert max(errs) < 2.5e-4, errs


@pytest.mark.parametrize("mistake", ["j^2 for j(j+1)", "mu R^2 for 2 mu R^2"])
def test_centrifugal_pin_catches_planted_mistakes(mistake):
    def mutate(ens):
        sp = ens.sp
        jj = np.array([j * (j + 1) for j, _ in ens.ch], float)
        bad = np.array([j * j for j, _ in ens.ch], float) if mistake.startswith("j^2") else 2.0 * jj
        delta = (bad - jj)[:, None] / (2.0 * sp.mass * ens.r[None, :] ** 2)
        ens.V += delta[None]
        ens.Vhalf = np.exp(-0.5j * ens.dtau * ens.V)
    assert max(_rotational_errors(mutate)) > 0.1
