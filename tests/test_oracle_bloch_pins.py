"""Pins of the frozen two-level (Bloch) oracle against closed forms: the
detuned Rabi formula under a static field with its RK4 order, free
precession with T1/T2 relaxation, the resonant rotating-wave Rabi
oscillation under a CW drive, the dipole's orientation dependence, and
Bloch-vector length conservation."""
import math

import numpy as np
import pytest

import workloads as W
from oracle.bloch import BlochEnsemble, rk4_step
from oracle.constants import F_AU, HARTREE_EV, T_AU, HBAR_EVS
from oracle.coupled import PrescribedOracle


def _ens(n=1, w0_ev=2.0, d=2.5, T1=0.0, T2=0.0, dtau=0.1, quat=None):
    sp = W.Species(model="bloch", w0_ev=w0_ev, dipole=d, T1=T1, T2=T2)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quat is None else np.asarray(quat, np.float64)
    return BlochEnsemble(sp, q, dtau)


def _run_static(h, t_end, w0_ev, d, E_au):
    e = _ens(w0_ev=w0_ev, d=d, dtau=h)
    for _ in range(int(round(t_end / h))):
        e.step(np.array([[0.0, 0.0, E_au * F_AU]]))   # along the molecular (z) axis
    return e.populations()[0, 1]


def test_static_field_detuned_rabi_and_rk4_order():
    """Constant field: P_e = W^2/(W^2 + w0^2) sin^2(sqrt(W^2 + w0^2) t/2),
    W = 2 d E; the RK4 error falls 16x per halving of the step."""
    w0_ev, d, E = 1.0, 2.0, 0.01
    w0 = w0_ev / HARTREE_EV
    Om = 2 * d * E
    t_end = 400.0
    g = np.hypot(Om, w0)
    exact = Om ** 2 / g ** 2 * np.sin(g * t_end / 2) ** 2
    errs = [abs(_run_static(h, t_end, w0_ev, d, E) - exact) for h in (2.0, 1.0, 0.5)]
    assert exact > 0.1
    assert errs[2] < 1e-7
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


def test_free_precession_with_relaxation():
    """E = 0 from a superposition: coherences rotate at w0 and decay at 1/T2,
    the inversion relaxes to -1 at 1/T1."""
    T1, T2 = 20e-15, 8e-15
    e = _ens(w0_ev=1.5, T1=T1, T2=T2, dtau=0.05)
    y0 = np.array([0.6, 0.0, 0.8])
    e.y[:] = y0
    n = 4000
    for _ in range(n):
        e.step(np.zeros((1, 3)))
    t = n * 0.05
    w0 = 1.5 / HARTREE_EV
    g1, g2 = T_AU / T1, T_AU / T2
    want = np.array([y0[0] * np.exp(-g2 * t) * np.cos(w0 * t), -y0[0] * np.exp(-g2 * t) * np.sin(w0 * t),
                     -1 + (y0[2] + 1) * np.exp(-g1 * t)])
    assert np.abs(e.y[0] - want).max() < 1e-9


def test_resonant_cw_rotating_wave_rabi():
    """E = E0 cos(w0 t) on resonance: P_e follows sin^2(d E0 t / 2) (rotating
    wave), up to counter-rotating corrections of order d E0 / w0 (here 0.03)
    of the full swing."""
    sp = W.Species(model="bloch", w0_ev=2.0, dipole=2.0)
    n = 24000
    wl = W.custom("bloch cw", 8, 8, 48, n_per_sim=3, species=[sp], layer=(20, 24), seed=2, nsteps=n)
    t = np.arange(n) * wl.dt
    E0 = 5e8                                        # V/m
    wave = np.cos(2.0 / HBAR_EVS * t)
    axis = BlochEnsemble(sp, wl.quat, 1.0).axis
    amp = E0 * axis                                 # field along each molecule's axis
    o = PrescribedOracle(wl, amp, wave)
    rabi = 2.0 * E0 / F_AU                          # d E0 (a.u.)
    seen = []
    for step in (6000, 12000, 18000, 24000):
        o.run(step - o.n)
        want = np.sin(rabi * (step * wl.dt / T_AU) / 2) ** 2
        got = o.populations()[:, 1]
        assert np.abs(got - want).max() < 0.01, (step, got, want)
        seen.append(want)
    assert max(seen) > 0.9 and min(seen) < 0.3     # a Rabi cycle was covered


def test_orientation_and_dipole():
    """Only the field along the molecular axis drives; the dipole is d u
    along the axis."""
    q_z = [1.0, 0.0, 0.0, 0.0]                      # axis z
    q_x = [np.cos(np.pi / 4), 0.0, np.sin(np.pi / 4), 0.0]   # z turned onto x (rotation about y)
    e = _ens(n=2, w0_ev=1.0, d=1.5, dtau=0.5, quat=[q_z, q_x])
    assert np.allclose(e.axis[1], [1.0, 0.0, 0.0])
    for _ in range(200):
        mu = e.step(np.tile([0.0, 0.0, 5e9], (2, 1)))   # field along z
    assert e.populations()[0, 1] > 1e-4
    # the turned axis is x up to rounding of its quaternion (1e-16 along z)
    assert e.populations()[1, 1] < 1e-25 and np.abs(mu[1]).max() < 1e-12
    assert np.allclose(mu[0], [0.0, 0.0, 1.5 * e.y[0, 0]])
    assert abs(mu[0, 2]) > 0


@pytest.mark.parametrize("h", [0.1, 1.0])
def test_bloch_vector_length_conserved(h):
    """Without relaxation the Bloch vector keeps unit length up to the RK4
    amplitude error 1 - |R(i phi)| = phi^6/144 + O(phi^8) per step."""
    e = _ens(n=4, w0_ev=1.5, d=3.0, dtau=h, quat=np.random.default_rng(1).standard_normal((4, 4)))
    rng = np.random.default_rng(2)
    for _ in range(500):
        e.step(rng.standard_normal((4, 3)) * 2e9)
    L = np.linalg.norm(e.y, axis=1)
    phi = np.hypot(1.5 / HARTREE_EV, 2 * 3.0 * 4 * 2e9 / F_AU) * h
    assert np.abs(L - 1).max() < 500 * phi ** 6 / 144 + 1e-12


def test_rk4_step_is_fourth_order_taylor_for_linear_rhs():
    """For a held field the system is linear, y' = A y + b; one RK4 step is
    the fourth-order Taylor polynomial of the exact flow."""
    rng = np.random.default_rng(5)
    w0, om, g1, g2, h = 0.07, 0.03, 0.002, 0.005, 0.8
    A = np.array([[-g2, w0, 0.0], [-w0, -g2, -om], [0.0, om, -g1]])
    b = np.array([0.0, 0.0, -g1])
    y = rng.standard_normal(3)
    # Taylor of the affine flow: y + sum_k h^k/k! A^(k-1) (A y + b)
    f = A @ y + b
    want = y.copy()
    term = f
    for k in range(1, 5):
        want = want + h ** k / math.factorial(k) * term
        term = A @ term
    got = rk4_step(y[None, :], h, w0, np.array([om]), g1, g2)[0]
    assert np.abs(got - want).max() < 1e-15
