"""Pin of the coupled feedback loop as a whole: field -> molecules -> mean-
field polarization -> field, self-consistently.

A one-cell-thick sheet of frozen two-level molecules (one per cell, axis
along the x-polarised field) in vacuum, driven by a weak CW wave, reflects
and transmits like a thin polarizable sheet.  In linear response the
two-level polarizability with dephasing rate g2 is
    alpha(w) = d^2 [1/((w0 - w) - i g2) + 1/((w0 + w) + i g2)]   (a.u.),
the mean-field susceptibility of the cell layer (one molecule per dx^3)
chi = alpha e a0 / (F_au dx^3 eps0), and a sheet of thickness dx reflects
    r = i kappa / (1 - i kappa),  t = 1 / (1 - i kappa),  kappa = k dx chi / 2.
The denominator is the sheet's own field acting back on its molecules, so a
loop that dropped or mis-timed the feedback, mis-scaled the polarization or
the dipole, or used the wrong sign would miss these by more than the
tolerance (the feedback alone moves |r| by ~2% at resonance)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle.constants import C0, EA0, EPS0, F_AU, HBAR_EVS, T_AU
from oracle.coupled import CoupledOracle

E0, W_EV, T2, D = 1e6, 1.55, 10e-15, 5.0


def sheet_workload(delta_ev, nsteps=20000):
    sp = W.Species(model="bloch", w0_ev=W_EV + delta_ev, dipole=D, T2=T2)
    wl = W.custom("sheet", 4, 4, 96, src_k=20, pulses=[[E0, W_EV, 5e-15, 0.0]], src_kind="cw", layer=(60, 61),
                  n_per_sim=16, species=[sp], distinct=True, seed=1, nsteps=nsteps)
    q = np.tile([np.cos(np.pi / 4), 0.0, np.sin(np.pi / 4), 0.0], (16, 1))   # molecular axis along x
    return dataclasses.replace(wl, quat=q)


def closed_form(delta_ev, dx):
    w = W_EV / HBAR_EVS * T_AU
    w0 = (W_EV + delta_ev) / HBAR_EVS * T_AU
    g2 = T_AU / T2
    alpha = D * D * (1 / ((w0 - w) - 1j * g2) + 1 / ((w0 + w) + 1j * g2))
    chi = alpha * EA0 / (F_AU * dx ** 3 * EPS0)
    kap = (W_EV / HBAR_EVS / C0) * dx * chi / 2
    return 1j * kap / (1 - 1j * kap), 1 / (1 - 1j * kap), kap


def amplitudes(trace_r, trace_t):
    return (trace_r.max() - trace_r.min()) / 2 / E0, (trace_t.max() - trace_t.min()) / 2 / E0


@pytest.mark.parametrize("detune", [0.0, 1.0, -2.0])   # in units of the dephasing width hbar/T2
def test_polarizable_sheet_reflects_as_closed_form(detune):
    delta = detune * HBAR_EVS / T2
    wl = sheet_workload(delta)
    o = CoupledOracle(wl)
    per = int(round(2 * np.pi / (W_EV / HBAR_EVS) / wl.dt))
    tr, tt = [], []
    for n in range(wl.nsteps):
        o.step()
        if n >= wl.nsteps - 2 * per:           # steady state: the last two periods
            tr.append(o.f.Ex[0, 15, 0, 0])     # scattered-field region: the reflected wave
            tt.append(o.f.Ex[0, 80, 0, 0])     # beyond the sheet: the transmitted wave
    r_sim, t_sim = amplitudes(np.array(tr), np.array(tt))
    r, t, kap = closed_form(delta, wl.dx)
    assert abs(r_sim - abs(r)) < 6e-3 * abs(r), (r_sim, abs(r))
    assert abs(t_sim - abs(t)) < 5e-4, (t_sim, abs(t))
    # the feedback matters at this precision: without it |r| would be |kappa|
    if detune == 0.0:
        assert abs(abs(kap) - abs(r)) > 3 * 6e-3 * abs(r)
