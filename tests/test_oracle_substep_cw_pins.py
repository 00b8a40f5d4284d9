"""Pins of the oracle's molecular cadence (the molecules advance every N-th
field step by N dt, under that step's field) and of the CW drive (sin^2
turn-on, then a constant amplitude)."""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle.constants import HBAR_EVS
from oracle.coupled import CoupledOracle, PrescribedOracle
from oracle.fdtd import cw


def _prescribed(N, nsteps, dt_scale=1.0):
    sp = W.Species(nr=64, jmax=1, A=0.05)
    wl = W.custom("sub", 8, 8, 48, n_per_sim=6, species=[sp], layer=(20, 24), seed=4, nsteps=nsteps,
                  mol_substeps=N)
    return wl


def test_substeps_equal_a_run_at_the_longer_step():
    """N sub-steps over N K field steps are exactly K molecular steps of N dt
    under the field samples of steps 0, N, 2N, ..."""
    N, K = 5, 40
    wl = _prescribed(N, N * K)
    amp, wave = W.prescribed_drive(wl.n_molecules, N * K, wl.dt, E0=3e10, carrier_ev=6.0, fwhm=0.5e-15,
                                   t0=0.5e-15)
    a = PrescribedOracle(wl, amp, wave).run(N * K)
    wl1 = dataclasses.replace(wl, dt=wl.dt * N, mol_substeps=1)
    b = PrescribedOracle(wl1, amp, wave[::N]).run(K)
    assert np.array_equal(a.populations(), b.populations())
    assert np.array_equal(a.mu, b.mu)
    assert a.populations()[:, 1].max() > 1e-6     # the drive did something


def test_every_40th_step_tracks_every_step():
    """The paper's cadence: molecular dynamics every 40th field step (0.1 fs
    at its 2.5 as step) converges.  Weak resonant CW-like drive, 4000 steps."""
    nsteps = 4000
    wl1 = _prescribed(1, nsteps)
    wl40 = dataclasses.replace(wl1, mol_substeps=40)
    t = np.arange(nsteps) * wl1.dt
    w = np.cos(6.0 / HBAR_EVS * t) * np.minimum(t / 2e-15, 1.0)
    amp = np.tile([2e9, 0.0, 1e9], (wl1.n_molecules, 1))
    p1 = PrescribedOracle(wl1, amp, w).run(nsteps).populations()
    p40 = PrescribedOracle(wl40, amp, w).run(nsteps).populations()
    assert p1[:, 1].max() > 1e-6
    assert np.max(np.abs(p40[:, 1] - p1[:, 1]) / p1[:, 1].max()) < 0.05


def test_cw_waveform_and_vacuum_amplitude():
    t_on = 1e-15
    t = np.array([0.0, 0.5 * t_on, t_on, 3 * t_on])
    v = cw(t, 1.0, 1.5498, t_on, 0.0)
    w = 1.5498 / HBAR_EVS
    assert v[0] == 0.0
    assert np.allclose(v[1], 0.5 * np.cos(w * 0.5 * t_on))
    assert np.allclose(v[2:], np.cos(w * t[2:]))
    # vacuum TF/SF: full amplitude E0 in the total-field region after the turn-on;
    # the scattered-field region only holds the far CPML's return (< 1e-4, its pin)
    wl = W.custom("cw vacuum", 4, 4, 48, src_k=14, pulses=[[1e9, 1.5498, t_on, 0.0]], n_per_sim=0,
                  nsteps=3000, src_kind="cw")
    o = CoupledOracle(wl)
    peak = 0.0
    for n in range(wl.nsteps):
        o.step()
        if n > 2000:
            peak = max(peak, np.abs(o.f.Ex[0, 24]).max())
    assert abs(peak - 1e9) < 2e-3 * 1e9
    assert np.abs(o.f.Ex[0, 4:12]).max() < 1e-4 * 1e9
