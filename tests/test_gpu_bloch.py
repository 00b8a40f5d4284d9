"""Frozen two-level (Bloch) molecules on the GPU against the FP64 oracle,
through the C ABI: prescribed drives (every step and every 40th step, with
and without relaxation, up to 700,000 molecules), the coupled FDTD step with
Bloch molecules alone and beside a wavepacket species, and checkpoints.

Tolerances as for the wavepacket model: populations abs 1e-5, dipoles 1e-4
of their largest magnitude, fields relative L2 1e-4.
"""
import dataclasses

import numpy as np
import pytest

import workloads as W
from oracle.bloch import BlochEnsemble
from oracle.constants import HBAR_EVS
from oracle.coupled import CoupledOracle, PrescribedOracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_04487_gb300 import build
    build.build()
    from paper_2209_04487_gb300 import binding
    return binding


def _bloch(w0_ev=1.55, d=2.0, T1=0.0, T2=0.0):
    return W.Species(model="bloch", w0_ev=w0_ev, dipole=d, T1=T1, T2=T2)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("N,T1,T2,nmol,nsteps,E0", [
    (1, 0.0, 0.0, 37, 4000, 2e9), (1, 30e-15, 10e-15, 37, 4000, 2e9), (40, 0.0, 0.0, 37, 4000, 2e9),
    (4, 50e-15, 20e-15, 700_000, 240, 1e10),     # the paper's largest ensemble
])
def test_prescribed_bloch_matches_oracle(B, N, T1, T2, nmol, nsteps, E0):
    sp = _bloch(T1=T1, T2=T2)
    wl = W.custom("bloch prescribed", 8, 8, 48, n_per_sim=nmol, species=[sp], layer=(20, 24), seed=11,
                  nsteps=nsteps, mol_substeps=N)
    rng = np.random.default_rng(3)
    amp = rng.standard_normal((nmol, 3)) * E0
    t = np.arange(nsteps) * wl.dt
    wave = np.cos(1.55 / HBAR_EVS * t) * np.minimum(t / 2e-15, 1.0)
    sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED)
    sim.set_prescribed(amp, wave)
    sim.step(nsteps)
    o = PrescribedOracle(wl, amp, wave).run(nsteps)
    P, Po = sim.populations(), o.populations()
    assert Po[:, 1].max() > 1e-3
    assert np.abs(P - Po).max() < 1e-5
    assert np.abs(sim.dipoles() - o.mu).max() < 1e-4 * np.abs(o.mu).max()
    absb, Rr = sim.dissociation()
    assert np.all(absb == 0.0)
    Ro = o.excited_R()
    assert np.abs(Rr - Ro).max() < 1e-5 * sp.re
    # the dipole lies along each molecule's axis with |u| <= 1
    axis = BlochEnsemble(sp, wl.quat, 1.0).axis
    mu = sim.dipoles()
    u = np.einsum("ni,ni->n", mu, axis) / sp.dipole
    assert np.abs(mu - (sp.dipole * u)[:, None] * axis).max() < 1e-6 * sp.dipole
    assert np.abs(u).max() <= 1.0 + 1e-6


def test_coupled_bloch_matches_oracle(B):
    """Bloch molecules polarising the grid: a dense layer near resonance."""
    wl = W.custom("coupled bloch", 16, 16, 48, src_k=14, pulses=[[2e9, 1.55, 3e-15, 4e-15]], layer=(22, 26),
                  n_per_sim=400, species=[_bloch(d=3.0, T2=20e-15)], seed=6, nsteps=1500)
    sim = B.Simulation(wl)
    sim.step(wl.nsteps)
    o = CoupledOracle(wl).run(wl.nsteps)
    E = sim.fields(B.MS_FIELD_E)
    Eo = np.stack([o.f.Ex[0], o.f.Ey[0], o.f.Ez[0]])
    assert _rel(E, Eo) < 1e-4
    P, Po = sim.populations(), o.populations()
    assert Po[:, 1].max() > 1e-4
    assert np.abs(P - Po).max() < 1e-5
    assert np.abs(sim.dipoles() - o.mu).max() < 1e-4 * np.abs(o.mu).max()
    # the molecules changed the field: the same run without them differs
    bare = CoupledOracle(wl, with_molecules=False).run(wl.nsteps)
    assert _rel(np.stack([bare.f.Ex[0], bare.f.Ey[0], bare.f.Ez[0]]), Eo) > 1e-4


def test_bloch_beside_wavepacket_species_substepped(B):
    """A Bloch species and a wavepacket species in one coupled run, molecules
    every 5th step, CW drive."""
    species = [W.species_config0(jmax=1), _bloch(w0_ev=1.5, d=2.0, T1=40e-15)]
    wl = W.custom("mixed models", 16, 16, 48, src_k=14, pulses=[[1e10, 1.5498, 1e-15, 0.0]], layer=(22, 26),
                  n_per_sim=160, species=species, fractions=[0.5, 0.5], seed=19, nsteps=600, src_kind="cw",
                  mol_substeps=5)
    sim = B.Simulation(wl)
    assert sim.species_path(1) == B.MS_MOL_FUSED
    sim.step(wl.nsteps)
    o = CoupledOracle(wl).run(wl.nsteps)
    E = sim.fields(B.MS_FIELD_E)
    assert _rel(E, np.stack([o.f.Ex[0], o.f.Ey[0], o.f.Ez[0]])) < 1e-4
    P, Po = sim.populations(), o.populations()
    assert np.abs(P - Po).max() < 1e-5
    assert np.abs(sim.dipoles() - o.mu).max() < 1e-4 * np.abs(o.mu).max()
    for s in (0, 1):
        assert Po[wl.species_id == s, 1].max() > 1e-6


def test_bloch_checkpoint_is_bitwise(B, tmp_path):
    wl = W.custom("bloch ck", 16, 16, 48, src_k=14, pulses=[[5e9, 1.55, 2e-15, 3e-15]], layer=(22, 26),
                  n_per_sim=100, species=[_bloch(T1=20e-15, T2=9e-15)], seed=4, nsteps=200)
    ref = B.Simulation(wl)
    ref.step(200)
    want = (ref.populations(), ref.dipoles(), ref.fields(B.MS_FIELD_E))
    ref.close()
    a = B.Simulation(wl)
    a.step(77)
    path = str(tmp_path / "b.ck")
    a.save(path)
    a.close()
    b = B.Simulation(wl)
    b.load(path)
    b.step(123)
    for x, y in zip(want, (b.populations(), b.dipoles(), b.fields(B.MS_FIELD_E))):
        assert np.array_equal(x, y)
    # a wavepacket handle of the same sizes refuses the Bloch checkpoint
    c = B.Simulation(dataclasses.replace(wl, species=[W.species_config0(jmax=1)]))
    with pytest.raises(B.MSError) as e:
        c.load(path)
    assert e.value.code == B.MS_EINVAL
    b.close()
    c.close()


@pytest.mark.parametrize("detune", [0.0, -2.0])
def test_gpu_polarizable_sheet_reflects_as_closed_form(B, detune):
    """The coupled loop on the GPU against the thin-sheet closed form (the
    oracle's pin of the whole loop; see tests/test_oracle_coupled_loop_pins)."""
    from oracle.constants import HBAR_EVS
    from tests.test_oracle_coupled_loop_pins import E0, T2, W_EV, amplitudes, closed_form, sheet_workload
    delta = detune * HBAR_EVS / T2
    wl = sheet_workload(delta)
    per = int(round(2 * np.pi / (W_EV / HBAR_EVS) / wl.dt))
    sim = B.Simulation(wl)
    sim.step(wl.nsteps - 2 * per)
    tr, tt = [], []
    for _ in range(2 * per):
        sim.step(1)
        E = sim.fields(B.MS_FIELD_E)
        tr.append(E[0, 15, 0, 0])
        tt.append(E[0, 80, 0, 0])
    sim.close()
    r_sim, t_sim = amplitudes(np.array(tr, np.float64), np.array(tt, np.float64))
    r, t, _ = closed_form(delta, wl.dx)
    assert abs(r_sim - abs(r)) < 6e-3 * abs(r), (r_sim, abs(r))
    assert abs(t_sim - abs(t)) < 5e-4, (t_sim, abs(t))
