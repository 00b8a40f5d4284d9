"""The other benchmark configurations at full size, through the C ABI:

  * the 256^3 nanohole grid with 700,000 molecules at J <= 8 (116 GB of
    state), mixed kinetic pass;
  * the 192^3 split-ring grid with 400,000 molecules of three species
    (N_r 64/128/256, J 4/8/16; 120 GB of state), plain FP32 (the mixed pass
    has no N_r = 256 form), each species' plan picked by the autotuner;
  * 16 independent 64x64x128 nanohole cells with 20,000 molecules each at
    J <= 8, stepped in one launch per kernel.

The oracle cannot run these coupled systems, so each is checked in three
parts whose oracle inputs come from the test, never from the CUDA path:
  1. every molecule under a seeded prescribed drive (5e9 V/m through its
     maximum) for a few steps, a seeded sample integrated one by one by the
     oracle on the same drive;
  2. the coupled run (molecules and fields, from a seeded E field written
     into the molecular layer): properties that hold at any size -- every
     molecule's norm bookkeeping and finite values -- and its step time;
  3. the full field grid(s) without molecules from the same seeded field, a
     few steps, against the oracle on the whole grid.
Each part's device memory is returned before the next (the large states
first).
"""
import numpy as np
import pytest

import workloads as W
from oracle.coupled import CoupledOracle, PrescribedOracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_04487_gb300 import build
    build.build()
    from paper_2209_04487_gb300 import binding
    return binding


def _release():
    """Return the closed handles' device memory to the device (the binding
    allocates through PyTorch's caching allocator)."""
    import gc
    import torch
    gc.collect()
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def _state_bytes(wl):
    return sum(16 * sp.nr * sp.nrot * int((wl.species_id == i).sum()) for i, sp in enumerate(wl.species))


def _need(nbytes):
    import torch
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes:
        pytest.skip(f"needs {nbytes / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")


def _seeded_field(wl, E0=5e9, seed=5):
    """A smooth seeded E field in the molecular layer of every sim, [nsim][3][nz][ny][nx]."""
    rng = np.random.default_rng(seed)
    k0, k1 = wl.meta["layer"]
    x = np.arange(wl.nx) * 2 * np.pi / wl.nx
    y = np.arange(wl.ny) * 2 * np.pi / wl.ny
    out = np.zeros((wl.nsim, 3, wl.nz, wl.ny, wl.nx), np.float32)
    for s in range(wl.nsim):
        for c in range(3):
            a, b, p, q = rng.uniform(0.5, 1.0), rng.uniform(0.5, 1.0), rng.uniform(0, 2 * np.pi), \
                rng.uniform(0, 2 * np.pi)
            pat = a * np.cos(x[None, :] + p) + b * np.sin(2 * y[:, None] + q)
            out[s, c, k0 - 2:k1 + 2] = (E0 / 2 * pat)[None].astype(np.float32)
    return out


def _molecules_prescribed(B, wl, precision, sample, nsteps=12, state_form=0):
    """Part 1: all molecules under a seeded prescribed drive; the sample against the oracle."""
    amp, wave = W.prescribed_drive(wl.n_molecules, nsteps, wl.dt, E0=5e9, carrier_ev=6.0, fwhm=0.02e-15,
                                   t0=0.5 * nsteps * wl.dt, seed=79)
    sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED, precision=precision, state_form=state_form)
    sim.set_prescribed(amp, wave)
    sim.step(nsteps)
    P, mu = sim.populations(), sim.dipoles()
    absb, _ = sim.dissociation()
    sim.close()
    del sim
    _release()
    o = PrescribedOracle(wl, amp, wave, select=sample).run(nsteps)
    Po = o.populations()
    worst = (np.abs(P[sample] - Po).max(), np.abs(mu[sample] - o.mu).max() / np.abs(o.mu).max())
    print(f"{wl.name}: prescribed sample |dP| {worst[0]:.2e}, |dmu|/max {worst[1]:.2e}, P_e max {Po[:, 1].max():.2e}")
    assert Po[:, 1].max() > 1e-8
    assert worst[0] < 1e-5
    sel = Po[:, 1] > 1e-10
    assert np.max(np.abs(P[sample][sel, 1] - Po[sel, 1]) / Po[sel, 1]) < 1e-3
    assert worst[1] < 1e-4
    tot = P.sum(axis=1) + absb.sum(axis=1)
    assert np.isfinite(P).all() and np.abs(tot - 1).max() < 1e-6


def _fields_vs_oracle(B, wl, E, nsteps=6):
    """Part 2: the full grid(s) without molecules from the seeded field, against the oracle."""
    sim = B.Simulation(wl, with_molecules=False)
    for s in range(wl.nsim):
        sim.write_fields(B.MS_FIELD_E, s, E[s])
    sim.step(nsteps)
    o = CoupledOracle(wl, with_molecules=False)
    Ef = E.astype(np.float64)
    o.f.Ex[:], o.f.Ey[:], o.f.Ez[:] = Ef[:, 0], Ef[:, 1], Ef[:, 2]
    o.run(nsteps)
    for s in range(wl.nsim):
        got = np.stack([sim.fields(B.MS_FIELD_E, s), sim.fields(B.MS_FIELD_H, s)])
        want = np.stack([np.stack([o.f.Ex[s], o.f.Ey[s], o.f.Ez[s]]), np.stack([o.f.Hx[s], o.f.Hy[s], o.f.Hz[s]])])
        for k in range(2):
            rel = np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k])
            assert rel < 1e-4, (s, "EH"[k], rel)
    sim.close()
    del sim
    _release()


def _coupled_properties(B, wl, E, nsteps, **kw):
    """Part 3: the coupled run from the seeded field: norm bookkeeping, finite values, step time."""
    import time
    import torch
    sim = B.Simulation(wl, **kw)
    if kw.get("autotune"):
        print("tuned plans", [sim.plan(s) for s in range(len(wl.species))])
    for s in range(wl.nsim):
        sim.write_fields(B.MS_FIELD_E, s, E[s])
    sim.step(nsteps)
    P, mu = sim.populations(), sim.dipoles()
    absb, _ = sim.dissociation()
    tot = P.sum(axis=1) + absb.sum(axis=1)
    assert np.isfinite(P).all() and np.isfinite(mu).all()
    assert np.abs(tot - 1).max() < 1e-6
    assert P[:, 1].max() > 1e-8                          # the field reached the molecules
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(5)
    sim.populations()                                    # drains the stream
    dt = (time.perf_counter() - t0) / 5
    print(f"{wl.name}: {dt * 1e3:.1f} ms per coupled step (host clock), "
          f"{wl.n_molecules / dt:.3e} molecule-steps/s, {wl.cells / dt:.3e} cell-updates/s")
    sim.close()
    del sim
    _release()


def test_nanohole_700k_molecules_mixed(B):
    wl = W.config2()
    _need(2 * _state_bytes(wl) + 8e9)          # state + streaming scratch + grid
    sample = np.sort(np.random.default_rng(21).choice(wl.n_molecules, 8, replace=False))
    _molecules_prescribed(B, wl, B.MS_PREC_MIXED_F16X3, sample)
    E = _seeded_field(wl)
    _coupled_properties(B, wl, E, 8, precision=B.MS_PREC_MIXED_F16X3)
    _fields_vs_oracle(B, wl, E)


def test_splitring_three_species_400k(B):
    """Plans picked by the create-time autotuner (the configuration's
    scheduling), one per species."""
    wl = W.config3()
    _need(2 * _state_bytes(wl) + 12e9)
    rng = np.random.default_rng(22)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(wl.species_id == s)[0], 3, replace=False)
                                     for s in range(3)]))
    _molecules_prescribed(B, wl, B.MS_PREC_FP32, sample, nsteps=8)
    E = _seeded_field(wl)
    _coupled_properties(B, wl, E, 8, autotune=B.MS_TUNE_MEASURE)
    _fields_vs_oracle(B, wl, E)


def test_sixteen_nanohole_cells_in_one_launch(B):
    wl = W.config4()
    _need(2 * _state_bytes(wl) + 4e9)
    rng = np.random.default_rng(23)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(wl.sim_id == s)[0], 2, replace=False)
                                     for s in (0, 5, 10, 15)]))
    _molecules_prescribed(B, wl, B.MS_PREC_FP32, sample, nsteps=20)
    E = _seeded_field(wl)
    _coupled_properties(B, wl, E, 20)
    _fields_vs_oracle(B, wl, E)


@pytest.mark.parametrize("config", [2, 3])
def test_parity_reduced_state_at_full_size(B, config):
    """The parity-reduced rows (the rows the j = 0 start populates) on the
    full nanohole (700,000 molecules, J <= 8) and three-species (J 4/8/16)
    workloads: every molecule under the prescribed drive with a seeded
    sample against the oracle (which keeps every row), then the coupled run's
    bookkeeping."""
    wl = W.config2() if config == 2 else W.config3()
    _need(_state_bytes(wl) + 12e9)              # half the rows, state and scratch
    rng = np.random.default_rng(40 + config)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(wl.species_id == s)[0], 3, replace=False)
                                     for s in range(len(wl.species))]))
    _molecules_prescribed(B, wl, B.MS_PREC_FP32, sample, nsteps=8, state_form=B.MS_STATE_PARITY)
    E = _seeded_field(wl)
    _coupled_properties(B, wl, E, 8, state_form=B.MS_STATE_PARITY)
