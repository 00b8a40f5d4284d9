"""The other benchmark configurations at full size, through the C ABI, on
sampled outputs the oracle computes one by one:

  * the 256^3 nanohole grid with 700,000 molecules at J <= 8 (116 GB of
    state), mixed kinetic pass;
  * the 192^3 split-ring grid with 400,000 molecules of three species
    (N_r 64/128/256, J 4/8/16; 120 GB of state), plain FP32 (the mixed pass
    has no N_r = 256 form), each species' plan picked by the autotuner;
  * 16 independent 64x64x128 nanohole cells with 20,000 molecules each at
    J <= 8, stepped in one launch per kernel.

Reaching the pulse peak takes thousands of steps of these grids, so each run
starts from a seeded E field written into the molecular layer (5e9 V/m,
smooth in x, y) and runs coupled for a few steps: the molecules are
polarised by it and scatter back into the grid.  The local fields of a
seeded sample are recorded at every step (the very E^n their kernels used)
and the oracle integrates those molecules in FP64 under them.  Every
molecule's populations are checked for finiteness and norm bookkeeping.
"""
import numpy as np
import pytest

import workloads as W
from oracle.coupled import ensemble
from oracle.molecule import dtau_au

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


def _state_bytes(wl):
    return sum(16 * sp.nr * sp.nrot * int((wl.species_id == i).sum()) for i, sp in enumerate(wl.species))


def _need(nbytes):
    import torch
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < nbytes:
        pytest.skip(f"needs {nbytes / 1e9:.0f} GB of free device memory, {free / 1e9:.0f} GB free")


def _inject(B, sim, wl, E0=5e9, seed=5):
    """A smooth seeded field in the molecular layer of every sim."""
    rng = np.random.default_rng(seed)
    k0, k1 = wl.meta["layer"]
    x = np.arange(wl.nx) * 2 * np.pi / wl.nx
    y = np.arange(wl.ny) * 2 * np.pi / wl.ny
    for s in range(wl.nsim):
        E = np.zeros((3, wl.nz, wl.ny, wl.nx), np.float32)
        for c in range(3):
            a, b, p, q = rng.uniform(0.5, 1.0), rng.uniform(0.5, 1.0), rng.uniform(0, 2 * np.pi, 2)[0], \
                rng.uniform(0, 2 * np.pi)
            pat = a * np.cos(x[None, :] + p) + b * np.sin(2 * y[:, None] + q)
            E[c, k0 - 2:k1 + 2] = (E0 / 2 * pat)[None].astype(np.float32)
        sim.write_fields(B.MS_FIELD_E, s, E)


def _time_steps(sim, wl, n=5):
    """Coupled steps after the check: wall time with the stream drained,
    printed with the state's one-read-one-write bandwidth."""
    import time
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(n)
    sim.populations()            # drains the stream
    dt = (time.perf_counter() - t0) / n
    gbs = 2 * _state_bytes(wl) / dt / 1e9
    print(f"{wl.name}: {dt * 1e3:.1f} ms per step, {wl.n_molecules / dt:.3e} molecule-steps/s, "
          f"{wl.cells / dt:.3e} cell-updates/s, state read+write {gbs:.0f} GB/s")


def _check_sample(wl, sim, sample, rec, nsteps):
    P = sim.populations()
    mu = sim.dipoles()
    absb, _ = sim.dissociation()
    worst = {}
    for si, sp in enumerate(wl.species):
        sel = sample[wl.species_id[sample] == si]
        if sel.size == 0:
            continue
        idx = np.searchsorted(sample, sel)
        ens = ensemble(sp, wl.quat[sel], dtau_au(wl.dt * wl.mol_substeps))
        for n in range(nsteps):
            ens.step(rec[n][idx].astype(np.float64))
        Po, mo = ens.populations(), ens.mu_lab
        dP = np.abs(P[sel] - Po).max()
        pe = Po[:, 1] > 1e-10
        rel = np.max(np.abs(P[sel][pe, 1] - Po[pe, 1]) / Po[pe, 1]) if pe.any() else 0.0
        dmu = np.abs(mu[sel] - mo).max() / max(np.abs(mo).max(), 1e-300)
        worst[si] = (dP, rel, dmu, Po[:, 1].max())
        assert Po[:, 1].max() > 1e-8, (si, "the injected field did not reach the sample")
        assert dP < 1e-5, (si, dP)
        assert rel < 1e-3, (si, rel)
        assert dmu < 1e-4, (si, dmu)
    tot = P.sum(axis=1) + absb.sum(axis=1)
    assert np.isfinite(P).all() and np.isfinite(mu).all()
    assert np.abs(tot - 1).max() < 1e-6
    print({k: tuple(f"{v:.2e}" for v in w) for k, w in worst.items()}, "norm", np.abs(tot - 1).max())


def test_nanohole_700k_molecules_mixed(B):
    wl = W.config2()
    _need(2 * _state_bytes(wl) + 8e9)          # state + streaming scratch + grid
    sim = B.Simulation(wl, precision=B.MS_PREC_MIXED_F16X3)
    _inject(B, sim, wl)
    sample = np.sort(np.random.default_rng(21).choice(wl.n_molecules, 8, replace=False))
    nsteps = 12
    rec = sim.record_local_fields(sample, nsteps)
    _check_sample(wl, sim, sample, rec, nsteps)
    _time_steps(sim, wl)
    sim.close()


def test_splitring_three_species_400k(B):
    """Plans picked by the create-time autotuner (the configuration's
    scheduling), one per species."""
    wl = W.config3()
    _need(2 * _state_bytes(wl) + 12e9)
    sim = B.Simulation(wl, autotune=B.MS_TUNE_MEASURE)
    print("tuned plans", [sim.plan(s) for s in range(3)])
    _inject(B, sim, wl)
    rng = np.random.default_rng(22)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(wl.species_id == s)[0], 3, replace=False)
                                     for s in range(3)]))
    nsteps = 8
    rec = sim.record_local_fields(sample, nsteps)
    _check_sample(wl, sim, sample, rec, nsteps)
    _time_steps(sim, wl)
    sim.close()


def test_sixteen_nanohole_cells_in_one_launch(B):
    wl = W.config4()
    _need(2 * _state_bytes(wl) + 4e9)
    sim = B.Simulation(wl)
    _inject(B, sim, wl)
    rng = np.random.default_rng(23)
    sample = np.sort(np.concatenate([rng.choice(np.nonzero(wl.sim_id == s)[0], 2, replace=False)
                                     for s in (0, 5, 10, 15)]))
    nsteps = 20
    rec = sim.record_local_fields(sample, nsteps)
    _check_sample(wl, sim, sample, rec, nsteps)
    _time_steps(sim, wl)
    sim.close()
