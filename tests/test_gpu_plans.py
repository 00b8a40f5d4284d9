"""Every (layout, kernel, chunk width) plan a species can run computes the
same step: each is pinned in turn through ms_set_species_plan and compared
with the FP64 oracle at the plain tolerances.  The create-time autotuner
picks one of them, and pinning its pick reproduces the tuned run bit for bit.
"""
import numpy as np
import pytest

import workloads as W
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


def _plans(B):
    """(layout, kernel, chunk, grid): both tiled kernels (one and two radial
    points a thread) at their tile widths and three grids (as many CTAs as
    fit, one per SM, one per molecule)."""
    kc = [(B.MS_KERN_POINT, 0, 0)] + \
        [(k, t, g) for k in (B.MS_KERN_TILE, B.MS_KERN_PAIR) for t in (32, 16, 8) for g in (0, 1, -1)] + \
        [(B.MS_KERN_CHUNK, c, 0) for c in (32, 16, 8, 4)]
    return [(p, k, c, g) for p in (B.MS_MOL_FUSED, B.MS_MOL_STREAMING) for k, c, g in kc]


@pytest.mark.parametrize("nr,jmax,nmol", [(64, 1, 23), (128, 4, 9), (128, 6, 5), (64, 8, 4), (64, 10, 3)])
def test_every_plan_matches_oracle(B, nr, jmax, nmol):
    sp = W.Species(nr=nr, jmax=jmax, A=0.05)
    nsteps = 200
    wl = W.custom("plans", 8, 8, 48, n_per_sim=nmol, species=[sp], layer=(20, 24), seed=nr + jmax, nsteps=nsteps)
    amp, wave = W.prescribed_drive(nmol, nsteps, wl.dt, E0=3e10, carrier_ev=6.0, fwhm=0.5e-15, t0=0.4e-15)
    o = PrescribedOracle(wl, amp, wave).run(nsteps)
    Po = o.populations()
    assert Po[:, 1].max() > 1e-6
    ran = []
    results = {}
    for plan in _plans(B):
        sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED, mol_path=B.MS_MOL_STREAMING)
        try:
            sim.set_plan(0, *plan)
        except B.MSError as e:
            assert e.code == B.MS_EINVAL
            sim.close()
            continue
        assert sim.plan_ex(0) == plan
        sim.set_prescribed(amp, wave)
        sim.step(nsteps)
        P, mu = sim.populations(), sim.dipoles()
        sim.close()
        results[plan] = (P, mu)
        assert np.abs(P - Po).max() < 1e-5, plan
        sel = Po[:, 1] > 1e-10
        assert np.max(np.abs(P[sel, 1] - Po[sel, 1]) / Po[sel, 1]) < 1e-3, plan
        assert np.abs(mu - o.mu).max() < 1e-4 * np.abs(o.mu).max(), plan
        ran.append(plan)
    kinds = {k for _, k, _, _ in ran}
    assert B.MS_KERN_CHUNK in kinds and len(ran) >= 3, ran
    if jmax <= 4:
        assert B.MS_KERN_POINT in kinds
    tiles = {c for _, k, c, _ in ran if k == B.MS_KERN_TILE}
    assert tiles == ({8} if jmax >= 9 else {16, 32}), ran   # the tile widths of the basis size
    pairs = {c for _, k, c, _ in ran if k == B.MS_KERN_PAIR}
    assert pairs == ({8} if jmax >= 9 else ({16, 8} if jmax >= 5 else {32, 16})), ran
    # the grid only changes which CTA runs a molecule: identical results
    for k, ts in ((B.MS_KERN_TILE, tiles), (B.MS_KERN_PAIR, pairs)):
        for t in ts:
            runs = [results[p] for p in ran if p[1] == k and p[2] == t]
            assert len(runs) == 3
            for P, mu in runs[1:]:
                assert np.array_equal(P, runs[0][0]) and np.array_equal(mu, runs[0][1])


def test_autotuned_three_species_coupled(B):
    """Three species tuned at create time, coupled run against the oracle;
    pinning the tuned plans reproduces the run bit for bit."""
    species = [W.species_config0(jmax=1), W.Species(nr=128, jmax=4, A=0.05), W.Species(nr=64, jmax=6)]
    wl = W.custom("tuned", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 2e-15]], layer=(22, 26),
                  n_per_sim=120, species=species, fractions=[0.4, 0.3, 0.3], seed=31, nsteps=300)
    a = B.Simulation(wl, autotune=B.MS_TUNE_MEASURE)
    plans = [a.plan_ex(s) for s in range(3)]
    print("tuned plans", plans)
    a.step(wl.nsteps)
    got = (a.populations(), a.dipoles(), a.fields(B.MS_FIELD_E))
    a.close()
    o = CoupledOracle(wl).run(wl.nsteps)
    Eo = np.stack([o.f.Ex[0], o.f.Ey[0], o.f.Ez[0]])
    assert np.linalg.norm(got[2] - Eo) / np.linalg.norm(Eo) < 1e-4
    assert np.abs(got[0] - o.populations()).max() < 1e-5
    assert np.abs(got[1] - o.mu).max() < 1e-3 * np.abs(o.mu).max()
    b = B.Simulation(wl)
    for s, p in enumerate(plans):
        b.set_plan(s, *p)
    b.step(wl.nsteps)
    for x, y in zip(got, (b.populations(), b.dipoles(), b.fields(B.MS_FIELD_E))):
        assert np.array_equal(x, y)
    b.close()


def test_plan_validation(B):
    wl = W.custom("plan checks", 8, 8, 48, n_per_sim=5, species=[W.Species(nr=64, jmax=9)], layer=(20, 24),
                  nsteps=10)
    sim = B.Simulation(wl)
    for bad in ((B.MS_MOL_STREAMING, B.MS_KERN_POINT, 0),    # J = 9: no point-resident kernel
                (B.MS_MOL_STREAMING, B.MS_KERN_TILE, 32),    # J = 9: tiles of 8 points only
                (B.MS_MOL_STREAMING, B.MS_KERN_TILE, 16),
                (B.MS_MOL_STREAMING, B.MS_KERN_PAIR, 16),    # J = 9: two points a thread on 8-point tiles
                (B.MS_MOL_STREAMING, B.MS_KERN_CHUNK, 12),   # not a chunk width
                (B.MS_MOL_STREAMING, B.MS_KERN_CHUNK, 8, 1),  # a grid for a kernel that has none
                (7, B.MS_KERN_CHUNK, 8)):
        with pytest.raises(B.MSError) as e:
            sim.set_plan(0, *bad)
        assert e.value.code == B.MS_EINVAL
    sim.set_plan(0, B.MS_MOL_STREAMING, B.MS_KERN_DEFAULT, 0)
    sim.step(2)
    sim.close()


@pytest.mark.parametrize("nr,jmax,nmol", [(64, 6, 7), (128, 8, 5), (64, 10, 3)])
def test_tiled_plans_are_deterministic(B, nr, jmax, nmol):
    """Every tile width and grid of both tiled kernels, run twice from the
    same start: identical results bit for bit (the kernels' shared-memory
    regions, their tensor copies and the prefetch of the next molecule must
    not race)."""
    sp = W.Species(nr=nr, jmax=jmax, A=0.05)
    wl = W.custom("tiled determinism", 8, 8, 48, n_per_sim=nmol, species=[sp], layer=(20, 24),
                  seed=nr + jmax, nsteps=120)
    amp, wave = W.prescribed_drive(nmol, 120, wl.dt, E0=3e10, carrier_ev=6.0, fwhm=0.5e-15, t0=0.4e-15)
    kt = [(B.MS_KERN_TILE, t) for t in ((8,) if jmax >= 9 else (32, 16))]
    kt += [(B.MS_KERN_PAIR, t) for t in ((8,) if jmax >= 9 else ((16, 8) if jmax >= 5 else (32, 16)))]
    for k, t in kt:
        for g in (0, 1, -1):
            runs = []
            for _ in range(2):
                sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED, mol_path=B.MS_MOL_STREAMING)
                sim.set_plan(0, B.MS_MOL_STREAMING, k, t, g)
                sim.set_prescribed(amp, wave)
                sim.step(wl.nsteps)
                runs.append((sim.populations(), sim.dipoles()))
                sim.close()
            assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1]), (k, t, g)
