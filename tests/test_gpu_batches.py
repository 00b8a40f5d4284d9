"""The pipelined molecular step (ms_set_mol_batches): each streaming
species cut into runs whose kinetic and R-space passes overlap on two
streams.  Every molecule gets the same kernels on the same data, so every
batching must reproduce the sequential step bit for bit: eager and
graph-replayed, with several species, layouts and kernels, through the
allocation-free entry point, and with phase timing on."""
import numpy as np
import pytest

import workloads as W

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


def _workload(nsteps=48):
    # point-resident (J 1), tiled (J 4 at N_r 128: streaming), pair (J 6) species, coupled to the grid
    species = [W.species_config0(jmax=1), W.Species(nr=128, jmax=4, A=0.05), W.Species(nr=64, jmax=6)]
    return W.custom("batches", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 1e-15]], layer=(22, 26),
                    n_per_sim=157, species=species, fractions=[0.4, 0.3, 0.3], seed=41, nsteps=nsteps)


def _run(B, wl, batches, graphs=True, path=None, noalloc=False, timing=False):
    kw = {} if path is None else {"mol_path": path}
    sim = B.Simulation(wl, step_graphs=B.MS_GRAPHS_AUTO if graphs else B.MS_GRAPHS_OFF, **kw)
    sim.set_batches(batches)
    assert sim.batches == batches
    if timing:
        sim.timing_begin()
    if noalloc:
        for _ in range(wl.nsteps // 16):
            assert B.LIB.ms_step_noalloc(sim.h, 16) == B.MS_OK
    else:
        sim.step(wl.nsteps)
    ph = sim.timing_end() if timing else None
    out = (sim.fields(B.MS_FIELD_E), sim.fields(B.MS_FIELD_H), sim.populations(), sim.dipoles(),
           sim.dissociation()[0])
    sim.close()
    return out, ph


def _same(a, b, what):
    for x, y in zip(a, b):
        assert np.array_equal(x, y), what


@pytest.mark.parametrize("graphs", [True, False])
def test_batches_reproduce_sequential_step(B, graphs):
    wl = _workload()
    ref, _ = _run(B, wl, 0, graphs)
    assert np.abs(ref[3]).max() > 0.0 and ref[2][:, 1].max() > 0.0   # the molecules responded
    for nb in (1, 2, 3, 7):
        got, _ = _run(B, wl, nb, graphs)
        _same(got, ref, (nb, graphs))


def test_batches_with_fused_species_and_noalloc(B):
    wl = _workload(nsteps=32)
    ref, _ = _run(B, wl, 0, path=B.MS_MOL_STREAMING)
    got, _ = _run(B, wl, 4, path=B.MS_MOL_STREAMING, noalloc=True)
    _same(got, ref, "noalloc")
    ref, _ = _run(B, wl, 0, path=B.MS_MOL_AUTO)     # J <= 4 at N_r 128 runs fused
    got, _ = _run(B, wl, 2, path=B.MS_MOL_AUTO)
    _same(got, ref, "auto layout")


def test_batches_with_phase_timing(B):
    wl = _workload(nsteps=16)
    ref, _ = _run(B, wl, 0)
    got, ph = _run(B, wl, 2, timing=True)
    _same(got, ref, "timed")
    phases, nsteps, launches = ph
    assert nsteps == 16 and phases[1] > 0.0 and launches > 16 * 4


def test_batches_validation(B):
    wl = _workload(nsteps=4)
    sim = B.Simulation(wl)
    for bad in (-1, 17):
        assert B.LIB.ms_set_mol_batches(sim.h, bad) == B.MS_EINVAL
    assert sim.batches == 0
    sim.set_batches(16)
    sim.step(2)
    sim.set_batches(0)
    sim.step(2)
    assert sim.steps == 4
    sim.close()
