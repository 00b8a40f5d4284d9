"""ms_step_noalloc (the allocation-free stepping entry point) against ms_step.

Some callers cannot allocate device memory at the point where they step: code
running inside a fixed memory arena, or under a budget that forbids new
device allocations once a run has started.  ms_step_noalloc serves them: the
(T - 1)s scratch of the streaming form comes from a fixed device array
compiled into the library, one region per streaming species, instead of from
the handle's buffer.

Identical handles are advanced with ms_step (scratch from the handle) and
ms_step_noalloc (scratch from the library's array), and compared after every
call, so later calls start from the contents earlier ones left in the shared
array.  Covered: two calls in a row; two streaming species of different
sizes, whose regions must not overlap; calls interleaved with ms_step's
graph replay on the same handle; no allocator callback and no change of the
device's free memory during a call; the size limit.  Tolerances are the
coupled parity tolerances: fields relative L2 <= 1e-4, populations absolute
<= 1e-5, dipoles 1e-3 of their largest magnitude.
"""
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


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _workload(n_per_sim, species=None, fractions=None):
    return W.custom("no-alloc coupled", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 2e-15]],
                    layer=(22, 26), n_per_sim=n_per_sim, species=species or [W.Species(nr=128, jmax=4)],
                    fractions=fractions, seed=11, nsteps=240)


def _same(B, a, b):
    E, Er = a.fields(B.MS_FIELD_E), b.fields(B.MS_FIELD_E)
    H, Hr = a.fields(B.MS_FIELD_H), b.fields(B.MS_FIELD_H)
    P, Pr = a.populations(), b.populations()
    mu, mur = a.dipoles(), b.dipoles()
    assert np.isfinite(E).all() and np.isfinite(P).all()
    assert _rel(E, Er) < 1e-4 and _rel(H, Hr) < 1e-4
    assert np.abs(P - Pr).max() < 1e-5
    assert np.abs(mu - mur).max() <= 1e-3 * max(np.abs(mur).max(), 1e-300)
    return mur


def _noalloc(B, sim, n):
    code = B.LIB.ms_step_noalloc(sim.h, n)
    assert code == B.MS_OK, B.LIB.ms_status_string(code).decode()


def test_noalloc_matches_step_two_calls(B):
    wl = _workload(300)
    ref = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    nal = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    for call in range(2):
        ref.step(120)
        _noalloc(B, nal, 120)
        assert nal.steps == ref.steps == 120 * (call + 1)
        mur = _same(B, nal, ref)
        if call == 1:  # the molecules have responded to the pulse by the second call
            assert np.abs(mur).max() > 0.0
    ref.close()
    nal.close()


def test_noalloc_two_streaming_species_keep_their_own_regions(B):
    """Stage 1 of every species runs before stage 2 of any: with one shared
    region the second species' (T - 1)s would overwrite the first's."""
    species = [W.Species(nr=64, jmax=1), W.Species(nr=128, jmax=4)]
    wl = _workload(300, species=species, fractions=[0.5, 0.5])
    ref = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    nal = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    assert nal.species_path(0) == nal.species_path(1) == B.MS_MOL_STREAMING
    for call in range(2):
        ref.step(120)
        _noalloc(B, nal, 120)
        _same(B, nal, ref)
    ref.close()
    nal.close()


def test_noalloc_interleaved_with_graph_replay(B):
    """noalloc, then ms_step (whose replayed graph holds the handle's own
    scratch), then noalloc again, equals ms_step throughout."""
    wl = _workload(200)
    ref = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    mix = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    ref.step(48)
    _noalloc(B, mix, 16)
    mix.step(16)
    _noalloc(B, mix, 16)
    assert mix.steps == ref.steps == 48
    _same(B, mix, ref)
    ref.close()
    mix.close()


class _CountingAllocator:
    """PyTorch's caching allocator behind the library's callbacks, counting
    every request and release."""

    def __init__(self, B):
        inner = B._TorchAllocator()
        self.inner = inner
        self.calls = 0
        self.c_alloc = B._ALLOC(self._alloc)
        self.c_free = B._FREE(self._free)

    def _alloc(self, n, ctx):
        self.calls += 1
        return self.inner._alloc(n, ctx)

    def _free(self, p, ctx):
        self.calls += 1
        self.inner._free(p, ctx)


def test_noalloc_allocates_nothing(B):
    import torch
    wl = _workload(300)
    counter = _CountingAllocator(B)
    nal = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING, allocator=counter)
    ref = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    assert counter.calls > 0                 # create did use the allocator
    before = counter.calls
    _noalloc(B, nal, 8)                      # first call: loads the kernels if needed
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _noalloc(B, nal, 8)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert counter.calls == before           # no allocator callback in either call
    assert free1 == free0                    # and no device memory taken otherwise
    ref.step(16)
    _same(B, nal, ref)
    nal.close()
    ref.close()


def test_noalloc_rejects_scratch_beyond_limit(B):
    # 2 * 25 rotational rows * 128 points * 8 bytes = 51,200 bytes per molecule:
    # 1,400 molecules need 71.7 MB, above the 64 MiB array.
    wl = _workload(1400)
    sim = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    code = B.LIB.ms_step_noalloc(sim.h, 1)
    assert code == B.MS_EINVAL
    assert sim.steps == 0
    sim.step(1)  # the handle stays usable through ms_step
    assert sim.steps == 1
    sim.close()


def test_noalloc_limit_counts_every_streaming_species(B):
    # two species of 700 molecules each, 35.8 MB apiece: each fits alone,
    # together they do not
    species = [W.Species(nr=128, jmax=4), W.Species(nr=128, jmax=4, A=0.2)]
    wl = _workload(1400, species=species, fractions=[0.5, 0.5])
    sim = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    assert B.LIB.ms_step_noalloc(sim.h, 1) == B.MS_EINVAL
    assert sim.steps == 0
    sim.close()
