"""Failure detection on the GPU without faulting it: allocator failure,
a non-finite field, a bounded wait that runs out.  Every case ends in a
status code and leaves the context usable."""
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


def _wl():
    return W.custom("faults", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 2e-15]],
                    layer=(22, 26), n_per_sim=40, species=[W.species_config0(jmax=1)], seed=2,
                    nsteps=50)


def _failing_allocator(B, fail_at):
    """PyTorch-backed allocator whose fail_at-th request fails."""
    class Failing(B._TorchAllocator):
        def __init__(self):
            super().__init__()
            self.calls = 0
            self.frees = 0

        def _alloc(self, n, ctx):
            self.calls += 1
            if self.calls == fail_at:
                return None
            return super()._alloc(n, ctx)

        def _free(self, p, ctx):
            self.frees += 1
            super()._free(p, ctx)
    return Failing()


@pytest.mark.parametrize("fail_at", [1, 5, 20])
def test_allocator_failure_is_enomem_and_leaks_nothing(B, fail_at):
    alloc = _failing_allocator(B, fail_at)
    with pytest.raises(B.MSError) as e:
        B.Simulation(_wl(), allocator=alloc)
    assert e.value.code == B.MS_ENOMEM
    assert alloc.calls == fail_at
    assert alloc.frees == fail_at - 1      # every block obtained was handed back
    assert not alloc.live
    sim = B.Simulation(_wl())              # the device is still usable
    sim.step(2)
    sim.close()


def test_non_finite_field_latches_enumeric(B):
    wl = _wl()
    sim = B.Simulation(wl)
    sim.step(1)
    E = sim.fields(B.MS_FIELD_E)
    nz, ny, nx = wl.nz, wl.ny, wl.nx
    c = np.floor(wl.pos[0] / wl.dx).astype(int)          # molecule 0's cell (x, y, z)
    E[0, c[2], c[1], c[0]] = np.nan
    sim.write_fields(B.MS_FIELD_E, 0, E)
    with pytest.raises(B.MSError) as e:
        sim.step(1)
        sim.populations()
    assert e.value.code == B.MS_ENUMERIC
    sim.close()
    fresh = B.Simulation(wl)
    fresh.step(2)
    assert np.isfinite(fresh.populations()).all()
    fresh.close()


def test_bounded_wait_runs_out_with_a_status(B):
    assert B.LIB.ms_check_bounded_wait(200) == B.MS_ETIMEOUT
    assert B.LIB.ms_check_bounded_wait(0) == B.MS_EINVAL
    sim = B.Simulation(_wl())   # the context is still usable
    sim.step(3)
    assert np.isfinite(sim.populations()).all()
    sim.close()
