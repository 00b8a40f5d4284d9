"""ms_step_noalloc (the allocation-free stepping entry point) against ms_step.

Two identical handles in the streaming form: one advanced with ms_step (its
scratch comes from the handle), the other with ms_step_noalloc (its scratch is
the library's fixed device array).  Two calls in a row are compared, so the
second call starts from the contents the first left in the shared array.
Tolerances are the coupled parity tolerances: fields relative L2 <= 1e-4,
populations absolute <= 1e-5, dipoles 1e-3 of their largest magnitude.
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


def _workload(n_per_sim):
    return W.custom("no-alloc coupled", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 2e-15]],
                    layer=(22, 26), n_per_sim=n_per_sim, species=[W.Species(nr=128, jmax=4)],
                    seed=11, nsteps=240)


def test_noalloc_matches_step_two_calls(B):
    wl = _workload(300)
    ref = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    nal = B.Simulation(wl, mol_path=B.MS_MOL_STREAMING)
    for call in range(2):
        ref.step(120)
        code = B.LIB.ms_step_noalloc(nal.h, 120)
        assert code == B.MS_OK, B.LIB.ms_status_string(code).decode()
        assert nal.steps == ref.steps == 120 * (call + 1)
        E, Er = nal.fields(B.MS_FIELD_E), ref.fields(B.MS_FIELD_E)
        H, Hr = nal.fields(B.MS_FIELD_H), ref.fields(B.MS_FIELD_H)
        P, Pr = nal.populations(), ref.populations()
        mu, mur = nal.dipoles(), ref.dipoles()
        assert np.isfinite(E).all() and np.isfinite(P).all()
        assert _rel(E, Er) < 1e-4 and _rel(H, Hr) < 1e-4
        assert np.abs(P - Pr).max() < 1e-5
        assert np.abs(mu - mur).max() <= 1e-3 * max(np.abs(mur).max(), 1e-300)
        # the molecules have responded to the pulse by the second call
        if call == 1:
            assert np.abs(mur).max() > 0.0
    ref.close()
    nal.close()


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
