"""Determinism, checkpoint/resume and field record/replay, through the C ABI.

The coupled step has no atomics (the polarization scatter is a CSR segmented
sum, the molecular reductions run in a fixed order), so repeated runs, a
resumed run and a replayed molecular run are compared bit for bit.
"""
import ctypes

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


def _slab(nx, ny, nz):
    m = np.zeros((nz, ny, nx), np.uint8)
    m[30:] = W.configs.MAT_GLASS
    m[27:30, ny // 4:3 * ny // 4, nx // 4:3 * nx // 4] = W.configs.MAT_SILVER
    return m


def _workload(n_per_sim=120, nsim=2):
    """Two simulations (metal, glass, CPML, TF/SF) with two species."""
    species = [W.species_config0(jmax=1), W.Species(nr=64, jmax=2, A=0.05)]
    return W.custom("state", 16, 16, 48, nsim=nsim, src_k=14,
                    pulses=[[2e10, 1.5498, 2e-15, 2e-15], [1.5e10, 1.2, 2e-15, 2.5e-15]][:nsim],
                    geometry=_slab, layer=(20, 24), n_per_sim=n_per_sim, species=species,
                    fractions=[0.6, 0.4], seed=9, nsteps=240)


def _snapshot(B, sim, nsim):
    out = {"P": sim.populations(), "mu": sim.dipoles(), "abs": sim.dissociation()[0]}
    for s in range(nsim):
        out[f"E{s}"] = sim.fields(B.MS_FIELD_E, s)
        out[f"H{s}"] = sim.fields(B.MS_FIELD_H, s)
    return out


def _assert_identical(a, b):
    assert a.keys() == b.keys()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_two_runs_are_bitwise_identical(B):
    wl = _workload()
    runs = []
    for _ in range(2):
        sim = B.Simulation(wl)
        sim.step(160)
        runs.append(_snapshot(B, sim, wl.nsim))
        sim.close()
    _assert_identical(*runs)
    assert np.abs(runs[0]["mu"]).max() > 0.0  # the pulse reached the molecules


def test_checkpoint_resume_is_bitwise(B, tmp_path):
    wl = _workload()
    planes, omega = [12, 40], [1.5e15, 2.35e15, 3.0e15]
    ref = B.Simulation(wl)
    ref.set_detectors(planes, omega)
    ref.step(160)
    want = _snapshot(B, ref, wl.nsim)
    want["flux"] = np.stack([ref.flux(d) for d in range(2)])
    ref.close()

    first = B.Simulation(wl)
    first.set_detectors(planes, omega)
    first.step(80)
    path = str(tmp_path / "half.ck")
    first.save(path)
    first.close()

    resumed = B.Simulation(wl)
    resumed.set_detectors(planes, omega)   # same detector layout before loading
    resumed.load(path)
    assert resumed.steps == 80
    resumed.step(80)
    assert resumed.steps == 160
    got = _snapshot(B, resumed, wl.nsim)
    got["flux"] = np.stack([resumed.flux(d) for d in range(2)])
    _assert_identical(want, got)
    resumed.close()


def test_checkpoint_rejects_mismatch_and_garbage(B, tmp_path):
    wl = _workload()
    sim = B.Simulation(wl)
    sim.step(3)
    path = str(tmp_path / "a.ck")
    sim.save(path)
    other = B.Simulation(_workload(n_per_sim=100))
    with pytest.raises(B.MSError) as e:
        other.load(path)
    assert e.value.code == B.MS_EINVAL
    junk = tmp_path / "junk.ck"
    junk.write_bytes(b"not a checkpoint" * 64)
    with pytest.raises(B.MSError) as e:
        sim.load(str(junk))
    assert e.value.code == B.MS_EIO
    with pytest.raises(B.MSError) as e:
        sim.load(str(tmp_path / "missing.ck"))
    assert e.value.code == B.MS_EIO
    # a truncated file
    data = open(path, "rb").read()
    (tmp_path / "short.ck").write_bytes(data[: len(data) // 2])
    with pytest.raises(B.MSError) as e:
        sim.load(str(tmp_path / "short.ck"))
    assert e.value.code == B.MS_EIO
    # the handle still works, and its own checkpoint still loads
    sim.load(path)
    assert sim.steps == 3
    sim.step(2)
    other.close()
    sim.close()


def test_record_and_replay_reproduce_the_coupled_molecules(B):
    wl = _workload(nsim=1)
    n = 160
    coupled = B.Simulation(wl)
    rec = coupled.record_local_fields(np.arange(wl.n_molecules), n)
    assert rec.shape == (n, wl.n_molecules, 3)
    assert np.isfinite(rec).all() and np.abs(rec).max() > 0.0
    assert coupled.steps == n
    want = {"P": coupled.populations(), "mu": coupled.dipoles(), "abs": coupled.dissociation()[0]}
    coupled.close()

    replay = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED)
    replay.set_replay(rec)
    replay.step(n)
    got = {"P": replay.populations(), "mu": replay.dipoles(), "abs": replay.dissociation()[0]}
    _assert_identical(want, got)
    # one step beyond the replayed samples is refused
    with pytest.raises(B.MSError) as e:
        replay.step(1)
    assert e.value.code == B.MS_EINVAL
    replay.close()


def test_record_rejects_bad_ids(B):
    wl = _workload(nsim=1)
    sim = B.Simulation(wl)
    with pytest.raises(B.MSError) as e:
        sim.record_local_fields(np.array([0, wl.n_molecules]), 2)
    assert e.value.code == B.MS_EINVAL
    assert sim.steps == 0
    sim.close()


def _run(B, wl, graphs, plan, drive=None, prescribed=None, detectors=None):
    kw = {} if drive is None else {"drive": drive}
    sim = B.Simulation(wl, step_graphs=B.MS_GRAPHS_AUTO if graphs else B.MS_GRAPHS_OFF, **kw)
    if prescribed is not None:
        sim.set_prescribed(*prescribed)
    for item in plan:
        if item == "detectors":
            sim.set_detectors(*detectors)
        else:
            sim.step(item)
    out = _snapshot(B, sim, wl.nsim) if drive is None else {"P": sim.populations(), "mu": sim.dipoles()}
    if detectors is not None and drive is None:
        out["flux"] = sim.flux(0)
    sim.close()
    return out


@pytest.mark.parametrize("N", [1, 3])
def test_graph_replay_is_bitwise_identical_to_eager(B, N):
    """Cycles replayed from a captured CUDA graph give the eager result bit
    for bit: step counts that start and end mid-cycle, sub-stepping, and a
    detector change between calls (which forces a new capture)."""
    import dataclasses
    wl = dataclasses.replace(_workload(nsim=2), mol_substeps=N)
    planes = ([12, 40], [1.5e15, 2.35e15])
    plan = [5, 37, "detectors", 29, 1, 40]
    a = _run(B, wl, True, plan, detectors=planes)
    b = _run(B, wl, False, plan, detectors=planes)
    _assert_identical(a, b)
    assert np.abs(a["mu"]).max() > 0.0


def test_graph_replay_prescribed_recaptures_after_new_drive(B):
    wl = _workload(nsim=1)
    n = wl.n_molecules
    amp, wave = W.prescribed_drive(n, 200, wl.dt, E0=3e10, carrier_ev=6.0, fwhm=0.5e-15, t0=0.3e-15)

    def run(graphs):
        sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED,
                           step_graphs=B.MS_GRAPHS_AUTO if graphs else B.MS_GRAPHS_OFF)
        sim.set_prescribed(amp, wave)
        sim.step(64)
        sim.set_prescribed(amp * 0.5, wave)   # new arrays: the captured graph is stale
        sim.step(100)
        out = {"P": sim.populations(), "mu": sim.dipoles()}
        sim.close()
        return out
    _assert_identical(run(True), run(False))


_C = ctypes


class _CkHeader(ctypes.Structure):
    """The checkpoint header of csrc/ms_api.cu (version 4), for reading a
    saved state on the host."""
    _fields_ = [("magic", _C.c_char * 8), ("version", _C.c_uint32), ("drive", _C.c_uint32),
                ("steps", _C.c_int64), ("nx", _C.c_int32), ("ny", _C.c_int32), ("nz", _C.c_int32),
                ("nsim", _C.c_int32), ("nmol", _C.c_int64), ("nspecies", _C.c_int32), ("pml", _C.c_int32),
                ("ks", _C.c_int32), ("jk0", _C.c_int32), ("jk1", _C.c_int32), ("aux_len", _C.c_int32),
                ("ndet", _C.c_int32), ("nfreq", _C.c_int32), ("state_rows", _C.c_int32 * 8),
                ("mol_substeps", _C.c_int32), ("src_kind", _C.c_int32), ("species", _C.c_int32 * 24),
                ("nblobs", _C.c_uint64)]


def test_population_sums_equal_fp64_sums_of_the_state(B, tmp_path):
    """The per-molecule populations are compensated FP32 sums (TwoSum from the
    first term on, about 48 bits; FP64 at the store) of the FP32 products
    |s|^2 = fma(x, x, y y).  Read the state itself from a checkpoint and sum
    the same FP32 products in FP64 on the host: the two agree to 1e-11
    relative, so the compensated sums stand in for FP64 accumulation.  (The
    products' own rounding, 2^-24 per element, is common to both.)"""
    sp = W.Species(nr=128, jmax=4, A=0.05)
    n = 40
    wl = W.custom("fp64 sums", 8, 8, 48, n_per_sim=n, species=[sp], layer=(20, 24), seed=17, nsteps=300)
    amp, wave = W.prescribed_drive(n, 300, wl.dt, E0=3e10, carrier_ev=6.0, fwhm=0.5e-15, t0=0.5e-15)
    for path, kern in ((B.MS_MOL_FUSED, None), (B.MS_MOL_STREAMING, None), (B.MS_MOL_STREAMING, B.MS_KERN_PAIR)):
        sim = B.Simulation(wl, drive=B.MS_DRIVE_PRESCRIBED, mol_path=path)
        if kern is not None:   # the two-points-a-thread kernel sums point pairs
            sim.set_plan(0, path, kern, 0)
        sim.set_prescribed(amp, wave)
        sim.step(300)
        P = sim.populations()
        ck = str(tmp_path / f"state{path}_{kern}.ck")
        sim.save(ck)
        sim.close()
        raw = open(ck, "rb").read()
        h = _CkHeader.from_buffer_copy(raw)
        assert h.version == 4 and h.nspecies == 1 and h.nmol == n
        off = ctypes.sizeof(_CkHeader)
        nb = int(np.frombuffer(raw, np.uint64, 1, off)[0])        # first blob: the species' state
        rows = 2 * sp.nrot
        assert nb == n * rows * sp.nr * 8
        st = np.frombuffer(raw, np.float32, 2 * n * rows * sp.nr, off + 8).reshape(n, 2, sp.nrot, sp.nr, 2)
        x, y = st[..., 0].astype(np.float64), st[..., 1].astype(np.float64)
        yy = (st[..., 1] * st[..., 1]).astype(np.float64)           # FP32 product, rounded
        p32 = (x * x + yy).astype(np.float32).astype(np.float64)     # fma(x, x, yy): x*x exact in FP64
        dR = np.float64(np.float32((sp.rmax - sp.rmin) / (sp.nr - 1)))  # the kernels' FP32 grid step
        P64 = p32.sum(axis=(2, 3)) * dR
        exact = (x * x + y * y).sum(axis=(2, 3)) * dR
        # molecule order: the state is stored by species, in molecule-id order within it
        rel = np.abs(P - P64) / np.maximum(P64, 1e-300)
        rel_exact = np.abs(P - exact) / np.maximum(exact, 1e-300)
        print(f"layout {path} kernel {kern}: populations vs FP64 sums of the FP32 products {rel.max():.2e}, "
              f"vs the exact norms of the stored state {rel_exact.max():.2e}")
        assert P[:, 1].max() > 1e-6
        assert rel.max() < 1e-11
        assert rel_exact.max() < 1e-7


def test_parity_reduced_pair_kernel_state_paths(B, tmp_path):
    """The parity-reduced rows on the two-points-a-thread kernel (J = 6 and
    J = 9 species, coupled to the grid) through the paths that move or
    replay the state: eager stepping equals graph replay and the pipelined
    step bit for bit, and a checkpoint taken halfway resumes to the same
    result."""
    species = [W.Species(nr=64, jmax=6, A=0.05), W.Species(nr=64, jmax=9)]
    wl = W.custom("parity state", 16, 16, 48, src_k=14, pulses=[[2e10, 1.5498, 2e-15, 1e-15]],
                  layer=(22, 26), n_per_sim=90, species=species, fractions=[0.5, 0.5], seed=21, nsteps=96)

    def run(graphs, batches=0, split=None):
        sim = B.Simulation(wl, state_form=B.MS_STATE_PARITY,
                           step_graphs=B.MS_GRAPHS_AUTO if graphs else B.MS_GRAPHS_OFF)
        assert sim.species_path(0) == sim.species_path(1) == B.MS_MOL_STREAMING
        sim.set_batches(batches)
        if split is None:
            sim.step(wl.nsteps)
        else:
            sim.step(split)
            path = str(tmp_path / "parity.ck")
            sim.save(path)
            sim.close()
            sim = B.Simulation(wl, state_form=B.MS_STATE_PARITY)
            sim.load(path)
            sim.step(wl.nsteps - split)
        out = _snapshot(B, sim, wl.nsim)
        sim.close()
        return out

    ref = run(False)
    assert np.abs(ref["mu"]).max() > 0.0 and ref["P"][:, 1].max() > 0.0
    _assert_identical(ref, run(True))
    _assert_identical(ref, run(True, batches=3))
    _assert_identical(ref, run(False, split=40))
