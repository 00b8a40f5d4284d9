"""Host-side descriptor validation of ms_create (runs before any device
call, so it needs no GPU): invalid inputs return MS_EINVAL, valid inputs on
a machine without an sm_103 device return MS_EUNSUPPORTED, never a crash."""
import ctypes as C

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def B():
    from paper_2209_04487_gb300 import build
    build.build()
    from paper_2209_04487_gb300 import binding
    return binding


def _create(B, wl, mutate=None):
    keep = []
    src = np.ascontiguousarray(wl.src, np.float64)
    g = B.GridDesc(wl.nx, wl.ny, wl.nz, wl.nsim, wl.dx, wl.dt, wl.pml, B.MS_BC_PML, wl.src_k,
                   src.ctypes.data_as(C.POINTER(C.c_double)), B.MS_SRC_PULSE)
    eps = np.array([m[0] for m in wl.materials])
    wp = np.array([m[1] for m in wl.materials])
    ga = np.array([m[2] for m in wl.materials])
    mid = np.ascontiguousarray(wl.mat_id)
    keep += [src, eps, wp, ga, mid]
    m = B.MaterialsDesc(len(eps), eps.ctypes.data_as(C.POINTER(C.c_double)),
                        wp.ctypes.data_as(C.POINTER(C.c_double)),
                        ga.ctypes.data_as(C.POINTER(C.c_double)),
                        mid.ctypes.data_as(C.POINTER(C.c_uint8)))
    sp = (B.SpeciesDesc * 1)(B.species_desc(wl.species[0]))
    sid = np.ascontiguousarray(wl.species_id)
    simid = np.ascontiguousarray(wl.sim_id)
    pos = np.ascontiguousarray(wl.pos)
    q = np.ascontiguousarray(wl.quat)
    keep += [sp, sid, simid, pos, q]
    d = B.MoleculesDesc(1, sp, wl.n_molecules, sid.ctypes.data_as(C.POINTER(C.c_int32)),
                        simid.ctypes.data_as(C.POINTER(C.c_int32)),
                        pos.ctypes.data_as(C.POINTER(C.c_double)), q.ctypes.data_as(C.POINTER(C.c_double)))
    o = B.Options()
    o.drive = B.MS_DRIVE_FDTD
    o.mol_substeps = 1
    if mutate:
        mutate(g, m, d, o, keep)
    h = C.c_void_p()
    rc = B.LIB.ms_create(C.byref(g), C.byref(m), C.byref(d), C.byref(o), C.byref(h))
    if rc == B.MS_OK:
        B.LIB.ms_destroy(h)
    return rc


def _wl():
    return W.custom("v", 8, 8, 48, src_k=14, layer=(20, 24), n_per_sim=5, nsteps=10)


@pytest.mark.parametrize("precision", ["fp32", "mixed", "cw_substeps", "bloch"])
def test_valid_descriptor_reaches_the_device_check(B, precision):
    import torch

    def mutate(g, m, d, o, keep):
        o.precision = B.MS_PREC_MIXED_F16X3 if precision == "mixed" else B.MS_PREC_FP32
        if precision == "cw_substeps":
            g.src_kind = B.MS_SRC_CW
            o.mol_substeps = 40
        if precision == "bloch":       # the wavepacket fields are ignored, even invalid ones
            d.species[0].model = B.MS_MODEL_BLOCH
            d.species[0].bloch_w0_eV = 1.5
            d.species[0].bloch_T2_s = 1e-14
            d.species[0].nr = 100
    rc = _create(B, _wl(), mutate)
    if torch.cuda.is_available():
        assert rc == B.MS_OK
    else:
        assert rc == B.MS_EUNSUPPORTED


@pytest.mark.parametrize("what", ["courant", "nx", "pml", "src_in_pml", "material_id", "species_nr",
                                  "jmax", "position", "quaternion", "precision_unknown", "mixed_fused",
                                  "mixed_nr256", "alloc_half", "src_kind", "cw_turn_on", "substeps_negative",
                                  "substeps_huge", "model_unknown", "bloch_w0", "bloch_T1", "dipole_R_nan",
                                  "dipole_R_jmax", "dipole_R_parity"])
def test_invalid_descriptors_are_rejected(B, what):
    def mutate(g, m, d, o, keep):
        if what == "courant":
            g.dt_s = g.dx_m / 299792458.0
        elif what == "nx":
            g.nx = 0
        elif what == "pml":
            g.pml_cells = 30
        elif what == "src_in_pml":
            g.src_plane_z = 5
        elif what == "material_id":
            bad = np.full(8 * 8 * 48, 7, np.uint8)
            keep.append(bad)
            m.material_id = bad.ctypes.data_as(C.POINTER(C.c_uint8))
        elif what == "species_nr":
            d.species[0].nr = 100
        elif what == "jmax":
            d.species[0].jmax = 20
        elif what == "position":
            p = np.array(np.ctypeslib.as_array(d.pos_m, shape=(3 * d.n_molecules,)))
            p[2] = 1.0
            keep.append(p)
            d.pos_m = p.ctypes.data_as(C.POINTER(C.c_double))
        elif what == "quaternion":
            qz = np.zeros(4 * d.n_molecules)
            keep.append(qz)
            d.orient = qz.ctypes.data_as(C.POINTER(C.c_double))
        elif what == "precision_unknown":
            o.precision = 7
        elif what == "mixed_fused":
            o.precision = B.MS_PREC_MIXED_F16X3
            o.mol_path = B.MS_MOL_FUSED
        elif what == "mixed_nr256":
            o.precision = B.MS_PREC_MIXED_F16X3
            d.species[0].nr = 256
        elif what == "alloc_half":
            o.alloc = B._ALLOC(lambda n, c: None)
        elif what == "src_kind":
            g.src_kind = 2
        elif what == "cw_turn_on":
            g.src_kind = B.MS_SRC_CW
            bad = np.array([1e9, 1.5, 0.0, 0.0])
            keep.append(bad)
            g.src = bad.ctypes.data_as(C.POINTER(C.c_double))
        elif what == "substeps_negative":
            o.mol_substeps = -1
        elif what == "substeps_huge":
            o.mol_substeps = 1 << 20
        elif what in ("dipole_R_nan", "dipole_R_jmax", "dipole_R_parity"):
            tab = np.full(d.species[0].nr, 1.0)
            if what == "dipole_R_nan":
                tab[3] = np.nan
            elif what == "dipole_R_jmax":
                d.species[0].jmax = 5
            else:
                o.state_form = B.MS_STATE_PARITY
            keep.append(tab)
            d.species[0].dipole_R = tab.ctypes.data_as(C.POINTER(C.c_double))
        elif what == "model_unknown":
            d.species[0].model = 5
        elif what == "bloch_w0":
            d.species[0].model = B.MS_MODEL_BLOCH
            d.species[0].bloch_w0_eV = -1.0
        elif what == "bloch_T1":
            d.species[0].model = B.MS_MODEL_BLOCH
            d.species[0].bloch_w0_eV = 1.0
            d.species[0].bloch_T1_s = float("nan")
    rc = _create(B, _wl(), mutate)
    expect = {"species_nr": B.MS_EUNSUPPORTED, "jmax": B.MS_EUNSUPPORTED,
              "mixed_fused": B.MS_EUNSUPPORTED, "mixed_nr256": B.MS_EUNSUPPORTED,
              "dipole_R_jmax": B.MS_EUNSUPPORTED, "dipole_R_parity": B.MS_EUNSUPPORTED}.get(what, B.MS_EINVAL)
    assert rc == expect, (what, rc)


def test_null_handles(B):
    assert B.LIB.ms_step(None, 1) == B.MS_EINVAL
    assert B.LIB.ms_step_noalloc(None, 1) == B.MS_EINVAL
    assert B.LIB.ms_read_populations(None, 0, 0, None, None) == B.MS_EINVAL
    assert B.LIB.ms_set_prescribed_field(None, None, None, 1) == B.MS_EINVAL
    assert B.LIB.ms_set_replay_field(None, None, 1) == B.MS_EINVAL
    assert B.LIB.ms_record_local_fields(None, None, 1, None, 1) == B.MS_EINVAL
    assert B.LIB.ms_save(None, b"unused.ck") == B.MS_EINVAL
    assert B.LIB.ms_load(None, b"unused.ck") == B.MS_EINVAL
    assert B.LIB.ms_timing_begin(None) == B.MS_EINVAL
    assert B.LIB.ms_step_count(None) == -1
    B.LIB.ms_destroy(None)
