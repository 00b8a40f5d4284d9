"""ctypes binding of include/ms.h (argument marshalling only).

Every step of the coupled time step runs in libms.so's CUDA kernels; this
module converts NumPy arrays into the C descriptors, hands PyTorch's caching
allocator and current stream to the library, and copies results back.  If the
library cannot be loaded the import of this module fails: there is no
Python or CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

MS_OK, MS_EINVAL, MS_ENOMEM, MS_ECUDA, MS_ENUMERIC, MS_ETIMEOUT, MS_EUNSUPPORTED, MS_EIO = 0, -1, -2, -3, -4, -5, -6, -7
MS_BC_PML, MS_BC_PERIODIC = 0, 1
MS_PREC_FP32, MS_PREC_MIXED_F16X3 = 0, 1
MS_DRIVE_FDTD, MS_DRIVE_PRESCRIBED = 0, 1
MS_FIELD_E, MS_FIELD_H = 0, 1
MS_STATE_FULL, MS_STATE_PARITY = 0, 1
MS_SRC_PULSE, MS_SRC_CW = 0, 1
MS_MODEL_WAVEPACKET, MS_MODEL_BLOCH = 0, 1
MS_GRAPHS_AUTO, MS_GRAPHS_OFF = 0, 1
MS_KERN_DEFAULT, MS_KERN_POINT, MS_KERN_TILE, MS_KERN_CHUNK, MS_KERN_PAIR = 0, 1, 2, 3, 4
MS_TUNE_OFF, MS_TUNE_MEASURE = 0, 1
MS_MOL_AUTO, MS_MOL_FUSED, MS_MOL_STREAMING = 0, 1, 2

_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class GridDesc(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("nsim", C.c_int32),
                ("dx_m", C.c_double), ("dt_s", C.c_double), ("pml_cells", C.c_int32),
                ("bc_z", C.c_int32), ("src_plane_z", C.c_int32), ("src", C.POINTER(C.c_double)),
                ("src_kind", C.c_int32)]


class MaterialsDesc(C.Structure):
    _fields_ = [("n_materials", C.c_int32), ("eps_inf", C.POINTER(C.c_double)),
                ("wp_eV", C.POINTER(C.c_double)), ("gamma_eV", C.POINTER(C.c_double)),
                ("material_id", C.POINTER(C.c_uint8))]


class SpeciesDesc(C.Structure):
    _fields_ = [("nr", C.c_int32), ("jmax", C.c_int32), ("rmin", C.c_double), ("rmax", C.c_double),
                ("mass_me", C.c_double), ("morse_De", C.c_double), ("morse_a", C.c_double),
                ("morse_re", C.c_double), ("exc_A", C.c_double), ("exc_B", C.c_double),
                ("exc_beta", C.c_double), ("exc_rc", C.c_double), ("dipole_ea0", C.c_double),
                ("absorber_r", C.c_double), ("absorber_power", C.c_double), ("model", C.c_int32),
                ("bloch_w0_eV", C.c_double), ("bloch_T1_s", C.c_double), ("bloch_T2_s", C.c_double),
                ("dipole_R", C.POINTER(C.c_double))]


class MoleculesDesc(C.Structure):
    _fields_ = [("n_species", C.c_int32), ("species", C.POINTER(SpeciesDesc)),
                ("n_molecules", C.c_int64), ("species_id", C.POINTER(C.c_int32)),
                ("sim_id", C.POINTER(C.c_int32)), ("pos_m", C.POINTER(C.c_double)),
                ("orient", C.POINTER(C.c_double))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("mol_substeps", C.c_int32), ("drive", C.c_int32),
                ("alloc", _ALLOC), ("free", _FREE), ("alloc_ctx", C.c_void_p), ("stream", C.c_void_p),
                ("mol_path", C.c_int32), ("state_form", C.c_int32), ("step_graphs", C.c_int32),
                ("autotune", C.c_int32)]


def _load() -> C.CDLL:
    path = _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_2209_04487_gb300.build.build() "
                          "(or __graft_entry__.build()) first")
    lib = C.CDLL(path)
    P = C.POINTER
    sig = {
        "ms_create": (C.c_int, [P(GridDesc), P(MaterialsDesc), P(MoleculesDesc), P(Options), P(C.c_void_p)]),
        "ms_step": (C.c_int, [C.c_void_p, C.c_int64]),
        "ms_step_count": (C.c_int64, [C.c_void_p]),
        "ms_step_noalloc": (C.c_int, [C.c_void_p, C.c_int64]),
        "ms_read_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, P(C.c_float), C.c_size_t]),
        "ms_write_fields": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, P(C.c_float), C.c_size_t]),
        "ms_read_populations": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, P(C.c_double), P(C.c_double)]),
        "ms_read_dissociation": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, P(C.c_double),
                                           P(C.c_double), P(C.c_double), P(C.c_double)]),
        "ms_read_dipoles": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, P(C.c_double)]),
        "ms_set_prescribed_field": (C.c_int, [C.c_void_p, P(C.c_float), P(C.c_float), C.c_int64]),
        "ms_set_replay_field": (C.c_int, [C.c_void_p, P(C.c_float), C.c_int64]),
        "ms_record_local_fields": (C.c_int, [C.c_void_p, P(C.c_int64), C.c_int64, P(C.c_float), C.c_int64]),
        "ms_save": (C.c_int, [C.c_void_p, C.c_char_p]),
        "ms_check_bounded_wait": (C.c_int, [C.c_int32]),
        "ms_species_path": (C.c_int32, [C.c_void_p, C.c_int32]),
        "ms_species_plan": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_int32), P(C.c_int32), P(C.c_int32)]),
        "ms_set_mol_batches": (C.c_int, [C.c_void_p, C.c_int32]),
        "ms_mol_batches": (C.c_int32, [C.c_void_p]),
        "ms_set_species_plan": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
        "ms_species_plan_ex": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_int32)]),
        "ms_set_species_plan_ex": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_int32)]),
        "ms_set_detectors": (C.c_int, [C.c_void_p, P(C.c_int32), C.c_int32, P(C.c_double), C.c_int32]),
        "ms_read_flux": (C.c_int, [C.c_void_p, C.c_int32, P(C.c_double)]),
        "ms_read_dft": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32, P(C.c_double)]),
        "ms_load": (C.c_int, [C.c_void_p, C.c_char_p]),
        "ms_device_bytes": (C.c_size_t, [C.c_void_p]),
        "ms_timing_begin": (C.c_int, [C.c_void_p]),
        "ms_timing_end": (C.c_int, [C.c_void_p, P(C.c_double), P(C.c_int64), P(C.c_int64)]),
        "ms_destroy": (None, [C.c_void_p]),
        "ms_status_string": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


LIB = _load()

# every symbol include/ms.h declares
EXPORTED = ("ms_create", "ms_step", "ms_step_noalloc", "ms_step_count", "ms_read_fields", "ms_write_fields",
            "ms_read_populations", "ms_read_dissociation", "ms_read_dipoles",
            "ms_set_prescribed_field", "ms_set_replay_field", "ms_record_local_fields", "ms_save", "ms_load",
            "ms_check_bounded_wait", "ms_species_path", "ms_species_plan", "ms_set_species_plan",
            "ms_species_plan_ex", "ms_set_species_plan_ex", "ms_set_mol_batches", "ms_mol_batches",
            "ms_set_detectors", "ms_read_flux", "ms_read_dft",
            "ms_timing_begin", "ms_timing_end", "ms_device_bytes",
            "ms_destroy", "ms_status_string")


class MSError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {LIB.ms_status_string(code).decode()} ({code})")
        self.code = code


def _check(code: int, what: str):
    if code != MS_OK:
        raise MSError(code, what)


def _ptr(a: Optional[np.ndarray], ct):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ct))


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, kept alive by reference."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.c_alloc = _ALLOC(self._alloc)
        self.c_free = _FREE(self._free)

    def _alloc(self, n, ctx):
        try:
            t = self.torch.empty(int(n), dtype=self.torch.uint8, device="cuda")
        except Exception:
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, p, ctx):
        self.live.pop(p, None)


def species_desc(sp) -> SpeciesDesc:
    bloch = getattr(sp, "model", "wavepacket") == "bloch"
    d = SpeciesDesc(sp.nr, sp.jmax, sp.rmin, sp.rmax, sp.mass, sp.De, sp.a, sp.re, sp.A, sp.B,
                    sp.beta, sp.rc, sp.dipole, sp.absorber_r, sp.absorber_power,
                    MS_MODEL_BLOCH if bloch else MS_MODEL_WAVEPACKET, sp.w0_ev, sp.T1, sp.T2)
    if getattr(sp, "dipole_R", None) is not None:
        tab = np.ascontiguousarray(sp.dipole_R, np.float64)
        d.dipole_R = tab.ctypes.data_as(C.POINTER(C.c_double))
        d._keep_dipole_R = tab      # alive as long as the descriptor
    return d


def mixed_supported(wl) -> bool:
    """Whether every wavepacket species of the workload can take the mixed kinetic pass."""
    return all(sp.nr in (64, 128) for sp in wl.species if getattr(sp, "model", "wavepacket") != "bloch")


class Simulation:
    """One coupled simulation on the current CUDA device (workload in the
    layout of ``workloads.Workload``)."""

    def __init__(self, wl, *, drive: int = MS_DRIVE_FDTD, precision: int = MS_PREC_FP32,
                 with_molecules: bool = True, use_torch: bool = True, stream=None,
                 mol_path: int = MS_MOL_AUTO, allocator=None, state_form: int = 0,
                 step_graphs: int = 0, autotune: int = 0):
        self.wl = wl
        self._keep = []
        src = np.ascontiguousarray(wl.src, np.float64) if wl.src_k >= 0 else None
        self._keep.append(src)
        g = GridDesc(wl.nx, wl.ny, wl.nz, wl.nsim, wl.dx, wl.dt, wl.pml,
                     MS_BC_PML if wl.bc_z == "pml" else MS_BC_PERIODIC, wl.src_k, _ptr(src, C.c_double),
                     MS_SRC_CW if wl.src_kind == "cw" else MS_SRC_PULSE)
        eps = np.array([m[0] for m in wl.materials], np.float64)
        wp = np.array([m[1] for m in wl.materials], np.float64)
        ga = np.array([m[2] for m in wl.materials], np.float64)
        mid = np.ascontiguousarray(wl.mat_id, np.uint8)
        self._keep += [eps, wp, ga, mid]
        m = MaterialsDesc(len(wl.materials), _ptr(eps, C.c_double), _ptr(wp, C.c_double),
                          _ptr(ga, C.c_double), _ptr(mid, C.c_uint8))
        nmol = wl.n_molecules if with_molecules else 0
        self.nmol = nmol
        descs = [species_desc(s) for s in wl.species]       # they keep any d(R) tables alive
        self._keep += descs
        sp_arr = (SpeciesDesc * max(1, len(wl.species)))(*descs)
        sid = np.ascontiguousarray(wl.species_id[:nmol], np.int32)
        simid = np.ascontiguousarray(wl.sim_id[:nmol], np.int32)
        pos = np.ascontiguousarray(wl.pos[:nmol], np.float64)
        quat = np.ascontiguousarray(wl.quat[:nmol], np.float64)
        self._keep += [sp_arr, sid, simid, pos, quat]
        d = MoleculesDesc(len(wl.species), sp_arr, nmol, _ptr(sid, C.c_int32), _ptr(simid, C.c_int32),
                          _ptr(pos, C.c_double), _ptr(quat, C.c_double))
        opts = Options()
        opts.precision = precision
        opts.mol_substeps = wl.mol_substeps
        opts.drive = drive
        opts.mol_path = mol_path
        opts.state_form = state_form
        opts.step_graphs = step_graphs
        opts.autotune = autotune
        self.stream = None
        if use_torch:
            import torch
            self._alloc = allocator if allocator is not None else _TorchAllocator()
            opts.alloc = self._alloc.c_alloc
            opts.free = self._alloc.c_free
            # a real (non-legacy-default) stream, so that torch events recorded
            # on self.stream order with the library's launches
            self.stream = stream if stream is not None else torch.cuda.Stream()
            opts.stream = C.c_void_p(self.stream.cuda_stream)
        else:
            self._alloc = None
            opts.alloc = _ALLOC()
            opts.free = _FREE()
            opts.stream = None
        h = C.c_void_p()
        _check(LIB.ms_create(C.byref(g), C.byref(m), C.byref(d), C.byref(opts), C.byref(h)), "ms_create")
        self.h = h

    # -- stepping ---------------------------------------------------------------
    def step(self, n: int = 1):
        _check(LIB.ms_step(self.h, int(n)), "ms_step")

    def step_noalloc(self, n: int = 1):
        """Same as step(), with the streaming scratch taken from the library's
        fixed device array; allocates nothing."""
        _check(LIB.ms_step_noalloc(self.h, int(n)), "ms_step_noalloc")

    @property
    def steps(self) -> int:
        return int(LIB.ms_step_count(self.h))

    def set_prescribed(self, amp: np.ndarray, wave: np.ndarray):
        a = np.ascontiguousarray(amp, np.float32)
        w = np.ascontiguousarray(wave, np.float32)
        _check(LIB.ms_set_prescribed_field(self.h, _ptr(a, C.c_float), _ptr(w, C.c_float), w.size),
               "ms_set_prescribed_field")

    # -- reads --------------------------------------------------------------------
    def fields(self, which: int = MS_FIELD_E, sim: int = 0) -> np.ndarray:
        n = self.wl.nx * self.wl.ny * self.wl.nz
        out = np.empty(3 * n, np.float32)
        _check(LIB.ms_read_fields(self.h, which, sim, _ptr(out, C.c_float), out.size), "ms_read_fields")
        return out.reshape(3, self.wl.nz, self.wl.ny, self.wl.nx)

    def write_fields(self, which: int, sim: int, arr: np.ndarray):
        a = np.ascontiguousarray(arr, np.float32).ravel()
        _check(LIB.ms_write_fields(self.h, which, sim, _ptr(a, C.c_float), a.size), "ms_write_fields")

    def populations(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        count = self.nmol - first if count is None else count
        pg = np.empty(count)
        pe = np.empty(count)
        _check(LIB.ms_read_populations(self.h, first, count, _ptr(pg, C.c_double), _ptr(pe, C.c_double)),
               "ms_read_populations")
        return np.stack([pg, pe], axis=1)

    def dissociation(self, first: int = 0, count: Optional[int] = None):
        count = self.nmol - first if count is None else count
        ag, ae, rn, rd = (np.empty(count) for _ in range(4))
        _check(LIB.ms_read_dissociation(self.h, first, count, _ptr(ag, C.c_double), _ptr(ae, C.c_double),
                                        _ptr(rn, C.c_double), _ptr(rd, C.c_double)), "ms_read_dissociation")
        return np.stack([ag, ae], axis=1), np.stack([rn, rd], axis=1)

    def set_replay(self, E: np.ndarray):
        """Replay drive: E [nsteps][n_molecules][3] lab field (V/m)."""
        e = np.ascontiguousarray(E, np.float32)
        if e.ndim != 3 or e.shape[2] != 3:
            raise ValueError("replay field must be [nsteps][n_molecules][3]")
        _check(LIB.ms_set_replay_field(self.h, _ptr(e, C.c_float), e.shape[0]), "ms_set_replay_field")

    def record_local_fields(self, mol_ids, nsteps: int) -> np.ndarray:
        """Advance nsteps coupled steps; returns E^n at the listed molecules, [nsteps][m][3]."""
        ids = np.ascontiguousarray(mol_ids, np.int64)
        out = np.empty((int(nsteps), ids.size, 3), np.float32)
        _check(LIB.ms_record_local_fields(self.h, _ptr(ids, C.c_int64), ids.size, _ptr(out, C.c_float),
                                          int(nsteps)), "ms_record_local_fields")
        return out

    def save(self, path: str):
        _check(LIB.ms_save(self.h, os.fsencode(path)), "ms_save")

    def load(self, path: str):
        _check(LIB.ms_load(self.h, os.fsencode(path)), "ms_load")

    def dipoles(self, first: int = 0, count: Optional[int] = None) -> np.ndarray:
        count = self.nmol - first if count is None else count
        mu = np.empty((count, 3))
        _check(LIB.ms_read_dipoles(self.h, first, count, _ptr(mu, C.c_double)), "ms_read_dipoles")
        return mu

    def timing_begin(self):
        _check(LIB.ms_timing_begin(self.h), "ms_timing_begin")

    def timing_end(self):
        """(ms per phase [H, molecules, E, total, molecule stage 1, molecule stage 2],
        steps timed, kernels launched)"""
        out = (C.c_double * 6)()
        st = C.c_int64()
        ln = C.c_int64()
        _check(LIB.ms_timing_end(self.h, out, C.byref(st), C.byref(ln)), "ms_timing_end")
        return list(out), st.value, ln.value

    def set_detectors(self, planes, omega):
        """Running DFTs on z-planes `planes` at angular frequencies `omega` (rad/s)."""
        k = np.ascontiguousarray(planes, np.int32)
        w = np.ascontiguousarray(omega, np.float64)
        self._det = (k.size, w.size)
        _check(LIB.ms_set_detectors(self.h, _ptr(k, C.c_int32), k.size, _ptr(w, C.c_double), w.size),
               "ms_set_detectors")

    def flux(self, plane: int) -> np.ndarray:
        """[nsim][nfreq] Poynting flux spectrum through detector plane `plane`."""
        out = np.empty((self.wl.nsim, self._det[1]))
        _check(LIB.ms_read_flux(self.h, plane, _ptr(out, C.c_double)), "ms_read_flux")
        return out

    def dft(self, plane: int, sim: int, component: int, freq: int) -> np.ndarray:
        """[ny][nx] complex accumulator (component 0 Ex, 1 Ey, 2 Hx, 3 Hy)."""
        out = np.empty((self.wl.ny, self.wl.nx, 2))
        _check(LIB.ms_read_dft(self.h, plane, sim, component, freq, _ptr(out, C.c_double)), "ms_read_dft")
        return out[..., 0] + 1j * out[..., 1]

    def species_path(self, species: int = 0) -> int:
        """MS_MOL_FUSED or MS_MOL_STREAMING: the layout the species runs in."""
        return int(LIB.ms_species_path(self.h, species))

    def plan(self, species: int = 0):
        """(layout, MS_KERN_* kernel, chunk width) of a species' molecular step."""
        p, k, c = C.c_int32(), C.c_int32(), C.c_int32()
        _check(LIB.ms_species_plan(self.h, species, C.byref(p), C.byref(k), C.byref(c)), "ms_species_plan")
        return p.value, k.value, c.value

    def set_plan(self, species: int, path: int, kernel: int, chunk: int = 0, ctas_per_sm: int = 0):
        p = (C.c_int32 * 4)(path, kernel, chunk, ctas_per_sm)
        _check(LIB.ms_set_species_plan_ex(self.h, species, p), "ms_set_species_plan_ex")

    def set_batches(self, batches: int):
        """ms_set_mol_batches: 0 = stages in sequence, n >= 1 = pipelined runs."""
        _check(LIB.ms_set_mol_batches(self.h, batches), "ms_set_mol_batches")

    @property
    def batches(self) -> int:
        return int(LIB.ms_mol_batches(self.h))

    def plan_ex(self, species: int = 0):
        """(layout, kernel, chunk width, resident CTAs per SM of the persistent tiled kernel)."""
        p = (C.c_int32 * 4)()
        _check(LIB.ms_species_plan_ex(self.h, species, p), "ms_species_plan_ex")
        return tuple(p)

    @property
    def device_bytes(self) -> int:
        return int(LIB.ms_device_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            LIB.ms_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
