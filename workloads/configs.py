"""Workload builders: grid, materials, molecules and source parameters.

Every array is drawn from a seeded NumPy PCG64 generator so that the CUDA
path and the oracle receive byte-identical inputs.  Geometry follows the
paper's structures (split-ring array, Fig. 2; triangular-nanohole array,
Fig. 6; a thin molecular layer above the metal, Fig. 4b inset) at the sizes
of the five benchmark workloads; the readings used where the paper gives no
number are listed beside each builder.

Units: lengths and times SI (m, s), field amplitudes V/m, photon and Drude
energies eV; molecular parameters in atomic units (E_h, a0, m_e, e*a0).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

# Speed of light (exact SI) -- used only to state the Courant-0.5 time step
# that every workload prescribes (dt = dx / 2c).
_C0 = 299792458.0

# Material table shared by all workloads: (eps_inf, plasma energy [eV],
# damping [eV]); plasma energy 0 marks a non-dispersive dielectric.
MAT_VACUUM, MAT_GLASS, MAT_SILVER = 0, 1, 2
MATERIALS: List[Tuple[float, float, float]] = [
    (1.0, 0.0, 0.0),      # vacuum / molecular layer host
    (2.25, 0.0, 0.0),     # glass half-space, eps = 2.25
    (3.7, 9.0, 0.02),     # Drude silver: eps_inf 3.7, wp 9.0 eV, gamma 0.02 eV
]


@dataclass
class Species:
    """One molecular species (atomic units throughout).

    Ground surface: Morse, De*(1-exp(-a(r-re)))^2 - De (Eq. 6 form).
    Excited surface: A + B*exp(-beta*(r-rc)) (Eq. 7 is A=0, B=2De_e).
    The transition dipole is constant in R (the paper's choice) unless a
    table d(R) at the grid points is given.
    The absorber is cos(pi/2*(r-ra)/(rmax-ra))**power for r > ra.
    """
    nr: int = 64
    rmin: float = 1.0
    rmax: float = 10.0
    mass: float = 918.0
    jmax: int = 1
    De: float = 0.1
    a: float = 1.0
    re: float = 2.0
    A: float = 0.15
    B: float = 0.1
    beta: float = 1.5
    rc: float = 2.0
    dipole: float = 1.0
    absorber_r: float = 8.5
    absorber_power: float = 0.125
    # R-dependent transition dipole d(R) at the radial grid points (e a0), a
    # tuple of nr values; None = the constant `dipole` (the paper's choice)
    dipole_R: Optional[tuple] = None
    # "wavepacket" (the two-surface ro-vibrational model) or "bloch" (frozen
    # two-level emitter: transition energy w0_ev, dipole along the molecular
    # axis, optional relaxation times T1, T2 in s, 0 = none)
    model: str = "wavepacket"
    w0_ev: float = 0.0
    T1: float = 0.0
    T2: float = 0.0

    @property
    def nrot(self) -> int:
        return (self.jmax + 1) ** 2


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    nsim: int
    dx: float
    dt: float
    pml: int
    bc_z: str                      # "pml" or "periodic"
    src_k: int                     # absolute z index of the TF/SF plane, -1 = no source
    src: np.ndarray                # [nsim, 4]: E0 [V/m], carrier [eV], FWHM [s], t0 [s]
    materials: List[Tuple[float, float, float]]
    mat_id: np.ndarray             # uint8 [nsim, nz, ny, nx]
    species: List[Species]
    species_id: np.ndarray         # int32 [n]
    sim_id: np.ndarray             # int32 [n]
    pos: np.ndarray                # float64 [n, 3], metres, absolute in the sim's box
    quat: np.ndarray               # float64 [n, 4], (w, x, y, z), molecule frame -> lab
    nsteps: int
    meta: Dict = field(default_factory=dict)
    src_kind: str = "pulse"        # "pulse" (row: E0, carrier, FWHM, t0) or "cw" (E0, carrier, turn-on, t0)
    mol_substeps: int = 1          # molecules advance every mol_substeps-th field step

    @property
    def n_molecules(self) -> int:
        return int(self.species_id.shape[0])

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz * self.nsim


# ----------------------------------------------------------------------------
# geometry (cell-centre-in-shape staircase, one uint8 id per cell)
# ----------------------------------------------------------------------------

def _srr_mask(nx: int, ny: int) -> np.ndarray:
    """Split ring: outer side 30 cells (60 nm), arm 10 cells (20 nm), 5-cell
    (10 nm) gap centred in the -y arm, ring centred in the unit cell."""
    ci = (np.arange(nx) + 0.5)[None, :]
    cj = (np.arange(ny) + 0.5)[:, None]
    cx, cy = nx / 2.0, ny / 2.0
    outer = (np.abs(ci - cx) < 15) & (np.abs(cj - cy) < 15)
    inner = (np.abs(ci - cx) < 5) & (np.abs(cj - cy) < 5)
    # 5 cells wide: on an even grid the gap sits half a cell off the axis
    gap = (ci - cx >= -2.5) & (ci - cx < 2.5) & (cj < cy - 5) & (cj > cy - 15)
    return outer & ~inner & ~gap


def _triangle_hole_mask(nx: int, ny: int, side: float) -> np.ndarray:
    """Equilateral triangular hole of the given side (cells), one edge along
    x, centroid at the unit-cell centre.  True = inside the hole."""
    ci = (np.arange(nx) + 0.5)[None, :] - nx / 2.0
    cj = (np.arange(ny) + 0.5)[:, None] - ny / 2.0
    h = side * np.sqrt(3.0) / 2.0
    y0 = -h / 3.0                                   # base line (centroid at 0)
    inside = ((cj >= y0)
              & (cj <= y0 + np.sqrt(3.0) * (ci + side / 2.0))
              & (cj <= y0 + np.sqrt(3.0) * (side / 2.0 - ci)))
    return inside


def _srr_geometry(nx, ny, nz, ring_k=(50, 65), glass_k=65) -> np.ndarray:
    m = np.zeros((nz, ny, nx), np.uint8)
    m[glass_k:] = MAT_GLASS
    ring = _srr_mask(nx, ny)
    for k in range(*ring_k):
        m[k][ring] = MAT_SILVER
    return m


def _nanohole_geometry(nx, ny, nz, film_k, glass_k, side) -> np.ndarray:
    m = np.zeros((nz, ny, nx), np.uint8)
    m[glass_k:] = MAT_GLASS
    hole = _triangle_hole_mask(nx, ny, side)
    for k in range(*film_k):
        m[k][~hole] = MAT_SILVER
    return m


# ----------------------------------------------------------------------------
# molecules
# ----------------------------------------------------------------------------

def _random_quaternions(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform rotations: normalised 4D Gaussian vectors (Haar on SO(3))."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _place(rng: np.random.Generator, n: int, nx: int, ny: int, layer: Tuple[int, int],
           dx: float, distinct: bool) -> np.ndarray:
    """Uniform continuous positions in the layer box (absolute metres).  With
    distinct=True the cells are drawn without replacement first, then a
    uniform point inside each cell."""
    k0, k1 = layer
    if distinct:
        ncell = nx * ny * (k1 - k0)
        if n > ncell:
            raise ValueError("more molecules than layer cells")
        c = rng.choice(ncell, size=n, replace=False)
        i = c % nx
        j = (c // nx) % ny
        k = k0 + c // (nx * ny)
        base = np.stack([i, j, k], axis=1).astype(np.float64)
        p = (base + rng.random((n, 3))) * dx
    else:
        u = rng.random((n, 3))
        p = np.empty((n, 3))
        p[:, 0] = u[:, 0] * nx * dx
        p[:, 1] = u[:, 1] * ny * dx
        p[:, 2] = (k0 + u[:, 2] * (k1 - k0)) * dx
    return p


def species_config0(jmax: int = 1, nr: int = 64) -> Species:
    """The benchmark species: 64-point grid on [1,10] a0, mass 918 m_e,
    Morse (0.1, 1.0, 2.0), excited 0.15+0.1 exp(-1.5(r-2)), 1 e*a0."""
    return Species(nr=nr, jmax=jmax)


def _pulse_row(E0, carrier_ev, fwhm, t0):
    return [E0, carrier_ev, fwhm, t0]


def custom(name: str, nx: int, ny: int, nz: int, *, nsim: int = 1, pml: int = 10,
           bc_z: str = "pml", src_k: int = 18, pulses: Optional[Sequence] = None,
           geometry: Optional[Callable[[int, int, int], np.ndarray]] = None,
           layer: Tuple[int, int] = (40, 44), n_per_sim: int = 0,
           species: Optional[List[Species]] = None,
           fractions: Optional[Sequence[float]] = None,
           seed: int = 0, distinct: bool = False, nsteps: int = 100,
           dx: float = 2e-9, src_kind: str = "pulse", mol_substeps: int = 1) -> Workload:
    """General builder used by the five benchmark workloads and by tests."""
    dt = dx / (2.0 * _C0)
    if pulses is None:
        pulses = [_pulse_row(1e9, 1.5498, 10e-15, 1000 * dt)] * nsim
    src = np.asarray(pulses, np.float64).reshape(nsim, 4)
    mat = np.zeros((nsim, nz, ny, nx), np.uint8)
    if geometry is not None:
        g = geometry(nx, ny, nz)
        mat[:] = g[None]
    species = species or [species_config0()]
    fractions = fractions or [1.0]
    rng_pos = np.random.default_rng(2209 + seed)
    rng_rot = np.random.default_rng(4487 + seed)
    sid, simid, pos, quat = [], [], [], []
    for s in range(nsim):
        if n_per_sim == 0:
            continue
        counts = np.floor(np.asarray(fractions) * n_per_sim).astype(int)
        counts[0] += n_per_sim - counts.sum()
        p = _place(rng_pos, n_per_sim, nx, ny, layer, dx, distinct)
        # species labels: a seeded permutation of the exact counts
        lab = np.concatenate([np.full(c, i, np.int32) for i, c in enumerate(counts)])
        rng_pos.shuffle(lab)
        sid.append(lab)
        simid.append(np.full(n_per_sim, s, np.int32))
        pos.append(p)
        quat.append(_random_quaternions(rng_rot, n_per_sim))
    if sid:
        species_id = np.concatenate(sid).astype(np.int32)
        sim_id = np.concatenate(simid).astype(np.int32)
        posa = np.concatenate(pos)
        quata = np.concatenate(quat)
    else:
        species_id = np.zeros(0, np.int32)
        sim_id = np.zeros(0, np.int32)
        posa = np.zeros((0, 3))
        quata = np.zeros((0, 4))
    return Workload(name=name, nx=nx, ny=ny, nz=nz, nsim=nsim, dx=dx, dt=dt, pml=pml,
                    bc_z=bc_z, src_k=src_k, src=src, materials=list(MATERIALS),
                    mat_id=mat, species=species, species_id=species_id, sim_id=sim_id,
                    pos=posa, quat=quata, nsteps=nsteps,
                    meta=dict(layer=layer, seed=seed), src_kind=src_kind, mol_substeps=mol_substeps)


# ----------------------------------------------------------------------------
# the five benchmark workloads
# ----------------------------------------------------------------------------

def config0(n_molecules: int = 1000, jmax: int = 1, nsteps: int = 2000) -> Workload:
    """Vacuum 32x32x64, 800 nm / 10 fs / 1e9 V/m pulse at z=8 past the PML
    (absolute 18), 1,000 molecules in z in [30,34) past the PML (absolute
    40..43), peak of the pulse at t0 = 1000 dt."""
    dt = 2e-9 / (2.0 * _C0)
    return custom("config0: vacuum 32x32x64, 1000 molecules (Nr 64, J<=1)", 32, 32, 64,
                  src_k=18, pulses=[_pulse_row(1e9, 1.5498, 10e-15, 1000 * dt)],
                  layer=(40, 44), n_per_sim=n_molecules,
                  species=[species_config0(jmax=jmax)], seed=0, nsteps=nsteps)


def config1(n_molecules: int = 50000, nsteps: int = 10000, nx: int = 128, ny: int = 128,
            nz: int = 192, t0: float = 20e-15) -> Workload:
    """Split-ring array 128x128x192: silver ring z 50..64, glass z >= 65,
    50,000 molecules in a 20 nm layer z 40..49, Nr 128, J <= 4.  t0: time of
    the pulse peak at the source plane (20 fs; shorter runs that must see the
    peak pass the layer give an earlier one)."""
    sp = Species(nr=128, jmax=4)
    return custom(f"config1: SRR {nx}x{ny}x{nz}, {n_molecules} molecules (Nr 128, J<=4)",
                  nx, ny, nz, src_k=20,
                  pulses=[_pulse_row(1e9, 1.5498, 10e-15, t0)],
                  geometry=_srr_geometry, layer=(40, 50), n_per_sim=n_molecules,
                  species=[sp], seed=1, nsteps=nsteps)


def config2(n_molecules: int = 700000, nsteps: int = 2000, n: int = 256,
            t0: float = 20e-15) -> Workload:
    """Triangular-nanohole array 256^3: 100 nm silver film z 51..100 with a
    side-115-cell (230 nm) equilateral hole, glass z >= 101, molecules on
    distinct cells of the 11-plane layer z 40..50, Nr 128, J <= 8.  t0: time
    of the pulse peak at the source plane."""
    sp = Species(nr=128, jmax=8)
    geo = lambda nx, ny, nz: _nanohole_geometry(nx, ny, nz, (51, 101), 101, 115.0)
    return custom(f"config2: nanohole {n}^3, {n_molecules} molecules (Nr 128, J<=8)",
                  n, n, n, src_k=20, pulses=[_pulse_row(1e9, 1.5498, 10e-15, t0)],
                  geometry=geo, layer=(40, 51), n_per_sim=n_molecules, species=[sp],
                  seed=2, distinct=True, nsteps=nsteps)


def config3_species() -> List[Species]:
    return [Species(nr=64, jmax=4, mass=918.0, De=0.05),
            Species(nr=128, jmax=8, mass=8000.0, De=0.1),
            Species(nr=256, jmax=16, mass=14000.0, De=0.2)]


def config3(n_molecules: int = 400000, nsteps: int = 200, n: int = 192,
            t0: float = 20e-15) -> Workload:
    """Split-ring geometry on 192^3 with three species mixed 0.5/0.3/0.2.
    t0: time of the pulse peak at the source plane."""
    return custom(f"config3: SRR {n}^3, {n_molecules} molecules of 3 species", n, n, n,
                  src_k=20, pulses=[_pulse_row(1e9, 1.5498, 10e-15, t0)],
                  geometry=_srr_geometry, layer=(40, 50), n_per_sim=n_molecules,
                  species=config3_species(), fractions=[0.5, 0.3, 0.2], seed=3,
                  nsteps=nsteps)


def config4(n_per_sim: int = 20000, nsteps: int = 50000, nsim: int = 16,
            carriers: Optional[Sequence[int]] = None, t0: float = 40e-15) -> Workload:
    """16 independent 64x64x128 nanohole cells (42-cell hole, film z 35..84,
    glass >= 85), 20,000 config-0 molecules at J <= 8 per cell in z 30..34,
    carriers 1.2 + 1.2 i/15 eV, 20 fs FWHM, t0 40 fs, 1e9 V/m.  carriers:
    optional subset of the sweep's indices i (0..15), one cell each (nsim is
    then their number); t0: time of the pulse peak at the source plane."""
    sp = species_config0(jmax=8)
    geo = lambda nx, ny, nz: _nanohole_geometry(nx, ny, nz, (35, 85), 85, 42.0)
    if carriers is None:
        ev = [1.2 + 1.2 * i / max(nsim - 1, 1) for i in range(nsim)]
    else:
        ev = [1.2 + 1.2 * i / 15.0 for i in carriers]
        nsim = len(ev)
    pulses = [_pulse_row(1e9, e, 20e-15, t0) for e in ev]
    return custom(f"config4: {nsim} x nanohole 64x64x128, {n_per_sim} molecules each",
                  64, 64, 128, nsim=nsim, src_k=18, pulses=pulses, geometry=geo,
                  layer=(30, 35), n_per_sim=n_per_sim, species=[sp], seed=4,
                  nsteps=nsteps)


CONFIG_BUILDERS = {0: config0, 1: config1, 2: config2, 3: config3, 4: config4}


def prescribed_drive(n_molecules: int, nsteps: int, dt: float, *, E0: float = 1e9,
                     carrier_ev: float = 1.5498, fwhm: float = 10e-15,
                     t0: Optional[float] = None, seed: int = 77):
    """Prescribed lab-frame drive for molecule-only runs: E_k(t_n) = amp_k *
    wave[n].  amp_k has a seeded uniform direction and a magnitude uniform in
    [0.5, 1.5]*E0 [V/m]; wave[n] is the Gaussian-envelope cosine pulse sampled
    at t_n = n*dt (dimensionless, peak 1)."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n_molecules, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    amp = d * (E0 * (0.5 + rng.random((n_molecules, 1))))
    if t0 is None:
        t0 = 0.5 * nsteps * dt
    hbar_evs = 6.582119569e-16
    t = np.arange(nsteps) * dt
    w = carrier_ev / hbar_evs
    wave = np.exp(-4.0 * np.log(2.0) * ((t - t0) / fwhm) ** 2) * np.cos(w * (t - t0))
    return amp.astype(np.float32), wave.astype(np.float32)
