"""The coupled Maxwell-Schroedinger time step, FP64, in the paper's order.

Test infrastructure only (see the package header): the library never calls it.

Section "Efficient numerical implementation of quantum dynamics ...": each
molecule takes the local electric field at its grid point as input, returns
its induced dipole, and the mean-field polarization (dipole times number
density; one simulated molecule per molecule, so P = sum mu / dx^3 per cell)
enters Ampere's law as the current dP/dt (Eq. 1), which changes the field
seen by the other molecules.

One step n -> n+1:
  1. H^{n-1/2} -> H^{n+1/2} from E^n (Eq. 1, CPML, TF/SF, incident line);
  2. gather E^n at each molecule's cell (components owned by the cell);
  3. every molecule advances t_n -> t_{n+1} under that field;
  4. P^{n+1}(c) = sum over the molecules of cell c of mu_k (lab frame);
  5. J_D^{n+1/2} and E^{n+1} with the polarization change P^{n+1} - P^n.
"""
from __future__ import annotations

import numpy as np

from .bloch import BlochEnsemble
from .constants import EA0
from .fdtd import YeeOracle
from .molecule import SpeciesEnsemble, dtau_au
from .spectra import FluxDFT


def ensemble(sp, quat, dtau):
    """The molecular model of a species: ro-vibrational wavepackets, or frozen
    two-level emitters (Bloch equations)."""
    if getattr(sp, "model", "wavepacket") == "bloch":
        return BlochEnsemble(sp, quat, dtau)
    return SpeciesEnsemble(sp, quat, dtau)


def molecule_cells(wl):
    """Cell indices floor(pos/dx) (a point on a cell face belongs to the
    upper cell)."""
    c = np.floor(np.asarray(wl.pos) / wl.dx).astype(np.int64)
    return c[:, 0], c[:, 1], c[:, 2]


class CoupledOracle:
    def __init__(self, wl, *, aux_len=None, with_molecules=True, detectors=None):
        self.wl = wl
        if aux_len is None:
            aux_len = max(4096, wl.nsteps // 2 + 64)
        self.f = YeeOracle(wl.nx, wl.ny, wl.nz, wl.nsim, wl.dx, wl.dt, wl.mat_id,
                           wl.materials, pml=wl.pml, bc_z=wl.bc_z, src_k=wl.src_k,
                           src=wl.src, aux_len=aux_len, src_kind=getattr(wl, "src_kind", "pulse"))
        self.nmol = wl.n_molecules if with_molecules else 0
        self.ci, self.cj, self.ck = molecule_cells(wl)
        # molecules advance every N-th field step by N dt (the paper's cadence:
        # every 40th step); their polarization change enters that step's E update
        self.N = int(getattr(wl, "mol_substeps", 1))
        self.dtau = dtau_au(wl.dt * self.N)
        self.groups = []
        if self.nmol:
            for s, sp in enumerate(wl.species):
                idx = np.nonzero(wl.species_id == s)[0]
                if idx.size:
                    self.groups.append((idx, ensemble(sp, wl.quat[idx], self.dtau)))
        self.mu = np.zeros((self.nmol, 3))
        # detectors = (planes_z, omega): running DFTs after every E half step
        self.dft = FluxDFT(self.f, *detectors) if detectors is not None else None

    def scatter(self, dmu):
        """Per-cell polarization change (C/m^2) from per-molecule dipole
        changes (a.u.), mean-field density 1/dx^3."""
        wl = self.wl
        shp = (wl.nsim, wl.nz, wl.ny, wl.nx)
        out = np.zeros((3,) + shp)
        scale = EA0 / wl.dx ** 3
        for c in range(3):
            np.add.at(out[c], (wl.sim_id, self.ck, self.cj, self.ci), dmu[:, c] * scale)
        return out

    def step(self):
        molecular = self.f.n % self.N == 0
        self.f.step_h()
        if self.nmol and molecular:
            E = self.f.gather(self.wl.sim_id, self.ci, self.cj, self.ck)
            mu = np.empty_like(self.mu)
            for idx, ens in self.groups:
                mu[idx] = ens.step(E[idx])
            dP = self.scatter(mu - self.mu)
            self.mu = mu
            self.f.step_e(dP)
        else:
            self.f.step_e()
        if self.dft is not None:
            self.dft.accumulate()

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    # -- per-molecule observables in the workload's molecule order ------------
    def _collect(self, fn, width):
        out = np.zeros((self.nmol, width))
        for idx, ens in self.groups:
            out[idx] = fn(ens)
        return out

    def populations(self):
        return self._collect(lambda e: e.populations(), 2)

    def absorbed(self):
        return self._collect(lambda e: e.absorbed, 2)

    def excited_R(self):
        return self._collect(lambda e: np.stack(e.excited_R(), axis=1), 2)


class PrescribedOracle:
    """Molecules only, driven by E_k(t_n) = amp_k * wave[n] (lab frame, V/m)."""

    def __init__(self, wl, amp, wave, select=None):
        self.wl = wl
        sel = np.arange(wl.n_molecules) if select is None else np.asarray(select)
        self.sel = sel
        self.amp = np.asarray(amp, np.float64)[sel]
        self.wave = np.asarray(wave, np.float64)
        self.N = int(getattr(wl, "mol_substeps", 1))
        self.dtau = dtau_au(wl.dt * self.N)
        sid = wl.species_id[sel]
        self.groups = []
        for s, sp in enumerate(wl.species):
            idx = np.nonzero(sid == s)[0]
            if idx.size:
                self.groups.append((idx, ensemble(sp, wl.quat[sel][idx], self.dtau)))
        self.n = 0
        self.mu = np.zeros((sel.size, 3))

    def step(self):
        if self.n % self.N == 0:  # molecular steps only (every N-th step, by N dt)
            E = self.amp * self.wave[self.n]
            for idx, ens in self.groups:
                self.mu[idx] = ens.step(E[idx])
        self.n += 1

    def run(self, nsteps):
        for _ in range(nsteps):
            self.step()
        return self

    def _collect(self, fn, width):
        out = np.zeros((self.sel.size, width))
        for idx, ens in self.groups:
            out[idx] = fn(ens)
        return out

    def populations(self):
        return self._collect(lambda e: e.populations(), 2)

    def absorbed(self):
        return self._collect(lambda e: e.absorbed, 2)

    def excited_R(self):
        return self._collect(lambda e: np.stack(e.excited_R(), axis=1), 2)
