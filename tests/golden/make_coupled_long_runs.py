"""Writes the expected values of the long coupled parity runs.

Runs the FP64 oracle (``oracle/``, nothing else) on two seeded workloads from
``workloads/`` and stores what the GPU tests compare against:

* ``coupled_splitring_2000.npz`` -- the split-ring array (128 x 128 x 192,
  Drude silver rings on glass, CPML, TF/SF source) with 1,000 molecules of
  the workload's species (N_r 128, J <= 4) in its 20 nm layer, coupled for
  2,000 steps, the 10 fs pulse peaking at the source plane at 1,200 dt so
  that it crosses the layer and the rings inside the run;
* ``coupled_sweep3_2000.npz`` -- three cells of the frequency sweep
  (64 x 64 x 128 triangular-nanohole film on glass; carriers 1.2, 1.76 and
  2.4 eV, i = 0, 7, 15 of the sixteen) with 200 molecules each (N_r 64,
  J <= 8), in one handle, coupled for 2,000 steps, the 20 fs pulse peaking
  at 1,000 dt.

Stored per run: per-molecule populations, absorbed norm, lab dipoles and
Eq. 8's numerator and denominator (FP64); E and H (FP32, rounded from the
FP64 oracle) at a seeded sample of cells of each sim plus one full z-plane,
with the sample's flat indices; the L2 norm of every field component on
every z-plane of every sim (FP64), which covers the whole grid.

Usage: python tests/golden/make_coupled_long_runs.py [splitring|sweep3 ...]
(about an hour of CPU per run).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle.coupled import CoupledOracle  # noqa: E402

NSTEPS = 2000


def splitring_workload():
    dt = 2e-9 / (2.0 * 299792458.0)
    return W.config1(n_molecules=1000, nsteps=NSTEPS, t0=1200 * dt)


def sweep3_workload():
    dt = 2e-9 / (2.0 * 299792458.0)
    return W.config4(n_per_sim=200, nsteps=NSTEPS, carriers=[0, 7, 15], t0=1000 * dt)


# sample: n_random seeded cells per sim plus the full z-plane `plane`
SAMPLES = {"splitring": (16384, 45, splitring_workload),
           "sweep3": (8192, 32, sweep3_workload)}


def sample_cells(wl, n_random, plane, seed=909):
    rng = np.random.default_rng(seed)
    per = wl.nx * wl.ny * wl.nz
    rand = np.sort(rng.choice(per, size=n_random, replace=False))
    pl = plane * wl.nx * wl.ny + np.arange(wl.nx * wl.ny)
    return np.unique(np.concatenate([rand, pl])).astype(np.int64)


def run(name):
    n_random, plane, build = SAMPLES[name]
    wl = build()
    t = time.time()
    o = CoupledOracle(wl).run(wl.nsteps)
    wall = time.time() - t
    f = o.f
    cells = sample_cells(wl, n_random, plane)
    comps = [f.Ex, f.Ey, f.Ez, f.Hx, f.Hy, f.Hz]
    fields = np.stack([np.stack([c[s].reshape(-1)[cells] for c in comps]) for s in range(wl.nsim)])
    plane_norms = np.stack([np.stack([np.sqrt((c[s] ** 2).sum(axis=(1, 2))) for c in comps])
                            for s in range(wl.nsim)])
    out = os.path.join(HERE, f"coupled_{name}_{wl.nsteps}.npz")
    np.savez_compressed(
        out,
        nsteps=wl.nsteps, n_molecules=wl.n_molecules, src=wl.src,
        populations=o.populations(), absorbed=o.absorbed(), excited_R=o.excited_R(), mu=o.mu,
        cells=cells, fields=fields.astype(np.float32), plane_norms=plane_norms,
        oracle_seconds=wall)
    print(f"{name}: {wl.name}, {wl.nsteps} steps in {wall:.0f} s -> {out}")


if __name__ == "__main__":
    for nm in (sys.argv[1:] or list(SAMPLES)):
        run(nm)
