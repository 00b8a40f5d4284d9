"""The measurement helpers of bench.py (no GPU): the timed window's preroll
sits on the pulse peak at the molecular layer, and the FDTD roofline's
algorithmic bytes count what each half step must move."""
import numpy as np

import bench
import workloads as W


def test_peak_preroll_centres_the_window_on_the_pulse_peak():
    wl = W.config1(n_molecules=10)
    warmup, steps = 5, 100
    pre = bench.peak_preroll(wl, warmup, steps)
    centre = pre + warmup + steps // 2
    # the peak leaves the source plane at t0 and crosses (layer centre - source) cells at two steps a cell
    t0_steps = wl.src[0][3] / wl.dt
    k0, k1 = wl.meta["layer"]
    assert abs(centre - (t0_steps + 2 * ((k0 + k1) // 2 - wl.src_k))) <= 1
    assert 0 < pre < wl.nsteps
    assert bench.peak_preroll(wl, 10**6, 10) == 0     # never negative


def test_fdtd_bytes_count_cells_absorbers_and_drude_cells():
    wl = W.config1(n_molecules=10)
    hb, eb = bench.fdtd_bytes(wl)
    cells = wl.cells
    pml_cells = 2 * wl.pml * wl.nx * wl.ny
    drude = int((np.asarray(wl.mat_id) == W.configs.MAT_SILVER).sum())
    assert drude > 0
    assert hb == 36 * cells + 16 * pml_cells
    assert eb == 37 * cells + 16 * pml_cells + 24 * drude
    # a periodic box without metal has neither extra
    wv = W.custom("vac", 8, 8, 32, pml=0, bc_z="periodic", src_k=-1, n_per_sim=0, nsteps=1)
    assert bench.fdtd_bytes(wv) == (36 * wv.cells, 37 * wv.cells)
