#!/usr/bin/env python
"""Benchmark of the coupled Maxwell-Schroedinger step on GB300.

Workload (default): the split-ring-resonator array, a 128x128x192 Yee grid
(2 nm cells, silver Drude rings on glass, CPML in z, TF/SF pulse) driving
50,000 molecules (128-point radial grid, J <= 4, two surfaces) -- one step
is one coupled time step of the whole path (H update, molecular
split-operator step with gather of the local field, polarization scatter,
E update with the Drude current).

Prints ONE JSON line.  value = molecule-steps/s of the whole coupled step
(all ranks); the Yee cell-updates/s of the same steps ride along.
N > 1 ranks (torchrun) run independent replicas (weak scaling).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Yee cell-updates/s + molecule-steps/s, mixed vs plain FP32 at stated error"
UNIT = "molecule-steps/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--molecules", type=int, default=50000)
    p.add_argument("--preroll", type=int, default=None,
                   help="untimed steps before warm-up; default: the timed steps are centred on the "
                        "pulse peak at the molecular layer")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mol-path", default="auto", choices=["auto", "fused", "streaming"])
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the extra forms (mixed split-FP16 tensor-core kinetic pass, spectra, ...)")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return 6800.0, "recipe fallback 6.8 TB/s (of fallback)"


def _kernel_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary, valid only while
    the kernel's source is unchanged (sha256 of the .cu file)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel:
            src = os.path.join(ROOT, "paper_2209_04487_gb300", "csrc", f[1])
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
            return float(f[3]) if sha == f[2] else None
    return None


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device_index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The maximum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def _workload(nmol):
    import workloads as W
    return W.config1(n_molecules=nmol)


# ---------------------------------------------------------------------------
# the oracle, timed on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def _oracle_sample(wl, field_steps=2, mol_sub=500, mol_steps=3):
    """Bounded sample of the same workload through the FP64 oracle: field
    steps on the full grid and molecule steps on a subset; returns the
    whole-step molecule-steps/s extrapolated linearly in molecules."""
    import numpy as np

    from oracle.fdtd import YeeOracle
    from oracle.molecule import SpeciesEnsemble, dtau_au
    f = YeeOracle(wl.nx, wl.ny, wl.nz, wl.nsim, wl.dx, wl.dt, wl.mat_id, wl.materials, pml=wl.pml,
                  bc_z=wl.bc_z, src_k=wl.src_k, src=wl.src, aux_len=4096)
    t0 = time.perf_counter()
    for _ in range(field_steps):
        f.step()
    t_field = (time.perf_counter() - t0) / field_steps
    ens = SpeciesEnsemble(wl.species[0], wl.quat[:mol_sub], dtau_au(wl.dt))
    E = np.random.default_rng(0).standard_normal((mol_sub, 3)) * 1e9
    t0 = time.perf_counter()
    for _ in range(mol_steps):
        ens.step(E)
    t_mol = (time.perf_counter() - t0) / mol_steps * (wl.n_molecules / mol_sub)
    t_step = t_field + t_mol
    return wl.n_molecules / t_step, t_step, t_field, t_mol


def _cpu_desc():
    return os.cpu_count() or 1


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = _workload(a.molecules)
    for _ in range(a.warmup):
        _oracle_sample(wl, field_steps=1, mol_sub=100, mol_steps=1)
    vals, tsteps = [], []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        v, ts, _, _ = _oracle_sample(wl, field_steps=1, mol_sub=200, mol_steps=1)
        vals.append(v)
        tsteps.append(ts)
    wall = time.perf_counter() - t0
    value = wl.n_molecules * len(tsteps) / sum(tsteps)
    sample = (f"per step: 1 FP64 field step on the full {wl.nx}x{wl.ny}x{wl.nz} grid + 200 of "
              f"{wl.n_molecules} molecules, molecule time scaled x{wl.n_molecules // 200}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(tsteps) / len(tsteps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(wl, peak_preroll(wl, a.warmup, a.steps)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cpu_desc(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def peak_preroll(wl, warmup: int, steps: int) -> int:
    """Untimed steps that centre the timed window on the pulse peak at the
    molecular layer: the peak leaves the TF/SF plane at t0 and crosses one
    cell per two steps (Courant number 1/2)."""
    k0, k1 = wl.meta["layer"]
    n_peak = int(round(float(wl.src[0][3]) / wl.dt)) + 2 * ((k0 + k1) // 2 - wl.src_k)
    return max(0, n_peak - warmup - steps // 2)


def fdtd_bytes(wl):
    """Algorithmic bytes of the two half steps per step: H reads E and reads
    and writes H (36 B per cell), E reads H, the material id and reads and
    writes E (37 B); the CPML cells add two psi values read and written
    (16 B) to each, and the Drude cells of the metal slab the current
    (24 B) to the E step."""
    import numpy as np
    cells = wl.cells * wl.nsim
    pml_cells = 2 * wl.pml * wl.nx * wl.ny * wl.nsim if wl.bc_z == "pml" else 0
    metal = {i for i, m in enumerate(wl.materials) if m[1] > 0}
    drude = int(np.isin(np.asarray(wl.mat_id), list(metal)).sum()) if metal else 0
    return 36 * cells + 16 * pml_cells, 37 * cells + 16 * pml_cells + 24 * drude


def fdtd_roofline(wl, h_ms, e_ms, peak):
    hb, eb = fdtd_bytes(wl)
    out = {"bound": "hbm", "peak": peak, "unit": "GB/s"}
    for name, b, ms in (("yee_h_kernel", hb, h_ms), ("yee_e_kernel", eb, e_ms)):
        ach = b / (ms / 1e3) / 1e9
        out[name] = {"achieved": ach, "frac": ach / peak, "bytes_per_launch": b, "ms_per_launch": ms,
                     "traffic": _kernel_traffic(name)}
    out["note"] = ("per half step, CUDA events around each phase (the E phase also holds the one-thread "
                   "step-counter kernel); the fields are evicted from L2 by the molecular state every step")
    return out


def _config(wl, preroll):
    sp = wl.species[0]
    return {"workload": "split-ring array 128x128x192 (2 nm, Ag Drude rings on glass, CPML z, TF/SF "
                        f"pulse) + {wl.n_molecules} molecules (Nr {sp.nr}, J<={sp.jmax}, 2 surfaces)",
            "cells": wl.cells, "molecules": wl.n_molecules, "nr": sp.nr, "jmax": sp.jmax,
            "form": "plain FP32 (FP64 accumulators)",
            "preroll": f"{preroll} untimed steps: the timed steps are centred on the pulse peak at the "
                       "molecular layer, where the local fields, and the coupling series' term count, are largest",
            "l2": "inputs larger than L2 "
            f"(wavepacket state {2 * sp.nrot * sp.nr * 8 * wl.n_molecules / 1e9:.2f} GB per step)",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    a = _args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a)
        return
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2209_04487_gb300 import build
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()
    from paper_2209_04487_gb300 import binding as B

    wl = _workload(a.molecules)
    path = {"auto": B.MS_MOL_AUTO, "fused": B.MS_MOL_FUSED, "streaming": B.MS_MOL_STREAMING}[a.mol_path]
    preroll = peak_preroll(wl, a.warmup, a.steps) if a.preroll is None else a.preroll
    ck_path = None   # the main form's state at the start of its timed window (for e2e)

    def time_form(mol_path, precision, clocks=False, state_form=0, detectors=None, w=None, save_to=None,
                  tune=False):
        """Preroll, warm-up, then a.steps timed steps of one form (CUDA events on
        the library's stream, max over ranks) and its phase timings."""
        sim = B.Simulation(w or wl, mol_path=mol_path, precision=precision, state_form=state_form,
                           autotune=B.MS_TUNE_MEASURE if tune else B.MS_TUNE_OFF)
        plan = sim.plan(0)
        if detectors is not None:
            sim.set_detectors(*detectors)
        form_path = sim.species_path(0)
        # the molecules' work depends on the local field (the coupling series
        # runs until its terms fall below 1e-10): the timed steps sit at the
        # pulse peak, not in the near-zero field before the pulse arrives
        sim.step(preroll)
        sim.step(a.warmup)
        if save_to is not None:
            sim.save(save_to)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        clk = Clocks(local) if clocks else None
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        sim.timing_begin()
        ev0.record(sim.stream)   # the stream the library launches on
        sim.step(a.steps)
        ev1.record(sim.stream)
        torch.cuda.synchronize()
        ph, nst, nlaunch = sim.timing_end()
        cl = clk.stop() if clk else None
        ms_ = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
        if dist:
            dist.barrier()
        Pf = sim.populations()
        nerr = float(np.abs(Pf.sum(axis=1) + sim.dissociation()[0].sum(axis=1) - 1.0).max())
        sim.close()
        del sim
        torch.cuda.empty_cache()
        return {"ms": ms_, "phases": ph, "nsteps": nst, "launches": nlaunch, "clocks": cl, "P": Pf,
                "norm_err": nerr, "path": form_path, "plan": plan}

    # the e2e leg resumes from this state: in memory-backed storage when it fits
    import shutil
    import tempfile
    sp0 = wl.species[0]
    ck_bytes = 16 * sp0.nr * sp0.nrot * wl.n_molecules + 60 * wl.cells * wl.nsim
    ck_dir = None
    if not a.no_e2e:
        for d in ("/dev/shm", None):
            try:
                if d is not None and (not os.path.isdir(d) or shutil.disk_usage(d).free < 2 * ck_bytes):
                    continue
                ck_dir = tempfile.mkdtemp(prefix="ms_bench_", dir=d)
                if shutil.disk_usage(ck_dir).free < 2 * ck_bytes:
                    shutil.rmtree(ck_dir)
                    ck_dir = None
                    continue
                break
            except OSError:
                ck_dir = None
        if ck_dir is not None:
            ck_path = os.path.join(ck_dir, f"rank{rank}.ck")
    main_form = time_form(path, B.MS_PREC_FP32, clocks=True, save_to=ck_path)
    ms, phases, nsteps, launches = main_form["ms"], main_form["phases"], main_form["nsteps"], main_form["launches"]
    cl, P, norm_err = main_form["clocks"], main_form["P"], main_form["norm_err"]
    fused = main_form["path"] == B.MS_MOL_FUSED

    def form_entry(f):
        return {"value": job_rate(wl.n_molecules * a.steps, world, f["ms"] / 1e3), "unit": UNIT,
                "ms_per_step": f["ms"] / a.steps,
                "molecular_step_ms": f["phases"][1] / max(f["nsteps"], 1),
                "layout": "fused" if f["path"] == B.MS_MOL_FUSED else "streaming",
                "populations_max_abs_diff_vs_default": float(np.abs(f["P"] - P).max())}

    # the other forms of the same workload: the streaming layout (FP32) and the
    # mixed form (kinetic pass as a split-FP16 tensor-core GEMM, streaming layout)
    other = {}
    if not a.no_mixed:
        if fused:
            other["plain_fp32_streaming"] = form_entry(time_form(B.MS_MOL_STREAMING, B.MS_PREC_FP32))
        # spectral detection: transmission plane in the glass, reflection plane
        # below the source, 64 frequencies over 1.0 .. 2.5 eV
        spec_planes = [wl.src_k - 4, wl.nz - wl.pml - 2]
        spec_omega = np.linspace(1.0, 2.5, 64) / 6.582119569e-16
        spec = form_entry(time_form(path, B.MS_PREC_FP32, detectors=(spec_planes, spec_omega)))
        spec["note"] = f"running DFTs on z-planes {spec_planes}, 64 frequencies, flux spectra (FP64 accumulators)"
        other["plain_fp32_with_spectra"] = spec
        if all(sp_.jmax <= 4 for sp_ in wl.species):
            par = form_entry(time_form(path, B.MS_PREC_FP32, state_form=B.MS_STATE_PARITY))
            par["note"] = ("parity-reduced state: only (ground, even j) and (excited, odd j) rows, the rows the "
                           "j = 0 start populates; same results as the full state")
            other["plain_fp32_parity_reduced"] = par
        # the paper's production cadence: molecules every 40th field step (by 40 dt)
        # under a CW drive switched on over 5 fs
        import dataclasses
        nsub = 40
        wcw = dataclasses.replace(wl, src_kind="cw", mol_substeps=nsub,
                                  src=np.array([[r[0], r[1], 5e-15, 0.0] for r in wl.src]))
        f = time_form(path, B.MS_PREC_FP32, w=wcw)
        t0 = preroll + a.warmup
        nmolsteps = sum(1 for n in range(t0, t0 + a.steps) if n % nsub == 0)
        other["cw_substeps40"] = {
            "value": job_rate(wl.n_molecules * nmolsteps, world, f["ms"] / 1e3), "unit": UNIT,
            "field_steps_per_s": job_rate(a.steps, world, f["ms"] / 1e3),
            "cell_updates_per_s": job_rate(wl.cells * a.steps, world, f["ms"] / 1e3),
            "ms_per_step": f["ms"] / a.steps, "molecular_steps_timed": nmolsteps,
            "layout": "fused" if f["path"] == B.MS_MOL_FUSED else "streaming",
            "note": f"CW drive (5 fs sin^2 turn-on), molecules every {nsub}th field step by {nsub} dt"}
        # the frozen molecules of Fig. 5d: the same ensemble as two-level emitters
        # (Bloch equations, RK4), transition at the carrier
        import workloads as W
        wbl = dataclasses.replace(wl, species=[W.Species(model="bloch", w0_ev=float(wl.src[0][1]),
                                                         dipole=wl.species[0].dipole)])
        fb = time_form(path, B.MS_PREC_FP32, w=wbl)
        bl = form_entry(fb)
        bl.pop("populations_max_abs_diff_vs_default")
        bl["cell_updates_per_s"] = job_rate(wl.cells * a.steps, world, fb["ms"] / 1e3)
        bl["note"] = ("frozen two-level molecules (Bloch equations, one RK4 step per field step, FP64 state); "
                      "the step is field-bound")
        other["bloch_frozen"] = bl
        # the same workload with the species' plan picked by the create-time autotuner
        ft = time_form(B.MS_MOL_AUTO, B.MS_PREC_FP32, tune=True)
        tuned = form_entry(ft)
        tuned["plan"] = {"layout": ft["plan"][0], "kernel": ft["plan"][1], "chunk": ft["plan"][2]}
        tuned["note"] = ("ms_options.autotune: every plan the species can run timed on a sandbox of 2,048 "
                         "molecules at create (kernel 1 point-resident, 2 tiled, 3 chunked)")
        other["plain_fp32_autotuned"] = tuned
        # the small workload (32x32x64, 1,000 molecules): launch-bound, so the
        # captured-graph replay of ms_step matters; timed with host wall clock
        # around ms_step(a.steps) and a synchronize, graphs on and off
        import workloads as W
        w0 = W.config0()
        small = {}
        for name, gflag in (("graphs", B.MS_GRAPHS_AUTO), ("eager", B.MS_GRAPHS_OFF)):
            sm = B.Simulation(w0, step_graphs=gflag)
            sm.step(1000 - a.warmup - 8)        # the pulse peak of this workload is at step 1000
            sm.step(a.warmup + 8)
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(sm.stream)
            sm.step(a.steps)
            ev1.record(sm.stream)
            torch.cuda.synchronize()
            ms_ = max_over_ranks(ev0.elapsed_time(ev1), dist, "cuda")
            small[name] = {"value": job_rate(w0.n_molecules * a.steps, world, ms_ / 1e3), "unit": UNIT,
                           "ms_per_step": ms_ / a.steps}
            sm.close()
        small["note"] = ("config0 vacuum 32x32x64 with 1,000 molecules (Nr 64, J <= 1) at its pulse peak; "
                         "ms_step replays whole cycles from a captured CUDA graph (graphs) or launches "
                         "every kernel (eager)")
        other["small_workload"] = small
        if B.mixed_supported(wl):
            mixed = form_entry(time_form(B.MS_MOL_STREAMING, B.MS_PREC_MIXED_F16X3))
            mixed["stated_error_vs_fp64"] = ("populations 3.7e-7 to 6.1e-7 abs, dipoles 4e-7 to 5.2e-7 rel after 300 "
                                             "strongly driven steps; norm drift rms 7.5e-7, max 1.9e-6 over 64 "
                                             "molecules in 2000 steps (plain FP32: rms 5.9e-7, max 1.9e-6)")
            other["mixed_f16x3"] = mixed

    sec = ms / 1e3
    value = job_rate(wl.n_molecules * a.steps, world, sec)
    cells_rate = job_rate(wl.cells * a.steps, world, sec)
    sp = wl.species[0]
    state = 16 * sp.nr * sp.nrot                       # FP32 state of one molecule (bytes)
    per_step = lambda k: phases[k] / max(nsteps, 1)    # ms per step of one timed phase
    peak, peak_src = _peaks()
    records = 168  # per molecule: field 16 B, rotation 36, dipole 3x8 read + 2x3x8 written, populations 16,
    #                absorbed norm 2x16
    if fused:
        # dominant kernel: the fused molecular step (stage 2), one launch per step;
        # the state read and written once
        rs_bytes = (2 * state + records) * wl.n_molecules
        kernel = f"mol_rpoint_kernel<{sp.jmax},{sp.nr},fused>"
        note = "algorithmic bytes of the fused molecular step: the state read and written once, 168 B of records"
        roof_kin = None
    else:
        # dominant kernel: the R-space pass (stage 2); in the streaming form it reads
        # s and d2 and writes s'
        rs_bytes = (3 * state + records) * wl.n_molecules
        kernel = f"mol_rpoint_kernel<{sp.jmax},{sp.nr}>" if sp.jmax <= 4 else f"R-space pass <{sp.nr}>"
        note = "algorithmic bytes of the R-space kernel: state and d2 read, new state written, 168 B of records"
        # the kinetic pass (stage 1: field records + kinetic kernel): s read, d2 written
        kin_bytes = (2 * state + 16) * wl.n_molecules
        kin_ms = per_step(4)
        roof_kin = {"bound": "hbm", "achieved": kin_bytes / (kin_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": kin_bytes / (kin_ms / 1e3) / 1e9 / peak, "kernel": f"mol_kinetic_kernel<{sp.nr}>",
                    "bytes_per_launch": kin_bytes, "ms_per_launch": kin_ms}
    rs_ms = per_step(5)
    roof = {"bound": "hbm", "achieved": rs_bytes / (rs_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": rs_bytes / (rs_ms / 1e3) / 1e9 / peak,
            "traffic": _kernel_traffic("mol_rpoint_kernel_fused" if fused else "mol_rpoint_kernel"),
            "kernel": kernel, "bytes_per_launch": rs_bytes, "ms_per_launch": rs_ms, "peak_source": peak_src,
            "note": note}
    # the whole molecular step against the method's minimum: the state read
    # and written once per step plus about 40 B of field and observables
    step_bytes = (2 * state + 40) * wl.n_molecules
    roof_step = {"bound": "hbm", "achieved": step_bytes / (per_step(1) / 1e3) / 1e9, "peak": peak,
                 "unit": "GB/s", "frac": step_bytes / (per_step(1) / 1e3) / 1e9 / peak,
                 "bytes_per_step": step_bytes, "ms_per_step": per_step(1),
                 "note": "molecular step (all its kernels) vs one read and one write of the FP32 state"}
    roof_fdtd = fdtd_roofline(wl, per_step(0), per_step(2), peak)

    e2e = None
    if not a.no_e2e:
        # through the public API: a handle created from the host inputs resumes the
        # run from the checkpoint of the main form's timed window (file -> host ->
        # device), then steps once at a time, reading every population back
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = B.Simulation(wl, mol_path=path)
        host_in = (wl.mat_id.nbytes + wl.pos.nbytes + wl.quat.nbytes + wl.species_id.nbytes
                   + wl.sim_id.nbytes)
        if ck_path is not None:
            s2.load(ck_path)
            host_in += os.path.getsize(ck_path)
        for _ in range(a.steps):
            s2.step(1)
            s2.populations()
        t1 = time.perf_counter()
        s2.close()
        if ck_dir is not None:
            shutil.rmtree(ck_dir, ignore_errors=True)
        e2e_s = max_over_ranks(t1 - t0, dist, "cuda")
        start = ("the checkpoint of the timed window (ms_load)" if ck_path is not None
                 else "t = 0 (no room for the checkpoint: early-time steps)")
        e2e = {"value": job_rate(wl.n_molecules * a.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": host_in / a.steps, "d2h_bytes_per_step": 16 * wl.n_molecules,
               "note": f"ms_create from host inputs, resume from {start}, then per step ms_step(1) and a "
                       "D2H read of all populations; host wall clock"}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        v, ts, tf, tm = _oracle_sample(wl)
        cpu = {"value": v, "unit": UNIT, "cores": _cpu_desc(), "kind": "oracle",
               "sample": f"FP64 numpy oracle: 2 field steps on the full grid ({tf:.2f} s/step) + 3 steps "
                         f"of 500 of {wl.n_molecules} molecules ({tm:.2f} s/step scaled); numpy "
                         "element-wise ops single-threaded, BLAS matmuls on up to all cores"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": _config(wl, preroll), "cell_updates_per_s": cells_rate,
                "phases_ms_per_step": {"h": phases[0] / nsteps, "molecules": phases[1] / nsteps,
                                       "e": phases[2] / nsteps, "molecules_stage1": phases[4] / nsteps,
                                       "molecules_stage2": phases[5] / nsteps},
                "roofline": roof, "roofline_kinetic": roof_kin, "roofline_molecular_step": roof_step,
                "roofline_fdtd": roof_fdtd,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * world,
                "clocks": cl, "norm_bookkeeping_max_err": norm_err,
                "error_vs_fp64": ("this workload's molecules at full size held to the FP64 oracle on a seeded sample "
                                  "under prescribed drives (populations 1e-5 abs, P_e 1e-3 rel, dipoles 1e-4 rel; "
                                  "test_splitring_full_size_molecules_sampled, "
                                  "test_splitring_peak_regime_prescribed_sampled), the full grid's fields within "
                                  "rel L2 1e-4 (test_splitring_full_grid_fields), and the coupled run to the pulse "
                                  "peak within 6e-6 of norm bookkeeping for every molecule "
                                  "(test_splitring_coupled_to_pulse_peak), in tests/test_gpu_parity.py"),
                "forms": {"plain_fp32": {"value": value, "unit": UNIT, "ms_per_step": ms / a.steps,
                                         "molecular_step_ms": phases[1] / nsteps,
                                         "layout": "fused" if fused else "streaming"}, **other}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
