#!/usr/bin/env python
"""Benchmark of the coupled Maxwell-Schroedinger step on GB300.

Workload (default, --config 2): the triangular-nanohole array, a 256^3 Yee
grid (2 nm cells, 100 nm Drude-silver film with a 230 nm triangular hole, on
glass, CPML in z, TF/SF pulse) driving 700,000 molecules (128-point radial
grid, J <= 8, two surfaces) -- one step is one coupled time step of the
whole path (H update, molecular split-operator step with gather of the
local field, polarization scatter, E update with the Drude current).
--config 1 (split-ring array 128x128x192, 50,000 molecules at J <= 4),
3 (three species on 192^3) and 4 (sixteen 64x64x128 nanohole cells) run the
other workloads; the split-ring array also carries the extra forms.

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
DT = 2e-9 / (2.0 * 299792458.0)
# configurations 2-4 time their window at the pulse peak after this many steps
# from the start (the peak leaves the source plane at PEAK_T0 steps)
PEAK_T0 = 200


def _args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4])
    p.add_argument("--molecules", type=int, default=None, help="molecules (default: the configuration's)")
    p.add_argument("--preroll", type=int, default=None,
                   help="untimed steps before warm-up; default: the timed steps are centred on the "
                        "pulse peak at the molecular layer")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--mol-path", default="auto", choices=["auto", "fused", "streaming"])
    p.add_argument("--no-forms", action="store_true",
                   help="skip the extra forms (mixed precision, the split-ring forms, ...)")
    p.add_argument("--sweep", type=int, default=0, metavar="STEPS",
                   help="with --config 4: run the sixteen-carrier sweep for STEPS steps from t = 0 with the "
                        "configuration's own pulse (peak at 40 fs) on a reduced copy of --sweep-molecules per cell, "
                        "and add the dissociation yield and Eq. 8's <R>_e per carrier to the line")
    p.add_argument("--sweep-molecules", type=int, default=2000)
    p.add_argument("--state", default="full", choices=["full", "parity"],
                   help="state form of the headline run: every row, or only the rows the j = 0 start populates")
    p.add_argument("--batches", type=int, default=0,
                   help="pipelined molecular step: runs per species (ms_set_mol_batches; 0 = stages in sequence)")
    p.add_argument("--plan", default=None, metavar="KERNEL:CHUNK[:CTAS][,...]",
                   help="pin the species' R-space plans in the streaming layout (tile, pair or chunk), e.g. "
                        "pair:16 for every species or keep,pair:16,pair:8 per species (keep: the library's "
                        "rule); default: the library's rule")
    p.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    return p.parse_args(argv)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (of measured)"
    return 6800.0, "recipe fallback 6.8 TB/s (of fallback)"


def _kernel_traffic(kernel: str):
    """DRAM bytes per molecule from the committed ncu summary, valid only while
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


def workload(cfg: int, nmol=None):
    """The benchmark workload of a configuration.  Configurations 2-4 carry
    their pulse with its peak at PEAK_T0 steps, so that the timed window at
    the peak follows a few hundred untimed steps instead of thousands; grid,
    materials, molecules and the pulse's shape and strength are the
    configuration's."""
    import workloads as W
    if cfg == 1:
        return W.config1(n_molecules=nmol or 50000)
    if cfg == 2:
        return W.config2(n_molecules=nmol or 700000, t0=PEAK_T0 * DT)
    if cfg == 3:
        return W.config3(n_molecules=nmol or 400000, t0=PEAK_T0 * DT)
    per = (nmol or 320000) // 16
    return W.config4(n_per_sim=per, t0=PEAK_T0 * DT)


def describe(cfg: int, wl) -> str:
    sp = wl.species
    mols = ", ".join(f"Nr {s.nr} J<={s.jmax}" for s in sp)
    geo = {1: "split-ring array (Ag Drude rings on glass)", 2: "triangular-nanohole array in a 100 nm Ag film",
           3: "split-ring array (Ag Drude rings on glass)", 4: "triangular-nanohole cells in a 100 nm Ag film"}[cfg]
    cells = f"{wl.nsim} x {wl.nx}x{wl.ny}x{wl.nz}" if wl.nsim > 1 else f"{wl.nx}x{wl.ny}x{wl.nz}"
    return (f"config {cfg}: {geo}, {cells} (2 nm, CPML z, TF/SF pulse) + {wl.n_molecules} molecules "
            f"({mols}, 2 surfaces)")


# ---------------------------------------------------------------------------
# the oracle, timed on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

class OracleSampler:
    """Bounded sample of the workload through the FP64 oracle: each step is
    one field step on the full grid and one molecular step of the first
    mol_sub molecules of each species (driven by a seeded 1e9 V/m field)."""

    def __init__(self, wl, mol_sub=100):
        import numpy as np

        from oracle.fdtd import YeeOracle
        from oracle.molecule import SpeciesEnsemble, dtau_au
        self.np = np
        self.f = YeeOracle(wl.nx, wl.ny, wl.nz, wl.nsim, wl.dx, wl.dt, wl.mat_id, wl.materials, pml=wl.pml,
                           bc_z=wl.bc_z, src_k=wl.src_k, src=wl.src, aux_len=4096)
        self.groups = []
        for s, sp in enumerate(wl.species):
            idx = np.nonzero(wl.species_id == s)[0]
            if idx.size == 0:
                continue
            sub = idx[:mol_sub]
            E = np.random.default_rng(s).standard_normal((sub.size, 3)) * 1e9
            self.groups.append((SpeciesEnsemble(sp, wl.quat[sub], dtau_au(wl.dt)), E, idx.size / sub.size))

    def step(self):
        """(s of the field step, s of the molecular step of the whole ensemble
        scaled linearly in molecules, s measured)"""
        t0 = time.perf_counter()
        self.f.step()
        t_field = time.perf_counter() - t0
        t_mol = 0.0
        for ens, E, scale in self.groups:
            t1 = time.perf_counter()
            ens.step(E)
            t_mol += (time.perf_counter() - t1) * scale
        return t_field, t_mol, time.perf_counter() - t0


def _oracle_in_subprocess(cfg, nmol, threads, mol_sub):
    """The oracle sample in a fresh interpreter whose BLAS and OpenMP pools
    have `threads` threads (None: the library defaults, all cores)."""
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    if threads is not None:
        for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[v] = str(threads)
    spec = json.dumps({"config": cfg, "molecules": nmol, "mol_sub": mol_sub})
    p = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec], env=env,
                       capture_output=True, text=True, timeout=900)
    if p.returncode != 0:
        raise RuntimeError(f"oracle sample failed: {p.stderr[-2000:]}")
    return json.loads(p.stdout.strip().splitlines()[-1])


def _oracle_sample_main(spec):
    d = json.loads(spec)
    wl = workload(d["config"], d["molecules"])
    smp = OracleSampler(wl, d["mol_sub"])
    smp.step()                                  # warm-up
    tf, tm, tall = smp.step()
    print(json.dumps({"t_field": tf, "t_mol": tm, "t_measured": tall, "n_molecules": wl.n_molecules}))


def cpu_baseline(cfg, nmol, wl, mol_sub=100):
    """The oracle at one thread and at all cores (rate of a whole coupled
    step, molecule time scaled from the sample)."""
    cores = os.cpu_count() or 1
    out = {}
    for name, th in (("one_thread", 1), ("all_cores", None)):
        r = _oracle_in_subprocess(cfg, nmol, th, mol_sub)
        out[name] = {"value": wl.n_molecules / (r["t_field"] + r["t_mol"]), "unit": UNIT,
                     "cores": 1 if th == 1 else cores, "s_per_field_step": r["t_field"],
                     "s_per_molecule_step_all_molecules": r["t_mol"], "s_measured": r["t_measured"]}
    allc = out["all_cores"]
    return {"value": allc["value"], "unit": UNIT, "cores": allc["cores"], "kind": "oracle",
            "sample": (f"FP64 numpy oracle in a fresh process: 1 field step on the full grid + 1 step of the first "
                       f"{mol_sub} molecules of each species, molecule time scaled linearly to all "
                       f"{wl.n_molecules}; BLAS on all {cores} cores (numpy element-wise work is single-threaded)"),
            "one_thread": out["one_thread"], "all_cores": allc}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = workload(a.config, a.molecules)
    mol_sub = 100
    smp = OracleSampler(wl, mol_sub)
    for _ in range(a.warmup):
        smp.step()
    t_steps, full = [], []
    t0 = time.perf_counter()
    for _ in range(a.steps):
        tf, tm, tall = smp.step()
        t_steps.append(tall)
        full.append(tf + tm)
    wall = time.perf_counter() - t0
    value = wl.n_molecules * len(full) / sum(full)
    sample = (f"each step: 1 FP64 oracle field step on the full grid + 1 step of the first {mol_sub} molecules of "
              f"each species; value scales the molecule time linearly to all {wl.n_molecules} molecules (a full "
              f"step would take {1e3 * sum(full) / len(full):.0f} ms); ms_per_step is the sample's measured time")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * sum(t_steps) / len(t_steps),
            "ms_per_full_step_extrapolated": 1e3 * sum(full) / len(full),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config(a.config, wl, peak_preroll(wl, a.warmup, a.steps)),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
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
    cells = wl.cells
    pml_cells = 2 * wl.pml * wl.nx * wl.ny * wl.nsim if wl.bc_z == "pml" else 0
    metal = {i for i, m in enumerate(wl.materials) if m[1] > 0}
    drude = int(np.isin(np.asarray(wl.mat_id), list(metal)).sum()) if metal else 0
    return 36 * cells + 16 * pml_cells, 37 * cells + 16 * pml_cells + 24 * drude


def fdtd_roofline(wl, h_ms, e_ms, peak):
    hb, eb = fdtd_bytes(wl)
    out = {"bound": "hbm", "peak": peak, "unit": "GB/s"}
    for name, b, ms in (("yee_h_kernel", hb, h_ms), ("yee_e_kernel", eb, e_ms)):
        ach = b / (ms / 1e3) / 1e9
        out[name] = {"achieved": ach, "frac": ach / peak, "bytes_per_launch": b, "ms_per_launch": ms}
    out["note"] = ("per half step, CUDA events around each phase (the E phase also holds the one-thread "
                   "step-counter kernel); the fields are evicted from L2 by the molecular state every step")
    return out


def _config(cfg, wl, preroll):
    state = sum(16 * s.nr * s.nrot * int((wl.species_id == i).sum()) for i, s in enumerate(wl.species))
    pulse = ("the pulse's peak leaves the source plane at step "
             f"{int(round(float(wl.src[0][3]) / wl.dt))}")
    return {"workload": describe(cfg, wl), "cells": wl.cells, "molecules": wl.n_molecules,
            "species": [{"nr": s.nr, "jmax": s.jmax} for s in wl.species],
            "form": "plain FP32 (FP64 accumulators)",
            "preroll": f"{preroll} untimed steps ({pulse}): the timed steps are centred on the pulse peak at the "
                       "molecular layer, where the local fields, and the coupling series' term count, are largest",
            "l2": f"inputs larger than L2 (wavepacket state {state / 1e9:.2f} GB, read and written every step)",
            "parallelism": "replicas"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

STATE_RECORDS = 168  # per molecule: field 16 B, rotation 36, dipole 3x8 read + 2x3x8 written,
#                      populations 16, absorbed norm 2x16


def main():
    a = _args()
    if a.oracle_sample is not None:
        _oracle_sample_main(a.oracle_sample)
        return
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

    wl = workload(a.config, a.molecules)
    path = {"auto": B.MS_MOL_AUTO, "fused": B.MS_MOL_FUSED, "streaming": B.MS_MOL_STREAMING}[a.mol_path]
    preroll = peak_preroll(wl, a.warmup, a.steps) if a.preroll is None else a.preroll

    def pin(sim, w):
        """--plan: a streaming plan for every species, or one per species."""
        if a.plan:
            specs = a.plan.split(",")
            for i in range(len(w.species)):
                f = (specs[i] if len(specs) > 1 else specs[0]).split(":")
                if f[0] == "keep":
                    continue
                kern = {"tile": B.MS_KERN_TILE, "pair": B.MS_KERN_PAIR, "chunk": B.MS_KERN_CHUNK}[f[0]]
                sim.set_plan(i, B.MS_MOL_STREAMING, kern, int(f[1]), int(f[2]) if len(f) > 2 else 0)

    def time_form(w, mol_path, precision, pre, clocks=False, state_form=0, detectors=None, tune=False,
                  pinned=False):
        """Preroll, warm-up, then a.steps timed steps of one form (CUDA events on
        the library's stream, max over ranks) and its phase timings."""
        sim = B.Simulation(w, mol_path=mol_path, precision=precision, state_form=state_form,
                           autotune=B.MS_TUNE_MEASURE if tune else B.MS_TUNE_OFF)
        if pinned:
            pin(sim, w)
            sim.set_batches(a.batches)
        plans = [sim.plan_ex(i) for i in range(len(w.species))]
        if detectors is not None:
            sim.set_detectors(*detectors)
        form_path = sim.species_path(0)
        sim.step(pre)
        sim.step(a.warmup)
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
                "norm_err": nerr, "path": form_path, "plans": plans}

    main_state = B.MS_STATE_PARITY if a.state == "parity" else 0
    # the three-species configuration's plans (tile shapes, molecules per CTA) come from the autotuner
    tune_main = a.config == 3 and not a.plan
    main_form = time_form(wl, path, B.MS_PREC_FP32, preroll, clocks=True, pinned=True, state_form=main_state,
                          tune=tune_main)
    ms, phases, nsteps, launches = main_form["ms"], main_form["phases"], main_form["nsteps"], main_form["launches"]
    cl, P, norm_err = main_form["clocks"], main_form["P"], main_form["norm_err"]
    fused = main_form["path"] == B.MS_MOL_FUSED

    def form_entry(f, w, ref_P=None):
        e = {"value": job_rate(w.n_molecules * a.steps, world, f["ms"] / 1e3), "unit": UNIT,
             "ms_per_step": f["ms"] / a.steps, "molecular_step_ms": f["phases"][1] / max(f["nsteps"], 1),
             "layout": "fused" if f["path"] == B.MS_MOL_FUSED else "streaming",
             "norm_bookkeeping_max_err": f["norm_err"]}
        if ref_P is not None:
            e["populations_max_abs_diff_vs_plain"] = float(np.abs(f["P"] - ref_P).max())
        return e

    forms = {"plain_fp32": {"value": job_rate(wl.n_molecules * a.steps, world, ms / 1e3), "unit": UNIT,
                            "ms_per_step": ms / a.steps, "molecular_step_ms": phases[1] / nsteps,
                            "layout": "fused" if fused else "streaming", "norm_bookkeeping_max_err": norm_err}}
    sweep = None
    if a.sweep > 0 and a.config == 4:
        sweep = carrier_sweep(a, B, np, torch)
    if not a.no_forms:
        # the mixed form of the same workload: the kinetic pass as a split-FP16
        # tensor-core GEMM (streaming layout), at its stated error
        if B.mixed_supported(wl):
            fm = time_form(wl, B.MS_MOL_STREAMING, B.MS_PREC_MIXED_F16X3, preroll)
            mixed = form_entry(fm, wl, P)
            mixed["gain_vs_plain_fp32"] = ms / fm["ms"]
            mixed["stated_error_vs_fp64"] = (
                "tests/test_gpu_parity.py: populations <= 1.5e-7 abs, P_e <= 6e-7 and dipoles <= 2.9e-7 rel after "
                "300 strongly driven steps; norm drift max 7.3e-7 over 64 molecules in 2000 steps (plain FP32: "
                "1.3e-7)")
            forms["mixed_f16x3"] = mixed
        if a.config != 1 and a.state == "full":
            # the parity-reduced state of the same workload: only the rows the
            # j = 0 start populates (half of them), identical dynamics
            fp = time_form(wl, path, B.MS_PREC_FP32, preroll, state_form=B.MS_STATE_PARITY)
            par = form_entry(fp, wl, P)
            par["gain_vs_full_state"] = ms / fp["ms"]
            par["note"] = ("parity-reduced state: only (ground, even j) and (excited, odd j) rows, the rows the "
                           "j = 0 start populates (each coupling changes j by one and swaps the surfaces); the "
                           "dropped rows of the full state stay exactly zero, so the results are those of the "
                           "full state up to FP32 rounding order (tests/test_gpu_parity.py, "
                           "test_parity_reduced_matches_oracle)")
            forms["parity_reduced"] = par
        if a.config != 1:
            forms.update(splitring_forms(a, B, np, torch, dist, world, time_form, form_entry))
        else:
            forms.update(splitring_forms(a, B, np, torch, dist, world, time_form, form_entry, main=main_form))

    sec = ms / 1e3
    value = job_rate(wl.n_molecules * a.steps, world, sec)
    cells_rate = job_rate(wl.cells * a.steps, world, sec)
    per_step = lambda k: phases[k] / max(nsteps, 1)    # ms per step of one timed phase
    peak, peak_src = _peaks()
    nm = [int((wl.species_id == i).sum()) for i in range(len(wl.species))]
    rows_of = (lambda sp: sp.nrot) if a.state == "parity" else (lambda sp: 2 * sp.nrot)
    states = [8 * s.nr * rows_of(s) for s in wl.species]   # FP32 state of one molecule (bytes)
    st_bytes = sum(b * n for b, n in zip(states, nm))
    one = len(wl.species) == 1
    sp = wl.species[0]
    if fused:
        # dominant kernel: the fused molecular step (stage 2), one launch per step;
        # the state read and written once
        rs_bytes = 2 * st_bytes + STATE_RECORDS * wl.n_molecules
        kernel = f"mol_rpoint_kernel<{sp.jmax},{sp.nr},fused>" if one else "fused molecular steps"
        note = "algorithmic bytes of the fused molecular step: the state read and written once, 168 B of records"
        roof_kin = None
        traffic_key = "mol_rpoint_kernel_fused"
    else:
        # dominant kernel: the R-space pass (stage 2); in the streaming form it reads
        # s and d2 and writes s'
        rs_bytes = 3 * st_bytes + STATE_RECORDS * wl.n_molecules
        if one and sp.jmax <= 4:
            kernel, traffic_key = f"mol_rpoint_kernel<{sp.jmax},{sp.nr}>", "mol_rpoint_kernel"
        elif one and main_form["plans"][0][1] in (B.MS_KERN_PAIR, B.MS_KERN_DEFAULT) and sp.jmax >= 5:
            # the pair kernel's rule: 8-point tiles, 16 for the parity-reduced rows to J = 8
            tile = 8 if sp.jmax >= 9 else (main_form["plans"][0][2] or (16 if a.state == "parity" else 8))
            kernel, traffic_key = f"mol_rspace_pair_kernel<{sp.jmax},{tile}>", "mol_rspace_pair_kernel"
            if a.state == "parity":
                kernel, traffic_key = f"mol_rspace_pair_kernel<{sp.jmax},{tile},parity>", "mol_rspace_pair_kernel_parity"
        elif one and sp.jmax <= 8:
            tile = main_form["plans"][0][2] or (16 if sp.jmax >= 5 else 32)   # the tiled kernel's rule
            kernel, traffic_key = f"mol_rspace_kernel<{sp.jmax},{tile}>", "mol_rspace_kernel"
        else:
            kernel, traffic_key = "R-space passes of every species", None
        note = ("algorithmic bytes of the R-space pass: state and d2 = (T - 1)s read, new state written, 168 B of "
                "records per molecule")
        # the kinetic pass (stage 1: field records + kinetic kernel): s read, d2 written
        kin_bytes = 2 * st_bytes + 16 * wl.n_molecules
        kin_ms = per_step(4)
        roof_kin = {"bound": "hbm", "achieved": kin_bytes / (kin_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": kin_bytes / (kin_ms / 1e3) / 1e9 / peak,
                    "kernel": f"mol_kinetic_kernel<{sp.nr}>" if one else "kinetic passes",
                    "bytes_per_launch": kin_bytes, "ms_per_launch": kin_ms}
    rs_ms = per_step(5)
    traffic = _kernel_traffic(traffic_key) if traffic_key else None
    roof = {"bound": "hbm", "achieved": rs_bytes / (rs_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": rs_bytes / (rs_ms / 1e3) / 1e9 / peak,
            "traffic": traffic * wl.n_molecules if traffic is not None else None,
            "kernel": kernel, "bytes_per_launch": rs_bytes, "ms_per_launch": rs_ms, "peak_source": peak_src,
            "note": note + "; traffic: ncu DRAM bytes per molecule (profiles/traffic.txt) times the molecules"}
    # the whole molecular step against the method's minimum: the state read
    # and written once per step plus about 40 B of field and observables
    step_bytes = 2 * st_bytes + 40 * wl.n_molecules
    roof_step = {"bound": "hbm", "achieved": step_bytes / (per_step(1) / 1e3) / 1e9, "peak": peak,
                 "unit": "GB/s", "frac": step_bytes / (per_step(1) / 1e3) / 1e9 / peak,
                 "bytes_per_step": step_bytes, "ms_per_step": per_step(1),
                 "note": "molecular step (all its kernels) vs one read and one write of the FP32 state"}
    roof_fdtd = fdtd_roofline(wl, per_step(0), per_step(2), peak)

    e2e = None
    if not a.no_e2e:
        # through the public API: ms_create from the host inputs (timed), the
        # untimed steps up to the window, then per step ms_step(1) and a D2H read
        # of every population (timed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = B.Simulation(wl, mol_path=path, state_form=main_state,
                          autotune=B.MS_TUNE_MEASURE if tune_main else B.MS_TUNE_OFF)
        pin(s2, wl)
        s2.set_batches(a.batches)
        torch.cuda.synchronize()
        t_create = time.perf_counter() - t0
        host_in = (wl.mat_id.nbytes + wl.pos.nbytes + wl.quat.nbytes + wl.species_id.nbytes
                   + wl.sim_id.nbytes + wl.src.nbytes)
        s2.step(preroll + a.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            s2.step(1)
            s2.populations()
        t_steps = time.perf_counter() - t0
        s2.close()
        del s2
        torch.cuda.empty_cache()
        e2e_s = max_over_ranks(t_create + t_steps, dist, "cuda")
        e2e = {"value": job_rate(wl.n_molecules * a.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": host_in / a.steps, "d2h_bytes_per_step": 16 * wl.n_molecules,
               "create_s": t_create, "steps_s": t_steps,
               "note": ("host wall clock: ms_create from the host inputs (their bytes counted once over the timed "
                        "steps), plus the timed steps at the window, each ms_step(1) and a D2H read of all "
                        "populations; the untimed steps up to the window are not counted")}

    cpu = None
    if rank == 0 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a.config, a.molecules, wl)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": dict(_config(a.config, wl, preroll), **({"state": "parity-reduced: the rows the j = 0 "
                                                                               "start populates"}
                                                                      if a.state == "parity" else {})),
                "cell_updates_per_s": cells_rate,
                "phases_ms_per_step": {"h": phases[0] / nsteps, "molecules": phases[1] / nsteps,
                                       "e": phases[2] / nsteps, "molecules_stage1": phases[4] / nsteps,
                                       "molecules_stage2": phases[5] / nsteps},
                "plans": [{"layout": p[0], "kernel": p[1], "chunk": p[2], "ctas_per_sm": p[3]}
                          for p in main_form["plans"]],
                "mol_batches": a.batches, "autotuned": tune_main,
                "roofline": roof, "roofline_kinetic": roof_kin, "roofline_molecular_step": roof_step,
                "roofline_fdtd": roof_fdtd,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches * world,
                "clocks": cl, "norm_bookkeeping_max_err": norm_err,
                "error_vs_fp64": ERROR_NOTES.get(a.config, ""),
                "forms": forms}
        if sweep is not None:
            line["carrier_sweep"] = sweep
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def carrier_sweep(a, B, np, torch):
    """The frequency sweep's deliverable (config 4): sixteen cells, carriers
    1.2 + 1.2 i/15 eV, the configuration's 20 fs pulse peaking at 40 fs, run
    from t = 0 for a.sweep steps on a reduced copy of the molecules; per
    carrier the dissociation yield (norm removed by the absorber, per
    molecule, on each surface), P_e and Eq. 8's ensemble <R>_e = sum num /
    sum den.  The first 2,000 steps of three of these cells are held to the
    FP64 oracle element by element in tests/test_gpu_coupled_long.py."""
    import workloads as W
    wl = W.config4(n_per_sim=a.sweep_molecules, nsteps=a.sweep)
    sim = B.Simulation(wl)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.step(a.sweep)
    P = sim.populations()
    absb, R = sim.dissociation()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    sim.close()
    out = []
    for s in range(wl.nsim):
        m = wl.sim_id == s
        out.append({"carrier_ev": float(wl.src[s][1]), "yield_g": float(absb[m, 0].mean()),
                    "yield_e": float(absb[m, 1].mean()), "P_e": float(P[m, 1].mean()),
                    "R_e": float(R[m, 0].sum() / R[m, 1].sum()) if R[m, 1].sum() > 0 else None})
    return {"steps": a.sweep, "t_end_fs": a.sweep * wl.dt * 1e15, "molecules_per_cell": a.sweep_molecules,
            "wall_s": wall, "per_carrier": out,
            "note": "molecule averages of the absorbed norm per surface (the dissociation yield) and of P_e, and "
                    "Eq. 8's ensemble <R>_e (a0) at the end of the run"}


ERROR_NOTES = {
    1: ("tests/test_gpu_parity.py, tests/test_gpu_coupled_long.py: the split-ring grid with 1,000 molecules coupled "
        "for 2,000 steps against the FP64 oracle (fields rel L2 <= 1e-4, populations 1e-5 abs, P_e 1e-3 rel); the "
        "50,000-molecule set under prescribed drives on a seeded sample; the coupled run to the pulse peak with "
        "norm bookkeeping within 1e-6 for every molecule"),
    2: ("tests/test_gpu_configs.py: all 700,000 molecules under a seeded prescribed drive with a seeded sample "
        "integrated by the FP64 oracle (populations 1e-5 abs, dipoles 1e-4 rel), the full 256^3 grid against the "
        "oracle, and the coupled run's norm bookkeeping within 1e-6 for every molecule"),
    3: "tests/test_gpu_configs.py: as for config 2, per species, with the autotuned plans",
    4: ("tests/test_gpu_configs.py and tests/test_gpu_coupled_long.py: three of the sixteen cells with 200 "
        "molecules each coupled for 2,000 steps against the FP64 oracle"),
}


def splitring_forms(a, B, np, torch, dist, world, time_form, form_entry, main=None):
    """The split-ring workload (config 1) in every form the library has, at
    its own pulse peak: plain FP32 (fused layout), streaming layout, with
    spectral detection, parity-reduced state, CW drive with molecules every
    40th step, frozen two-level molecules, the autotuned plan, the mixed
    form, and the small workload's graph replay."""
    import dataclasses

    import workloads as W
    w1 = workload(1)
    pre = peak_preroll(w1, a.warmup, a.steps)
    out = {}
    base = main if main is not None else time_form(w1, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre)
    P1 = base["P"]
    out["splitring_plain_fp32"] = form_entry(base, w1)
    out["splitring_plain_fp32_streaming"] = form_entry(time_form(w1, B.MS_MOL_STREAMING, B.MS_PREC_FP32, pre),
                                                       w1, P1)
    # spectral detection: transmission plane in the glass, reflection plane
    # below the source, 64 frequencies over 1.0 .. 2.5 eV
    spec_planes = [w1.src_k - 4, w1.nz - w1.pml - 2]
    spec_omega = np.linspace(1.0, 2.5, 64) / 6.582119569e-16
    spec = form_entry(time_form(w1, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre, detectors=(spec_planes, spec_omega)), w1, P1)
    spec["note"] = f"running DFTs on z-planes {spec_planes}, 64 frequencies, flux spectra (FP64 accumulators)"
    out["splitring_with_spectra"] = spec
    par = form_entry(time_form(w1, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre, state_form=B.MS_STATE_PARITY), w1, P1)
    par["note"] = ("parity-reduced state: only (ground, even j) and (excited, odd j) rows, the rows the "
                   "j = 0 start populates; same results as the full state")
    out["splitring_parity_reduced"] = par
    # the paper's production cadence: molecules every 40th field step (by 40 dt)
    # under a CW drive switched on over 5 fs
    nsub = 40
    wcw = dataclasses.replace(w1, src_kind="cw", mol_substeps=nsub,
                              src=np.array([[r[0], r[1], 5e-15, 0.0] for r in w1.src]))
    f = time_form(wcw, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre)
    t0 = pre + a.warmup
    nmolsteps = sum(1 for n in range(t0, t0 + a.steps) if n % nsub == 0)
    out["splitring_cw_substeps40"] = {
        "value": job_rate(w1.n_molecules * nmolsteps, world, f["ms"] / 1e3), "unit": UNIT,
        "field_steps_per_s": job_rate(a.steps, world, f["ms"] / 1e3),
        "cell_updates_per_s": job_rate(w1.cells * a.steps, world, f["ms"] / 1e3),
        "ms_per_step": f["ms"] / a.steps, "molecular_steps_timed": nmolsteps,
        "note": f"CW drive (5 fs sin^2 turn-on), molecules every {nsub}th field step by {nsub} dt"}
    # the frozen molecules of Fig. 5d: the same ensemble as two-level emitters
    # (Bloch equations, RK4), transition at the carrier
    wbl = dataclasses.replace(w1, species=[W.Species(model="bloch", w0_ev=float(w1.src[0][1]),
                                                     dipole=w1.species[0].dipole)])
    fb = time_form(wbl, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre)
    bl = form_entry(fb, wbl)
    bl["cell_updates_per_s"] = job_rate(w1.cells * a.steps, world, fb["ms"] / 1e3)
    bl["note"] = ("frozen two-level molecules (Bloch equations, one RK4 step per field step, FP64 state); "
                  "the step is field-bound")
    out["splitring_bloch_frozen"] = bl
    ft = time_form(w1, B.MS_MOL_AUTO, B.MS_PREC_FP32, pre, tune=True)
    tuned = form_entry(ft, w1, P1)
    tuned["plan"] = {"layout": ft["plans"][0][0], "kernel": ft["plans"][0][1], "chunk": ft["plans"][0][2],
                     "ctas_per_sm": ft["plans"][0][3]}
    tuned["note"] = ("ms_options.autotune: every plan the species can run timed on a sandbox of 2,048 "
                     "molecules at create (kernel 1 point-resident, 2 tiled, 3 chunked)")
    out["splitring_autotuned"] = tuned
    if main is not None:   # config 1 is the headline: its mixed form is reported there
        pass
    else:
        fm = time_form(w1, B.MS_MOL_STREAMING, B.MS_PREC_MIXED_F16X3, pre)
        mixed = form_entry(fm, w1, P1)
        mixed["gain_vs_plain_fp32"] = base["ms"] / fm["ms"]
        out["splitring_mixed_f16x3"] = mixed
    # the small workload (32x32x64, 1,000 molecules): launch-bound, so the
    # captured-graph replay of ms_step matters
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
    out["small_workload"] = small
    return out


if __name__ == "__main__":
    main()
