#!/usr/bin/env python
"""Throughput benchmark of the chemotaxis particle step on GB300.

Workload (default): the 3D clump workload: unit cube with reflecting walls,
1,000,000 cells of two species (diameters 0.002 / 0.004, D = 1 / 0.5) drawn
from 8 Gaussian clumps (sigma 0.05), chemical on a 256^3 grid (7-point
stencil, decay 0.1, secretion 0.1 by species 0, c0 = 0), dt = 1e-6, runs of
200 steps. A timed step is one pass of the whole step (bin, sort, pair force,
gradient interpolation, move, deposit, PDE). The timed region advances the
simulation in runs of 200 steps, each started from the seeded initial state
(the reset is inside the timed region and counted as launches).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0). With N > 1 (torchrun), every rank runs its own
replicate (seed + rank); no data moves between ranks (weak scaling), only the
timing barrier and the max over ranks.

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores on a self-similar sample of the same workload (fewer cells, clumps and
grid scaled so the per-cell and per-node work is unchanged), sized so the
whole run ends within a few minutes.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/sec at N=1M 3D (and % HBM roofline); adjoint/forward time ratio"
UNIT = "particle-steps/s"
WORKLOAD = "clumps_grid_3d"
RUN_STEPS = 200
BASE_SEED = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=200)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-steps", type=int, default=RUN_STEPS)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-slabs", action="store_true")
    return ap.parse_args()


def workload_config(p, n):
    return {
        "workload": "%s: 3D unit cube, reflecting walls, N=%d two species (diameters %g/%g, D=%g/%g), "
                    "8 Gaussian clumps sigma 0.05, %dx%dx%d grid (7-point, D_c=%g, gamma=%g, k_0=%g), dt=%g, "
                    "runs of %d steps from the initial state"
                    % (WORKLOAD, n, p["diameter"][0], p["diameter"][1], p["D"][0], p["D"][1], p["grid"][0],
                       p["grid"][1], p["grid"][2], p["Dc"], p["gamma"], p["secrete"][0], p["dt"], RUN_STEPS),
        "n_particles": n,
        "grid": list(p["grid"]),
        "dt": p["dt"],
        "run_steps": RUN_STEPS,
        "l2": "inputs larger than L2: c ping-pong 2 x 64 MiB + particles 40 MB per step > 126 MB L2",
    }


def measured_peaks():
    """(HBM GB/s, its source, SM max MHz)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured", float(d.get("sm_max_mhz", 2070.0))
    except Exception:
        return 6800.0, "fallback", 2070.0


# FP32 operations of one in-cutoff pair (Sect. 3.2 force), evaluated once per
# unordered pair (Newton's third law): the difference vector (3), r^2 (5),
# rsqrt, r, -r/eps, exp, minus the shift, times inter/eps, times 1/r, the
# fixed-point scale and the three components (3): 20 operations, an FMA
# counted as 2; plus d additions of the negated term to the partner.
def flop_per_pair(dim: int) -> float:
    return 20.0 + dim


# FP32 operations of a candidate distance test that finds no pair (the cell
# list's candidates of the neighbouring bins, Sect. 3.1): the difference
# vector (3) and r^2 (5).
FLOP_PER_TEST = 8.0
# FP32 lanes of GB300: 152 SMs x 128 lanes, an FMA (2 flop) per lane per cycle.
FP32_LANES = 152 * 128
# Algorithmic bytes of the particle part of a step per cell: read and write
# the float4 state and the species byte (34 B) and one cell-list key/index
# pass (8 B).
PARTICLE_BYTES = 42.0

# DRAM bytes (read + write) per launch from one ncu capture, for the roofline's
# traffic field ("k_step": the particle kernels of one step together, at
# step 10 of the 3D workload); None where a kernel changed after the capture.
NCU_TRAFFIC_BYTES = {"k_step": 138.16e6, "k_pde": 93.31e6, "k_scan": None, "k_scatter": None}


# ---------------------------------------------------------------------------
# nvidia-smi clock sampler
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,index,utilization.gpu,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.fh = None

    def start(self):
        try:
            self.fh = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    @staticmethod
    def _when(r):
        """Host time (seconds since the epoch) of a sample, or None."""
        try:
            import datetime
            return datetime.datetime.strptime(r[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except (ValueError, IndexError):
            return None

    def stop(self, windows=()):
        """The record of the samples. A sample is under load when it was
        taken inside one of `windows` ((start, end) host times between which
        the benchmark's kernels ran, by the same clock as nvidia-smi's
        timestamps) or when it reports a utilisation of 50 % or more (a
        utilisation that nvidia-smi averages over a longer time than a short
        run lasts)."""
        if self.proc is None:
            return None
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.seek(0)
        rows = [r.split(", ") for r in self.fh.read().strip().splitlines() if r.strip()]

        def busy(r):
            t = self._when(r)
            in_window = t is not None and any(a <= t <= b for a, b in windows)
            return in_window or (r[2].strip().isdigit() and int(r[2]) >= 50)

        load = [r for r in rows if len(r) >= 11 and busy(r)]
        use = load if load else rows
        mhz = [float(r[3]) for r in use if r[3].replace(".", "").isdigit()]
        mx = [float(r[4]) for r in use if r[4].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in use:
            for k, nm in enumerate(names):
                if len(r) > 7 + k and r[7 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


# ---------------------------------------------------------------------------
# oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_threads():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline_full(p, pos, sp, budget_s=12.0, max_steps=10):
    """The oracle (as it stands) advancing the full workload for a few steps."""
    import numpy as np
    from oracle import chemo_oracle as orc
    th = oracle_threads()
    orc.set_threads(th)
    c = np.zeros(orc.grid_shape(p))
    x = pos.astype(np.float64)
    s = sp.copy()
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        x, s, c, _ = orc.step(p, x, s, c, step_index=steps)
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    out = {"value": pos.shape[0] * steps / el, "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
           "sample": "%d full steps of the %d-cell 3D clump workload (FP64 oracle, OpenMP)" % (steps, pos.shape[0])}
    # the same oracle on one host thread, over a self-similar 1/64 sample
    # (same cell density and nodes per cell) for about 3 s
    try:
        orc.set_threads(1)
        q, qpos, qsp = scaled_sample(1.0 / 64.0, BASE_SEED)
        x = qpos.astype(np.float64)
        s = qsp.copy()
        c = np.zeros(orc.grid_shape(q))
        t0 = time.perf_counter()
        k = 0
        while k < 5:
            x, s, c, _ = orc.step(q, x, s, c, step_index=k)
            k += 1
            if time.perf_counter() - t0 > 3.0:
                break
        el1 = time.perf_counter() - t0
        out["one_thread"] = {"value": qpos.shape[0] * k / el1, "unit": UNIT, "cores": 1,
                             "sample": "%d steps of a self-similar %d-cell sample of the clump workload (%d^3 grid)"
                                       % (k, qpos.shape[0], q["grid"][0])}
    finally:
        orc.set_threads(th)
    return out


def scaled_sample(frac, seed):
    """Self-similar sample of the clump workload: frac of the cells, clump
    sigma and grid side scaled by frac^(1/3) so the cell density and the
    nodes per cell are unchanged."""
    from paper_1805_11007_gb300 import workloads as wl
    import numpy as np
    full = wl.WORKLOADS[WORKLOAD]
    n = max(2048, int(full["n"] * frac))
    lin = (n / full["n"]) ** (1.0 / 3.0)
    g = max(8, int(round(256 * lin)))
    p = wl.params(WORKLOAD, grid=[g, g, g], seed=seed)
    pos = wl.clump_positions(n, 3, p["lo"], p["hi"], seed, sigma=0.05 * lin)
    sp = wl.half_species(n, 2)
    return p, pos, sp


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    import numpy as np
    from oracle import chemo_oracle as orc
    from paper_1805_11007_gb300 import workloads as wl
    orc.build()
    th = oracle_threads()
    orc.set_threads(th)
    # calibrate the per-cell cost on a 1/64 sample, then size the sample so
    # warmup + steps take about 150 s
    p, pos, sp = scaled_sample(1.0 / 64.0, BASE_SEED)
    c = np.zeros(orc.grid_shape(p))
    t0 = time.perf_counter()
    orc.step(p, pos, sp, c)
    per_cell = (time.perf_counter() - t0) / pos.shape[0]
    budget = 150.0
    n_target = budget / max(1, args.steps + args.warmup) / max(per_cell, 1e-12)
    frac = min(1.0, max(2048.0, n_target) / wl.WORKLOADS[WORKLOAD]["n"])
    p, pos, sp = scaled_sample(frac, BASE_SEED)
    x = pos.astype(np.float64)
    s = sp.copy()
    c = np.zeros(orc.grid_shape(p))
    step = 0
    for _ in range(args.warmup):
        x, s, c, _ = orc.step(p, x, s, c, step_index=step)
        step += 1
    t0 = time.perf_counter()
    for _ in range(args.steps):
        x, s, c, _ = orc.step(p, x, s, c, step_index=step)
        step += 1
    el = time.perf_counter() - t0
    n = pos.shape[0]
    value = n * args.steps / el
    sample = ("self-similar sample of the clump workload: %d cells, clump sigma %.4f, %d^3 grid (per-cell and "
              "per-node work of the full workload); FP64 oracle on %d host threads" %
              (n, 0.05 * (n / 1e6) ** (1 / 3), p["grid"][0], orc.get_threads()))
    full_p = wl.params(WORKLOAD)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(full_p, 1_000_000), sample=sample),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.get_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def adjoint_ratio(chemo, wl, devc, stream):
    """(forward + backward) / forward time of the differentiable workload:
    forward = chemo_step_n of 200 steps; backward = chemo_record of the same
    200 steps (checkpoints every 20) plus chemo_gradient."""
    import torch
    w = wl.WORKLOADS["adjoint_2d"]
    p, pos, sp = wl.initial_state("adjoint_2d")
    n, steps, every = pos.shape[0], w["steps"], w["ckpt_every"]
    dpos = torch.from_numpy(pos).to(devc)
    dsp = torch.from_numpy(sp).to(devc)
    sim = chemo.chemo_create(p, dpos, dsp, stream=stream)
    try:
        # dL/dX(T) of the differentiable workload's loss, L = mean x
        # displacement + mean squared soft occupancy of a 64^2 analysis grid,
        # at the final state of a forward run (torch autograd on the device)
        from paper_1805_11007_gb300 import adjoint as adj
        chemo.chemo_step_n(sim, steps, stream=stream)
        xT = torch.zeros((n, 2), dtype=torch.float32, device=devc)
        chemo.chemo_read_state(sim, xT, None, None, stream=stream)
        xT.requires_grad_(True)
        loss = adj.mean_x_displacement(xT, dpos) + adj.occupancy_loss(xT, 64, p["lo"], p["hi"])
        g, = torch.autograd.grad(loss, xT)
        g = g.detach().contiguous()
        dth = torch.zeros(2 + p["n_species"], dtype=torch.float32, device=devc)
        c0 = torch.zeros(tuple(chemo.grid_shape(p)), dtype=torch.float32, device=devc)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        for rep in range(2):  # the first pass warms up graphs and allocations
            # the gradient drops the graphs it captured with its tape set: the
            # forward's graphs are captured again here, before the timed run
            chemo.chemo_step_n(sim, 32, stream=stream)
            chemo.chemo_write_state(sim, dpos, dsp, stream=stream)
            chemo.chemo_write_field(sim, c0, stream=stream)
            chemo.chemo_set_step_index(sim, 0, stream=stream)
            ev[0].record(stream)
            chemo.chemo_step_n(sim, steps, stream=stream)
            ev[1].record(stream)
            chemo.chemo_write_state(sim, dpos, dsp, stream=stream)
            chemo.chemo_write_field(sim, c0, stream=stream)
            chemo.chemo_set_step_index(sim, 0, stream=stream)
            ev[2].record(stream)
            chemo.chemo_record(sim, steps, every, stream=stream)
            ev[4].record(stream)
            chemo.chemo_gradient(sim, g, dth, stream=stream)
            ev[3].record(stream)
            # the same with every segment's states kept during the record (the
            # tape of this workload fits many times over in HBM): no re-run
            chemo.chemo_write_state(sim, dpos, dsp, stream=stream)
            chemo.chemo_write_field(sim, c0, stream=stream)
            chemo.chemo_set_step_index(sim, 0, stream=stream)
            ev[5].record(stream)
            chemo.chemo_record(sim, steps, every, stream=stream, store_bytes=-1)
            ev[6].record(stream)
            chemo.chemo_gradient(sim, g, dth, stream=stream)
            ev[7].record(stream)
            torch.cuda.synchronize()
        fwd = ev[0].elapsed_time(ev[1])
        both = ev[2].elapsed_time(ev[3])
        rec = ev[2].elapsed_time(ev[4])
        both_s = ev[5].elapsed_time(ev[7])
        rec_s = ev[5].elapsed_time(ev[6])
        return {"workload": "adjoint_2d: 2D walls, N=%d two species, %dx%d grid (%d PDE substeps), %d steps, "
                            "checkpoints every %d, loss mean x displacement + soft occupancy (64^2), gradients wrt chi, inter, D_0, D_1"
                            % (n, p["grid"][0], p["grid"][1], chemo.chemo_get_info(sim)["pde_substeps"], steps, every),
                "forward_ms": fwd, "forward_backward_ms": both, "record_ms": rec, "gradient_ms": both - rec,
                "ratio": both / fwd,
                "stored": {"how": "chemo_record_stored with every segment kept (checkpoints every %d as well); "
                                  "the gradient is the reverse sweep alone" % every,
                           "record_ms": rec_s, "gradient_ms": both_s - rec_s, "ratio": both_s / fwd},
                "gradients_finite": bool(torch.isfinite(dth).all().item())}
    finally:
        sim.close()


def ensemble_leg(chemo, wl, devc, stream, rank, world, dist, barrier, steps=500, serial_reps=16, serial_steps=100):
    """The 256-replicate ensemble (2D walls physics, sizes log-uniform in
    [1e3, 6.4e4], 128^2 grid each) advanced as one batched simulation per
    rank (replicates sharded across ranks by particle count), against the
    same replicates run one simulation at a time."""
    import numpy as np
    import torch
    from paper_1805_11007_gb300 import ensemble as en
    p, sizes, pos, sp = wl.ensemble_state()
    mine = en.shard_replicates(sizes, world)[rank]
    s_m, pos_m, sp_m = en.take(pos, sp, sizes, mine)
    # the cell list and launch choices of this ensemble, tuned on it
    t0 = time.perf_counter()
    p, tuned_ms = chemo.chemo_autotune(p, s_m, pos_m, sp_m, trial_steps=10, stream=stream)
    tune_s = time.perf_counter() - t0
    dpos = torch.from_numpy(pos_m).to(devc)
    dsp = torch.from_numpy(sp_m).to(devc)
    sim = chemo.chemo_create_batch(p, s_m, dpos, dsp, stream=stream)
    c0 = torch.zeros((len(s_m),) + tuple(chemo.grid_shape(p)), dtype=torch.float32, device=devc)

    def reset():
        chemo.chemo_write_state(sim, dpos, dsp, stream=stream)
        chemo.chemo_write_field(sim, c0, stream=stream)
        chemo.chemo_set_step_index(sim, 0, stream=stream)

    try:
        reset()
        chemo.chemo_step_n(sim, 20, stream=stream)
        reset()
        barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        chemo.chemo_step_n(sim, steps, stream=stream)
        ev[1].record(stream)
        barrier()
        chemo.chemo_check(sim, stream=stream)
        t = torch.tensor([ev[0].elapsed_time(ev[1])], dtype=torch.float64, device=devc)
        if dist is not None:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        # the ensemble's statistics at the end of the run, reduced on the
        # device per replicate and gathered from every rank (the one exchange
        # of a sharded ensemble; outside the timed region)
        obs = chemo.chemo_observables(sim, stream=stream)
        rows = np.array([np.concatenate([o["count"], o["msd"], [o["c_mass"]]]) for o in obs], np.float64)
        allrows = en.gather_replicates(rows, sizes, world, rank, dist.all_gather_object if dist is not None else None)
        reset()
        prof = chemo.chemo_profile_steps(sim, 50, stream=stream)
        info = chemo.chemo_get_info(sim)
    finally:
        sim.close()
    out = {"workload": "ensemble_2d: %d replicates of the 2D walls physics, N_r log-uniform in [1e3, 6.4e4] "
                       "(sum %d), %dx%d grid each (%d PDE substep), %d steps, one batched simulation per GPU"
                       % (len(sizes), int(sizes.sum()), p["grid"][0], p["grid"][1], info["pde_substeps"], steps),
           "value": float(sizes.sum()) * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
           "launches_per_step": info["launches_per_step"],
           "autotuned": {"search_mode": p["search_mode"], "bin_side": p["bin_side"], "warp_runs": p["warp_runs"],
                         "block_threads": p.get("block_threads", 0),
                         "pde_overlap": p["pde_overlap"], "trial_ms_per_step": tuned_ms, "tuning_s": tune_s},
           "kernel_ms": {k: prof[k] for k in ("k_step", "k_pde", "k_scan", "k_scatter", "step")},
           "observables": {"how": "chemo_observables per replicate after the timed run, gathered from every rank",
                           "cells": float(allrows[:, :2].sum()), "replicates": int(allrows.shape[0]),
                           "mean_c_mass": float(allrows[:, -1].mean())}}
    if rank == 0:
        # the same replicates one simulation at a time (each with its own
        # CUDA graphs), for the batching gain
        reps = mine[:serial_reps]
        sims = []
        try:
            for r in reps:
                s1, p1, q1 = en.take(pos, sp, sizes, [r])
                sims.append((chemo.chemo_create(wl.replicate_params(p, r), torch.from_numpy(p1).to(devc),
                                                torch.from_numpy(q1).to(devc), stream=stream), int(s1[0])))
            for sm, _ in sims:
                chemo.chemo_step_n(sm, 4, stream=stream)
            torch.cuda.synchronize()
            ev[2].record(stream)
            for sm, _ in sims:
                chemo.chemo_step_n(sm, serial_steps, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            ms1 = ev[2].elapsed_time(ev[3])
            psteps = sum(m for _, m in sims) * serial_steps
            out["one_at_a_time"] = {"value": psteps / (ms1 * 1e-3), "unit": UNIT, "replicates": len(sims),
                                    "steps": serial_steps, "ms_per_replicate_step": ms1 / (len(sims) * serial_steps)}
        finally:
            for sm, _ in sims:
                sm.close()
    return out


def variants_leg(chemo, wl, devc, stream, steps=200):
    """Device ms per step of the 2D walls workload (100,000 cells, 512^2 grid,
    12 PDE substeps) with each model variant switched on alone: the
    Euler-Maruyama / cloud-in-cell baseline, tamed Euler, the hard-sphere
    correction (with its re-sort), the Gaussian kernel density deposit, and
    type switching."""
    import torch
    base, pos, sp = wl.initial_state("walls_grid_2d")
    dpos = torch.from_numpy(pos).to(devc)
    dsp = torch.from_numpy(sp).to(devc)
    cases = {"baseline": {}, "tamed_euler": {"move_scheme": 1}, "hard_sphere": {"hard_sphere": 1},
             "kde_deposit": {"deposit_kernel": 1},
             "reactions": {"reactions": 1, "react_k0": [10.0, 0.0], "react_kc": [0.0, 5.0], "react_to": [1, 0]}}
    out = {"workload": "walls_grid_2d: 2D walls, N=%d two species, 512x512 grid (12 PDE substeps), %d steps from "
                       "the initial state" % (pos.shape[0], steps)}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for name, over in cases.items():
        p = dict(base, **over)
        with chemo.chemo_create(p, dpos, dsp, stream=stream) as sim:
            chemo.chemo_step_n(sim, 4, stream=stream)
            chemo.chemo_write_state(sim, dpos, dsp, stream=stream)
            chemo.chemo_set_step_index(sim, 0, stream=stream)
            ev[0].record(stream)
            chemo.chemo_step_n(sim, steps, stream=stream)
            ev[1].record(stream)
            torch.cuda.synchronize()
            chemo.chemo_check(sim, stream=stream)
            ms = ev[0].elapsed_time(ev[1]) / steps
            out[name] = {"ms_per_step": ms, "particle_steps_per_s": pos.shape[0] / (ms * 1e-3),
                         "launches_per_step": chemo.chemo_get_info(sim)["launches_per_step"]}
            if name == "baseline":
                prof = chemo.chemo_profile_steps(sim, 50, stream=stream)
                out[name]["kernel_ms"] = {k: prof[k] for k in ("k_step", "k_pde", "k_scan", "k_scatter", "step")}
    return out


def slabs_leg(chemo, wl, steps=20, counts=(1, 2, 3)):
    """Wall-clock ms per step of the 1M-cell 3D clump workload decomposed into
    K z-slabs (slabs.py), every sub-domain on this GPU on its own stream, the
    exchanges included (the host reads the selection counters once per step
    and synchronises), for each K in counts; K = 1 is the same driver with
    one sub-domain (it still selects and re-ingests its cells every step)."""
    import torch
    from paper_1805_11007_gb300 import slabs
    p, pos, sp = wl.initial_state("clumps_grid_3d")
    out = {"workload": "clumps_grid_3d: 3D, N=%d, 256^3 grid, %d steps after 3 warm-up steps" % (pos.shape[0], steps),
           "how": "slabs.create_local + SlabRun.step (particles, fold, field, halo, select, count read-back, "
                  "ingest per step); wall clock between device synchronisations"}
    for K in counts:
        run = slabs.create_local(p, pos, sp, K)
        try:
            for _ in range(3):
                run.step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                run.step()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / steps
            for sub in run.subs.values():
                sub.check()
            out["K=%d" % K] = {"ms_per_step": ms, "particle_steps_per_s": pos.shape[0] / (ms * 1e-3),
                               "halo_planes": run.layout.H, "cut_planes": run.layout.P,
                               "cells_per_subdomain": [int(s.sim.n) for s in run.subs.values()]}
        finally:
            slabs.close_run(run)
    return out


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    from paper_1805_11007_gb300 import build as gb
    gb.build()
    from paper_1805_11007_gb300 import chemo
    from paper_1805_11007_gb300 import workloads as wl

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    p, pos, sp = wl.initial_state(WORKLOAD, seed=BASE_SEED + rank)
    n = pos.shape[0]
    devc = torch.device("cuda", local)
    pos0 = torch.from_numpy(pos).to(devc)
    sp0 = torch.from_numpy(sp).to(devc)
    zero_c = torch.zeros(chemo.grid_shape(p), dtype=torch.float32, device=devc)
    stream = torch.cuda.current_stream()
    sim = chemo.chemo_create(p, pos0, sp0, stream=stream)
    info = chemo.chemo_get_info(sim)
    per_step = info["launches_per_step"]
    reset_launches = 3  # pack, scan, scatter

    state = {"in_run": 0, "resets": 0}

    def reset():
        chemo.chemo_write_state(sim, pos0, sp0, stream=stream)
        chemo.chemo_write_field(sim, zero_c, stream=stream)
        chemo.chemo_set_step_index(sim, 0, stream=stream)
        state["in_run"] = 0
        state["resets"] += 1

    def advance(k):
        while k > 0:
            if state["in_run"] == RUN_STEPS:
                reset()
            m = min(k, RUN_STEPS - state["in_run"])
            chemo.chemo_step_n(sim, m, stream=stream)
            state["in_run"] += m
            k -= m

    # chemo_step_n captures its CUDA graphs (2 and 16 steps, every buffer
    # parity) on first use; do that here, outside the timed region, then
    # start the run again
    reset()
    chemo.chemo_step_n(sim, 18, stream=stream)
    reset()
    advance(args.warmup)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    resets0 = state["resets"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    busy = [time.time()]  # host times around the GPU work, for the clock record
    ev0.record(stream)
    advance(args.steps)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    resets_in = state["resets"] - resets0
    chemo.chemo_check(sim, stream=stream)
    busy.append(time.time())
    t_local = torch.tensor([ms], dtype=torch.float64, device=devc)
    if dist is not None:
        dist.all_reduce(t_local, op=dist.ReduceOp.MAX)
    ms_max = float(t_local.item())
    value = n * args.steps * world / (ms_max * 1e-3)
    ms_per_step = ms_max / args.steps

    # per-kernel device times over one whole run (same kernels, streams and
    # overlap as a step), and the in-cutoff pair interactions per step
    reset()
    nprof = min(args.profile_steps, RUN_STEPS)
    busy.append(time.time())
    prof = chemo.chemo_profile_steps(sim, nprof, stream=stream)
    busy.append(time.time())
    state["in_run"] = nprof
    # the clock record covers the timed region and the profiled run after it
    # (a short timed region can end between two samples)
    clock_rec = clocks.stop(windows=[(busy[0], busy[1]), (busy[2], busy[3])])
    clock_rec["covers"] = "timed region + %d profiled steps" % nprof
    G = int(np.prod(p["grid"]))
    s = info["pde_substeps"]
    hbm, peak_kind, sm_mhz = measured_peaks()
    fp32_peak = FP32_LANES * 2.0 * sm_mhz * 1e6 / 1e12  # TFLOP/s
    pairs_per_step = prof["pairs_per_step"]
    kern = {k: prof[k] for k in ("k_step", "k_pde", "k_scan", "k_scatter")}
    dom = max(kern, key=kern.get)
    if dom == "k_step":
        # the particle kernels (pair force + move): HBM fraction of the
        # method's particle bytes (42 B per cell and step: the float4 state
        # and species read and written, and the cell list's key/index pass)
        # in their event time; they are bound by the pair search's issued
        # instructions, so the ALU view rides along: each unordered in-cutoff
        # pair once (pairs_per_step counts every pair for both of its cells)
        # plus 8 flop per candidate test that found no pair (counted by the
        # half-window kernels while profiling)
        unordered = 0.5 * pairs_per_step
        rejected = max(prof.get("tests_per_step", 0.0) - unordered, 0.0)
        flops = (flop_per_pair(p["dim"]) * unordered + FLOP_PER_TEST * rejected) / (kern[dom] * 1e-3) / 1e12
        half = info["search_mode"] == 4
        achieved = PARTICLE_BYTES * n / (kern[dom] * 1e-3) / 1e9
        roofline = {"kernel": ("k_pairs_half + k_step" if half else dom), "bound": "hbm",
                    "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                    "algorithmic_bytes": PARTICLE_BYTES * n,
                    "peak_source": ("%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                                    else "fallback 6.8 TB/s"),
                    "alu": {"achieved": flops, "peak": fp32_peak, "unit": "TFLOP/s", "frac": flops / fp32_peak,
                            "peak_source": "FP32 lanes x 2 x SM max clock (%d x 2 x %.0f MHz)"
                                           % (FP32_LANES, sm_mhz)}}
    else:
        bytes_per = {"k_pde": 8.0 * G * s, "k_scan": 36.0 * info["bin_slots"] / 8.0, "k_scatter": 36.0 * n}
        achieved = bytes_per[dom] / (kern[dom] * 1e-3) / 1e9
        roofline = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                    "frac": achieved / hbm,
                    "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                    else "fallback 6.8 TB/s"}
    roofline.update({"traffic": NCU_TRAFFIC_BYTES.get(dom), "kernel_ms": kern, "step_ms_profiled": prof["step"],
                     "profiled_steps": nprof, "pairs_per_step": pairs_per_step,
                     "tests_per_step": prof.get("tests_per_step")})
    floor_bytes = PARTICLE_BYTES * n + 8.0 * G * s
    step_floor = {"bytes_per_step": floor_bytes, "achieved_GBps": floor_bytes / (ms_per_step * 1e-3) / 1e9,
                  "frac": floor_bytes / (ms_per_step * 1e-3) / 1e9 / hbm}

    # end to end through the C ABI with host buffers: every step uploads the
    # state from pinned host memory, steps, and reads the positions back
    e2e = None
    if not args.no_e2e:
        pos_h = torch.from_numpy(pos.copy()).pin_memory()
        sp_h = torch.from_numpy(sp.copy()).pin_memory()
        reset()
        k_e2e = min(args.steps, RUN_STEPS)
        for _ in range(3):
            chemo.chemo_write_state(sim, pos_h, sp_h, stream=stream)
            chemo.chemo_step(sim, stream=stream)
            chemo.chemo_read_state(sim, pos_h, sp_h, stream=stream)
        pos_h.copy_(torch.from_numpy(pos))
        sp_h.copy_(torch.from_numpy(sp))
        reset()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            chemo.chemo_write_state(sim, pos_h, sp_h, stream=stream)
            chemo.chemo_step(sim, stream=stream)
            chemo.chemo_read_state(sim, pos_h, sp_h, stream=stream)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        tt = torch.tensor([el], dtype=torch.float64, device=devc)
        if dist is not None:
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e = {"value": n * k_e2e * world / float(tt.item()), "unit": UNIT,
               "h2d_bytes_per_step": int(pos_h.numel() * 4 + sp_h.numel()),
               "d2h_bytes_per_step": int(pos_h.numel() * 4 + sp_h.numel()), "steps": k_e2e,
               "how": "per step: chemo_write_state from pinned host (positions + species), chemo_step, "
                      "chemo_read_state to pinned host; the chemical grid stays on the device"}
    sim.close()

    variants = None
    if rank == 0 and not args.no_variants:
        variants = variants_leg(chemo, wl, devc, stream)

    slab_runs = None
    if rank == 0 and world == 1 and not args.no_slabs:
        slab_runs = slabs_leg(chemo, wl)

    ensemble = None
    if not args.no_ensemble:
        ensemble = ensemble_leg(chemo, wl, devc, stream, rank, world, dist, barrier)

    # adjoint / forward time of the differentiable workload (2D, 50k cells,
    # 512^2 grid with 12 PDE substeps, 200 steps, checkpoints every 20)
    adjoint = None
    if rank == 0 and not args.no_adjoint:
        adjoint = adjoint_ratio(chemo, wl, devc, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu = cpu_baseline_full(p, pos, sp)
        except Exception as exc:  # the baseline must not sink the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": oracle_threads(), "kind": "oracle",
                   "sample": "failed: %s" % exc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(p, n), parallelism="replicas x%d (independent seeds)" % world),
            "roofline": roofline, "step_floor": step_floor, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(args.steps * per_step + resets_in * reset_launches),
            "clocks": clock_rec,
            "pair_interactions_per_s": pairs_per_step * world / (ms_per_step * 1e-3),
            "adjoint": adjoint,
            "ensemble": ensemble,
            "variants": variants,
            "slabs": slab_runs,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
