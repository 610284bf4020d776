"""Runs a named workload for a fixed number of steps, for profilers.

    python -m paper_1805_11007_gb300.profile_run --workload clumps_grid_3d --steps 120 [--graphs 0|1]

Creates the simulation from the workload's seeded initial state (chemical
field zero), advances it ``--steps`` steps (through ``chemo_step`` one launch
sequence at a time, or ``chemo_step_n`` with CUDA graphs) and prints one line
with the elapsed time. The kernels each step launches, in order: ``k_step``
(pair force, drift, move, counts of the next cell list), ``k_scan`` (offsets),
``k_scatter`` (counting sort, fused deposit) and the PDE substeps
(``k_pde_stream`` / ``k_pde_multi``); with ``--workload adjoint_2d --adjoint 1``
the run is recorded and followed by one ``chemo_gradient``; ``ensemble_2d``
runs its replicates as one batched simulation.
"""
from __future__ import annotations

import argparse
import json
import time

import torch

from . import chemo
from . import workloads as wl


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="clumps_grid_3d", choices=sorted(wl.WORKLOADS))
    ap.add_argument("--steps", type=int, default=120)
    ap.add_argument("--graphs", type=int, default=1)
    ap.add_argument("--adjoint", type=int, default=0)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--search-mode", type=int, default=None)
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("profile_run needs a CUDA device")
    dev = torch.device("cuda:0")
    if wl.WORKLOADS[a.workload].get("replicates"):
        # an ensemble: all replicates in one batched simulation
        p, sizes, pos, sp = wl.ensemble_state(a.workload)
    else:
        p, pos, sp = wl.initial_state(a.workload, n=a.n)
        sizes = None
    if a.search_mode is not None:
        p = dict(p, search_mode=a.search_mode)
    dpos = torch.from_numpy(pos).to(dev)
    dsp = torch.from_numpy(sp).to(dev)
    sim0 = chemo.chemo_create(p, dpos, dsp) if sizes is None else chemo.chemo_create_batch(p, sizes, dpos, dsp)
    with sim0 as sim:
        if p.get("chem_mode", 0) == 0:
            shape = tuple(chemo.grid_shape(p)) if sizes is None else (len(sizes),) + tuple(chemo.grid_shape(p))
            chemo.chemo_write_field(sim, torch.zeros(shape, dtype=torch.float32, device=dev))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if a.adjoint:
            every = int(wl.WORKLOADS[a.workload].get("ckpt_every", 20))
            chemo.chemo_record(sim, a.steps, every)
            g = torch.zeros((sim.n, sim.dim), dtype=torch.float32, device=dev)
            g[:, 0] = 1.0 / max(sim.n, 1)
            dth = torch.zeros(2 + int(p["n_species"]), dtype=torch.float32, device=dev)
            chemo.chemo_gradient(sim, g, dth)
        elif a.graphs:
            chemo.chemo_step_n(sim, a.steps)
        else:
            for _ in range(a.steps):
                chemo.chemo_step(sim)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        chemo.chemo_check(sim)
        info = chemo.chemo_get_info(sim)
        print(json.dumps({"workload": a.workload, "n": int(sim.n), "steps": a.steps, "seconds": el,
                          "launches_per_step": info["launches_per_step"]}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
