"""Runs a named workload for a fixed number of steps, for profilers.

    python -m paper_1805_11007_gb300.profile_run --workload clumps_grid_3d --steps 120 [--graphs 0|1]

Creates the simulation from the workload's seeded initial state (chemical
field zero), advances it ``--steps`` steps (through ``chemo_step`` one launch
sequence at a time, or ``chemo_step_n`` with CUDA graphs) and prints one line
with the elapsed time. The kernels each step launches, in order: ``k_step``
(pair force, drift, move, counts of the next cell list), ``k_scan`` (offsets),
``k_scatter`` (counting sort, fused deposit) and the PDE substeps
(``k_pde_stream``); with ``--workload adjoint_2d --adjoint 1`` the run is
recorded and followed by one ``chemo_gradient``.
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
    p, pos, sp = wl.initial_state(a.workload, n=a.n)
    if a.search_mode is not None:
        p = dict(p, search_mode=a.search_mode)
    dev = torch.device("cuda:0")
    dpos = torch.from_numpy(pos).to(dev)
    dsp = torch.from_numpy(sp).to(dev)
    with chemo.chemo_create(p, dpos, dsp) as sim:
        if p.get("chem_mode", 0) == 0:
            chemo.chemo_write_field(sim, torch.zeros(chemo.grid_shape(p), dtype=torch.float32, device=dev))
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
