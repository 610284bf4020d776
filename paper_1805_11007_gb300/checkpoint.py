"""Checkpoint files of a simulation, built on the C ABI's state calls.

A checkpoint holds what a run needs to continue bit for bit: the state by
particle id (positions, species and, when tracked, the unwrapped
displacement), the chemical field, the absolute step index (the noise is
keyed by (id, step)), the replicate sizes and the model parameters. It is
one ``.npz`` file: arrays as arrays, the parameters as JSON.

    save_sim(sim, "run.npz")          # chemo_read_state / read_field / step_index
    sim2 = load_sim("run.npz")        # chemo_create(_batch) / write_state / write_field / set_step_index

``snapshot`` / ``restore`` do the same with an in-memory dict (host arrays).
"""
from __future__ import annotations

import json

import numpy as np

from . import chemo

FORMAT = 1


def _jsonable(o):
    if hasattr(o, "tolist"):
        return o.tolist()
    raise TypeError("parameter value %r is not serialisable" % (o,))


def snapshot(sim: chemo.Sim) -> dict:
    """The simulation's state as host arrays (synchronises its stream)."""
    pos, species, disp = chemo.read_state_host(sim)
    snap = {
        "format": FORMAT,
        "params": dict(sim.params),
        "sizes": [int(v) for v in sim.sizes],
        "step": int(chemo.chemo_step_index(sim)),
        "pos": pos,
        "species": species,
    }
    if disp is not None:
        snap["disp"] = disp
    if int(sim.params.get("chem_mode", 0)) == 0:
        snap["c"] = chemo.read_field_host(sim)
    return snap


def restore(snap: dict, stream=None) -> chemo.Sim:
    """A new simulation that continues the run of a snapshot."""
    if int(snap.get("format", -1)) != FORMAT:
        raise ValueError("unknown checkpoint format %r" % (snap.get("format"),))
    p = snap["params"]
    sizes = [int(v) for v in snap["sizes"]]
    pos = np.ascontiguousarray(snap["pos"], dtype=np.float32)
    species = np.ascontiguousarray(snap["species"], dtype=np.uint8)
    if len(sizes) > 1:
        sim = chemo.chemo_create_batch(p, sizes, pos, species, stream=stream)
    else:
        sim = chemo.chemo_create(p, pos, species, stream=stream)
    try:
        if snap.get("disp") is not None:
            chemo.chemo_write_state(sim, pos, species, np.ascontiguousarray(snap["disp"], dtype=np.float32),
                                    stream=stream)
        if snap.get("c") is not None:
            chemo.chemo_write_field(sim, np.ascontiguousarray(snap["c"], dtype=np.float32), stream=stream)
        chemo.chemo_set_step_index(sim, int(snap["step"]), stream=stream)
    except Exception:
        sim.close()
        raise
    return sim


def save(path, snap: dict) -> None:
    """Writes a snapshot to an .npz file."""
    arrays = {
        "format": np.int64(snap.get("format", FORMAT)),
        "params": np.array(json.dumps(snap["params"], default=_jsonable)),
        "sizes": np.asarray(snap["sizes"], dtype=np.int64),
        "step": np.int64(snap["step"]),
        "pos": np.asarray(snap["pos"], dtype=np.float32),
        "species": np.asarray(snap["species"], dtype=np.uint8),
    }
    for k in ("disp", "c"):
        if snap.get(k) is not None:
            arrays[k] = np.asarray(snap[k], dtype=np.float32)
    with open(path, "wb") as fh:
        np.savez(fh, **arrays)


def load(path) -> dict:
    """Reads a snapshot written by save."""
    with np.load(path, allow_pickle=False) as z:
        snap = {
            "format": int(z["format"]),
            "params": json.loads(str(z["params"])),
            "sizes": [int(v) for v in z["sizes"]],
            "step": int(z["step"]),
            "pos": z["pos"].copy(),
            "species": z["species"].copy(),
        }
        for k in ("disp", "c"):
            if k in z.files:
                snap[k] = z[k].copy()
    return snap


def save_sim(sim: chemo.Sim, path) -> None:
    save(path, snapshot(sim))


def load_sim(path, stream=None) -> chemo.Sim:
    return restore(load(path), stream=stream)
