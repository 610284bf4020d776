"""A CPU stand-in for a sub-domain (the interface of slabs.Subdomain) with a
toy step that has every dependency of the real one across a slab face:

* a cell's move depends on how many cells lie within the cutoff (own cells
  and ghosts), so a missing or extra ghost changes it;
* the own cells deposit on the two nearest node planes (linear weights in z),
  so deposits land on halo planes and must be folded into their owner;
* the field step is an explicit diffusion along z with `substeps` substeps,
  mirrored at the sub-domain's grid ends, so wrong halo planes reach the
  owned planes unless the halo is refreshed and wide enough.

The same class run as one sub-domain over the whole box is the reference of
the decomposed runs (tests/test_slabs_host.py). Float64 throughout, the
positions float32 as in the records."""
from __future__ import annotations

import numpy as np
import torch

from paper_1805_11007_gb300 import chemo


def _hash_unit(ids, step):
    """A deterministic number in [-1, 1) per (id, step) (an integer hash
    that wraps modulo 2^64)."""
    with np.errstate(over="ignore"):
        x = ids.astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15) + \
            np.full(ids.shape, step, np.uint64) * np.uint64(0xBF58476D1CE4E5B9)
        x ^= x >> np.uint64(31)
        x *= np.uint64(0x94D049BB133111EB)
        x ^= x >> np.uint64(29)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0


class FakeSubdomain:
    def __init__(self, layout, k, capacity, amp=None, push=None):
        self.layout, self.k = layout, k
        self.stream = None
        self.capacity = int(capacity)
        p = layout.params
        self.rc = layout.ghost_width / 1.01
        self.amp = amp if amp is not None else 0.5 * (layout.H - 1) * layout.h
        self.push = push if push is not None else 0.05 * self.rc
        self.q0, self.q1 = layout.local_planes(k)
        self.zlo = np.float32(layout.lo + self.q0 * layout.h) if self.q0 else np.float32(layout.lo)
        self.zhi = np.float32(layout.lo + self.q1 * layout.h) if self.q1 < layout.g - 1 else np.float32(layout.hi)
        self.plane = int(p["grid"][0]) * int(p["grid"][1])
        gz = self.q1 - self.q0 + 1
        self.c = np.zeros((gz, self.plane))
        self.S = np.zeros((gz, self.plane))
        self.R = np.zeros((gz, self.plane))
        self.step_index = 0
        self.rec = np.zeros(0, chemo.CELL_DTYPE)
        self.sides = [k] + layout.neighbours(k)
        self.sel = {j: torch.zeros((self.capacity, chemo.CELL_FLOATS), dtype=torch.float32) for j in self.sides}
        self.cnt = torch.zeros((len(self.sides), 2), dtype=torch.int64)
        self.inbuf = torch.zeros((self.capacity, chemo.CELL_FLOATS), dtype=torch.float32)
        nb = layout.neighbours(k)

        def mk(rng, m):
            return torch.zeros((m, max(rng[1] - rng[0], 0), self.plane), dtype=torch.float64)
        self.fold_buf = {j: mk(layout.shared(k, j), 2) for j in nb}
        self.halo_buf = {j: mk(layout.shared(j, k), 1) for j in nb}
        self.src_buf = {j: mk(layout.shared(j, k), 2) for j in nb}
        self.fold_in_buf = {j: mk(layout.shared(j, k), 2) for j in nb}
        self.halo_in_buf = {j: mk(layout.shared(k, j), 1) for j in nb}
        self.src_in_buf = {j: mk(layout.shared(k, j), 2) for j in nb}

    # state -----------------------------------------------------------------
    def load(self, records, c_local=None):
        self.rec = np.array(records, chemo.CELL_DTYPE)
        if c_local is not None:
            self.c = np.array(c_local, np.float64).reshape(self.c.shape)

    def _ids(self):
        return self.rec["tag"] & np.uint32(chemo.GHOST_ID)

    # step halves -------------------------------------------------------------
    def step_particles(self):
        r = self.rec
        own = self._ids() != chemo.GHOST_ID
        P = np.stack([r["x"], r["y"], r["z"]], axis=1).astype(np.float64)
        d2 = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
        near = (d2 < self.rc ** 2).sum(1) - 1
        ids = self._ids()[own]
        dz = self.amp * _hash_unit(ids, self.step_index) + self.push * near[own] / 16.0
        z = (r["z"][own].astype(np.float64) + dz).astype(np.float32)
        lo, hi = np.float32(self.layout.lo), np.float32(self.layout.hi)
        z = np.where(z < lo, 2 * lo - z, z)  # the system's walls reflect
        z = np.where(z > hi, 2 * hi - z, z)
        if np.any((z < self.zlo) | (z > self.zhi)):
            raise chemo.ChemoError(chemo.EDOMAIN, "fake step", "a cell left the sub-domain's box")
        r["z"][own] = z
        r["dz"][own] += dz.astype(np.float32)
        # deposit: linear weights on the two nearest node planes
        t = (z.astype(np.float64) - (self.layout.lo + self.q0 * self.layout.h)) / self.layout.h
        i0 = np.clip(np.floor(t).astype(np.int64), 0, self.c.shape[0] - 2)
        f = t - i0
        np.add.at(self.S, i0, (1.0 - f)[:, None] * np.ones(self.plane))
        np.add.at(self.S, i0 + 1, f[:, None] * np.ones(self.plane))
        self.R += 0.5 * self.S
        self.step_index += 1

    def step_field(self):
        s = self.layout.substeps
        for _ in range(s):
            up = np.concatenate([self.c[1:2], self.c[:-1]])       # mirror at the grid ends
            dn = np.concatenate([self.c[1:], self.c[-2:-1]])
            self.c = self.c + 0.1 * (up - 2 * self.c + dn) - 0.01 * self.R * self.c + self.S / s
        self.S[:] = 0.0
        self.R[:] = 0.0

    # grid exchanges ----------------------------------------------------------
    def _get(self, g, rng):
        return torch.from_numpy(g[rng[0] - self.q0:rng[1] - self.q0].copy())

    def fold_out(self, j):
        b, rng = self.fold_buf[j], self.layout.shared(self.k, j)
        b[0].copy_(self._get(self.S, rng))
        b[1].copy_(self._get(self.R, rng))
        return b

    def fold_in(self, j, b):
        a, e = self.layout.shared(j, self.k)
        self.S[a - self.q0:e - self.q0] += b[0].numpy()
        self.R[a - self.q0:e - self.q0] += b[1].numpy()

    def src_out(self, j):
        b, rng = self.src_buf[j], self.layout.shared(j, self.k)
        b[0].copy_(self._get(self.S, rng))
        b[1].copy_(self._get(self.R, rng))
        return b

    def src_in(self, j, b):
        a, e = self.layout.shared(self.k, j)
        self.S[a - self.q0:e - self.q0] = b[0].numpy()
        self.R[a - self.q0:e - self.q0] = b[1].numpy()

    def halo_out(self, j):
        b = self.halo_buf[j]
        b[0].copy_(self._get(self.c, self.layout.shared(j, self.k)))
        return b

    def halo_in(self, j, b):
        a, e = self.layout.shared(self.k, j)
        self.c[a - self.q0:e - self.q0] = b[0].numpy()

    # cells -------------------------------------------------------------------
    def select(self):
        self.cnt.zero_()
        own = self.rec[self._ids() != chemo.GHOST_ID]
        for i, j in enumerate(self.sides):
            z0, z1, o0, o1 = (np.float32(v) for v in self.layout.target(j))
            z = own["z"]
            m = own[(z >= z0) & (z < z1)].copy()
            mine = (m["z"] >= o0) & (m["z"] < o1)
            m["tag"] = np.where(mine, m["tag"], m["tag"] | np.uint32(chemo.GHOST_ID))
            n = m.shape[0]
            w = min(n, self.capacity)
            self.sel[j][:w] = torch.from_numpy(m[:w].view(np.float32).reshape(w, chemo.CELL_FLOATS))
            self.cnt[i, 0] = n
            self.cnt[i, 1] = int(mine.sum())

    def ingest(self, n):
        self.rec = self.inbuf[:n].numpy().copy().view(chemo.CELL_DTYPE).reshape(n)

    def check(self):
        pass

    def read_own_cells(self):
        return self.rec[self._ids() != chemo.GHOST_ID].copy()

    def read_own_field(self):
        a, b = self.layout.owned_planes(self.k)
        return self.c[a - self.q0:b - self.q0, 0].copy()

    def close(self):
        pass


def fake_run(layout, pos, species, c0, capacity, exchange_cls, ranks=None, **kw):
    """A SlabRun over FakeSubdomains (those of `ranks`, else all)."""
    from paper_1805_11007_gb300 import slabs
    recs = slabs.initial_records(layout, pos, species)
    subs = {}
    for k in (range(layout.K) if ranks is None else ranks):
        subs[k] = FakeSubdomain(layout, k, capacity, **kw)
        q0, q1 = layout.local_planes(k)
        subs[k].load(recs[k], np.repeat(c0[q0:q1 + 1, None], subs[k].plane, axis=1))
    return slabs.SlabRun(layout, subs, exchange_cls(subs), pos.shape[0])
