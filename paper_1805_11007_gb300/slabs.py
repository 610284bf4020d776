"""Slab decomposition of one 3D system along z.

The system (reflecting walls, a grid of g[2] node planes at spacing h) is cut
at node planes P_0 = 0 < P_1 < ... < P_K = g[2] - 1. Slab k owns

* the cells with Z_k <= z < Z_{k+1}, Z_k = lo + P_k h (the first slab from
  -inf, the last to +inf: the walls keep every cell in the box), and
* the node planes P_k .. P_{k+1} - 1 (the last slab also the wall plane).

Its sub-domain simulation (``chemo_create_subdomain``) covers the node planes
P_k - H .. P_{k+1} - 1 + H, clipped at the walls: H halo planes beyond each
inner face, which is open (no reflection there). One step of the paper
(Sect. 3: interaction, drift, move, deposit, PDE) then runs as

1. particles (``chemo_step_particles``): pair force on the own cells from own
   cells and ghosts (copies of the neighbours' cells within the largest
   cutoff of a face: the neighbourhood of Sect. 2.2), gradient, move,
   re-binning, cloud-in-cell deposit into the source grids; ghosts are
   neither moved nor deposited (their owners do both);
2. fold: what the own cells deposited on halo planes is added to the planes'
   owner (source and consumption grids);
3. with several PDE substeps, the owners' source planes are copied into the
   neighbours' halo as well;
4. field (``chemo_step_field``): the PDE substeps on the sub-domain's grid;
   the rows next to a cut see the wrong boundary rule, and that error moves
   one plane per substep, so with H >= substeps the owned planes stay exact;
5. halo: c on the owner's planes is copied into the neighbours' halo planes;
6. cells (``chemo_slab_select`` / ``chemo_slab_ingest``): every sub-domain
   selects its own cells for itself and both neighbours (z in the receiver's
   slab widened by the ghost width; those outside the receiver's own range
   as ghosts), the sets are exchanged and each sub-domain ingests its own
   set and the two it received. Cells that stepped over a face migrate here.

The noise is keyed by the cells' ids (carried in the records) and the step
index, and the pair sums are exact, so the decomposed run takes the steps of
the single-domain run; the fields differ by the order of the float additions
of the deposit (and the grid positions by the rounding of a sub-domain's
origin).

``SlabLayout`` and ``initial_records`` are host logic. ``SlabRun`` runs the
step over the sub-domains this process holds: all of them on one GPU
(``LocalExchange``: one CUDA stream per slab, events between them), or one
per rank of a torch.distributed group (``DistExchange``: point-to-point
send/recv, staged through host memory when the backend is gloo).
"""
from __future__ import annotations

import math

import numpy as np

from . import chemo

INF = np.float32(np.inf)


def resolved_substeps(params: dict) -> int:
    """PDE substeps per step: pde_substeps, else the stability rule of the
    explicit scheme (sum over axes of 2 D_c dt / h_a^2 at most 0.9 per
    substep), as the library resolves them."""
    s = int(params.get("pde_substeps", 0) or 0)
    if s > 0:
        return s
    lam = 0.0
    for a in range(int(params["dim"])):
        h = (float(params["hi"][a]) - float(params["lo"][a])) / (int(params["grid"][a]) - 1)
        lam += 2.0 * float(params["Dc"]) * float(params["dt"]) / (h * h)
    return max(1, int(math.ceil(lam / 0.9)))


def max_cutoff(params: dict) -> float:
    d = [float(v) for v in params["diameter"][: int(params["n_species"])]]
    return float(params.get("cutoff_factor", 1.0)) * max(0.5 * (a + b) for a in d for b in d)


class SlabLayout:
    """Cut planes, halo width, the sub-domains' parameters and the z ranges
    of ownership and selection (host logic only).

    planes: the K - 1 inner cut planes (node indices), else cut where the
    cells given as z fall into K equal shares (else equal plane counts).
    halo_planes: H, else max(2, substeps, ceil(max(ghost width, 10 sigma +
    max_drift) / h) + 1), sigma the largest noise amplitude sqrt(2 D dt) and
    max_drift the largest drift displacement dt |F + chi grad c| a step is
    expected to take (0 unless given): a cell may step at most (H - 1) h
    beyond a face (further is clamped and latched as EDOMAIN)."""

    def __init__(self, params: dict, nslabs: int, planes=None, halo_planes=None, z=None, max_drift=0.0):
        p = params
        if int(p["dim"]) != 3 or int(p.get("boundary", 0)) != 0 or int(p.get("chem_mode", 0)) != 0:
            raise ValueError("a slab decomposition needs a 3D system with walls and a grid")
        if nslabs < 1:
            raise ValueError("nslabs must be >= 1")
        self.params = dict(p)
        self.K = int(nslabs)
        self.g = int(p["grid"][2])
        self.lo = float(p["lo"][2])
        self.hi = float(p["hi"][2])
        self.h = (self.hi - self.lo) / (self.g - 1)
        self.substeps = resolved_substeps(p)
        self.ghost_width = 1.01 * max_cutoff(p)
        ns = int(p["n_species"])
        sigma = max(math.sqrt(2.0 * float(D) * float(p["dt"])) for D in p["D"][:ns])
        if halo_planes is None:
            reach = max(self.ghost_width, 10.0 * sigma + float(max_drift))
            halo_planes = max(2, self.substeps, int(math.ceil(reach / self.h)) + 1)
        self.H = int(halo_planes)
        # the sub-domain's box reaches (H - 1) h beyond a face: ghosts within
        # the ghost width and own cells that step over the face must fit
        if self.H < max(2, self.substeps) or (self.H - 1) * self.h < self.ghost_width:
            raise ValueError("halo of %d planes is too thin (needs >= 2, >= substeps and (H - 1) h >= the "
                             "ghost width)" % self.H)
        if planes is None:
            planes = self._balanced(z) if z is not None else [round(k * (self.g - 1) / self.K)
                                                              for k in range(1, self.K)]
        P = [0] + [int(v) for v in planes] + [self.g - 1]
        if len(P) != self.K + 1:
            raise ValueError("need %d inner cut planes" % (self.K - 1))
        if self.K > 1 and any(P[k + 1] - P[k] < self.H for k in range(self.K)):
            raise ValueError("every slab needs at least H = %d node planes (cuts %s)" % (self.H, P))
        self.P = P

    def _balanced(self, z):
        """Inner cuts at the planes nearest the K-quantiles of z, then pushed
        apart to keep every slab at least H planes thick."""
        zs = np.sort(np.asarray(z, np.float64))
        cuts = []
        for k in range(1, self.K):
            if len(zs):
                q = zs[min(len(zs) - 1, (k * len(zs)) // self.K)]
            else:
                q = self.lo + k * (self.hi - self.lo) / self.K
            cuts.append(int(round((q - self.lo) / self.h)))
        lo_min = self.H
        for k in range(len(cuts)):
            cuts[k] = max(cuts[k], lo_min)
            lo_min = cuts[k] + self.H
        hi_max = self.g - 1 - self.H
        for k in reversed(range(len(cuts))):
            cuts[k] = min(cuts[k], hi_max)
            hi_max = cuts[k] - self.H
        return cuts

    # node planes -------------------------------------------------------
    def local_planes(self, k):
        """(q0, q1): first and last global node plane of sub-domain k's grid."""
        q0 = max(0, self.P[k] - self.H)
        q1 = self.g - 1 if k == self.K - 1 else min(self.g - 1, self.P[k + 1] - 1 + self.H)
        return q0, q1

    def owned_planes(self, k):
        """[a, b): global node planes owned by slab k."""
        return self.P[k], (self.g if k == self.K - 1 else self.P[k + 1])

    def shared(self, a, b):
        """[lo, hi): global planes of sub-domain a's grid owned by slab b."""
        q0, q1 = self.local_planes(a)
        o0, o1 = self.owned_planes(b)
        return max(q0, o0), min(q1 + 1, o1)

    def neighbours(self, k):
        return [j for j in (k - 1, k + 1) if 0 <= j < self.K]

    def open_faces(self, k):
        q0, q1 = self.local_planes(k)
        return (chemo.OPEN_ZLO if q0 > 0 else 0) | (chemo.OPEN_ZHI if q1 < self.g - 1 else 0)

    def local_params(self, k):
        q0, q1 = self.local_planes(k)
        p = dict(self.params)
        lo, hi, grid = list(p["lo"]), list(p["hi"]), list(p["grid"])
        lo[2] = self.lo if q0 == 0 else self.lo + q0 * self.h
        hi[2] = self.hi if q1 == self.g - 1 else self.lo + q1 * self.h
        grid[2] = q1 - q0 + 1
        p["lo"], p["hi"], p["grid"] = lo, hi, grid
        p["pde_substeps"] = self.substeps
        return p

    # z ranges (float32, the precision of the positions) ------------------
    def own_range(self, k):
        z0 = -INF if k == 0 else np.float32(self.lo + self.P[k] * self.h)
        z1 = INF if k == self.K - 1 else np.float32(self.lo + self.P[k + 1] * self.h)
        return z0, z1

    def select_range(self, k):
        """Cells that sub-domain k holds: its own range widened by the ghost width."""
        z0, z1 = self.own_range(k)
        w = np.float32(self.ghost_width)
        return (z0 if k == 0 else np.float32(z0 - w)), (z1 if k == self.K - 1 else np.float32(z1 + w))

    def target(self, k):
        """(z0, z1, own0, own1) of sub-domain k as a selection target."""
        s0, s1 = self.select_range(k)
        o0, o1 = self.own_range(k)
        return float(s0), float(s1), float(o0), float(o1)


def make_tags(ids, species):
    return (np.asarray(ids, np.uint32) & np.uint32(chemo.GHOST_ID)) | \
        (np.asarray(species, np.uint32) << np.uint32(chemo.SPECIES_SHIFT))


def initial_records(layout: SlabLayout, pos, species, disp=None, ids=None):
    """The records each sub-domain ingests first (host logic): own cells
    with their ids, ghosts with GHOST_ID."""
    pos = np.asarray(pos, np.float32)
    n = pos.shape[0]
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.asarray(ids, np.uint32)
    if n and int(ids.max()) >= chemo.GHOST_ID:
        raise ValueError("ids must be below GHOST_ID")
    sp = np.asarray(species, np.uint32)
    z = pos[:, 2]
    out = []
    for k in range(layout.K):
        s0, s1 = layout.select_range(k)
        o0, o1 = layout.own_range(k)
        m = (z >= s0) & (z < s1)
        own = (z >= o0) & (z < o1)
        r = np.zeros(int(m.sum()), chemo.CELL_DTYPE)
        r["x"], r["y"], r["z"] = pos[m, 0], pos[m, 1], pos[m, 2]
        ghost_tags = make_tags(np.full(int(m.sum()), chemo.GHOST_ID), sp[m])
        r["tag"] = np.where(own[m], make_tags(ids[m], sp[m]), ghost_tags)
        if disp is not None:
            d = np.asarray(disp, np.float32)
            r["dx"], r["dy"], r["dz"] = d[m, 0], d[m, 1], d[m, 2]
        out.append(r)
    return out


# ---------------------------------------------------------------------------
# One sub-domain on the GPU
# ---------------------------------------------------------------------------
class Subdomain:
    """Sub-domain k of a layout: the library simulation and its exchange
    buffers (device memory, allocated once). Every device operation runs on
    the sub-domain's stream."""

    SRC, CONS = 1, 2  # chemo_slab_planes grid indices

    def __init__(self, layout: SlabLayout, k: int, capacity: int, stream=None):
        import torch
        self.torch = torch
        self.layout, self.k = layout, k
        self.stream = stream
        self.capacity = int(capacity)
        self.sim = chemo.chemo_create_subdomain(layout.local_params(k), self.capacity, layout.open_faces(k),
                                                stream=stream)
        p = layout.params
        self.plane = int(p["grid"][0]) * int(p["grid"][1])
        self.q0 = layout.local_planes(k)[0]
        self.sides = [k] + layout.neighbours(k)  # selection targets: itself, then its neighbours
        dev = torch.device("cuda")
        nb = layout.neighbours(k)
        with torch.cuda.stream(stream):
            self.sel = {j: torch.empty((self.capacity, chemo.CELL_FLOATS), dtype=torch.float32, device=dev)
                        for j in self.sides}
            self.cnt = torch.zeros((len(self.sides), 2), dtype=torch.int64, device=dev)
            self.inbuf = torch.empty((self.capacity, chemo.CELL_FLOATS), dtype=torch.float32, device=dev)
            self.fold_buf = {j: self._planes_buf(layout.shared(k, j), 2) for j in nb}
            self.halo_buf = {j: self._planes_buf(layout.shared(j, k), 1) for j in nb}
            self.src_buf = {j: self._planes_buf(layout.shared(j, k), 2) for j in nb}
            self.fold_in_buf = {j: self._planes_buf(layout.shared(j, k), 2) for j in nb}
            self.halo_in_buf = {j: self._planes_buf(layout.shared(k, j), 1) for j in nb}
            self.src_in_buf = {j: self._planes_buf(layout.shared(k, j), 2) for j in nb}

    def _planes_buf(self, rng, m):
        return self.torch.empty((m, max(rng[1] - rng[0], 0), self.plane), dtype=self.torch.float32,
                                device="cuda")

    def _planes(self, grid, op, rng, buf):
        a, b = rng
        if b > a:
            chemo.chemo_slab_planes(self.sim, grid, op, a - self.q0, b - a, buf, stream=self.stream)

    # step halves
    def step_particles(self):
        chemo.chemo_step_particles(self.sim, stream=self.stream)

    def step_field(self):
        chemo.chemo_step_field(self.sim, stream=self.stream)

    # grid exchanges: out -> the buffer sent to j; in -> apply what j sent
    def fold_out(self, j):
        b = self.fold_buf[j]
        rng = self.layout.shared(self.k, j)
        self._planes(self.SRC, chemo.PLANES_READ, rng, b[0])
        self._planes(self.CONS, chemo.PLANES_READ, rng, b[1])
        return b

    def fold_in(self, j, b):
        rng = self.layout.shared(j, self.k)
        self._planes(self.SRC, chemo.PLANES_ADD, rng, b[0])
        self._planes(self.CONS, chemo.PLANES_ADD, rng, b[1])

    def src_out(self, j):
        b = self.src_buf[j]
        rng = self.layout.shared(j, self.k)
        self._planes(self.SRC, chemo.PLANES_READ, rng, b[0])
        self._planes(self.CONS, chemo.PLANES_READ, rng, b[1])
        return b

    def src_in(self, j, b):
        rng = self.layout.shared(self.k, j)
        self._planes(self.SRC, chemo.PLANES_WRITE, rng, b[0])
        self._planes(self.CONS, chemo.PLANES_WRITE, rng, b[1])

    def halo_out(self, j):
        b = self.halo_buf[j]
        self._planes(0, chemo.PLANES_READ, self.layout.shared(j, self.k), b[0])
        return b

    def halo_in(self, j, b):
        self._planes(0, chemo.PLANES_WRITE, self.layout.shared(self.k, j), b[0])

    # cells
    def select(self):
        with self.torch.cuda.stream(self.stream):  # cleared in the order of the selection
            self.cnt.zero_()
        targets = [self.layout.target(j) + (self.sel[j], self.cnt[i]) for i, j in enumerate(self.sides)]
        chemo.chemo_slab_select(self.sim, targets, stream=self.stream)

    def ingest(self, n):
        chemo.chemo_slab_ingest(self.sim, self.inbuf, n=n, stream=self.stream)

    def write_field(self, c_local):
        with self.torch.cuda.stream(self.stream):
            c = self.torch.as_tensor(np.ascontiguousarray(c_local, np.float32)).cuda()
            chemo.chemo_write_field(self.sim, c, stream=self.stream)

    def read_own_field(self):
        """c on the owned planes, (planes, g[1], g[0]) on the host."""
        a, b = self.layout.owned_planes(self.k)
        p = self.layout.params
        with self.torch.cuda.stream(self.stream):
            buf = self.torch.empty((b - a, self.plane), dtype=self.torch.float32, device="cuda")
            self._planes(0, chemo.PLANES_READ, (a, b), buf)
            return buf.cpu().numpy().reshape(b - a, int(p["grid"][1]), int(p["grid"][0]))

    def read_own_cells(self):
        """The own cells as host records (one selection over everything)."""
        with self.torch.cuda.stream(self.stream):
            out = self.torch.empty((max(self.sim.n, 1), chemo.CELL_FLOATS), dtype=self.torch.float32,
                                   device="cuda")
            cnt = self.torch.zeros(2, dtype=self.torch.int64, device="cuda")
            chemo.chemo_slab_select(self.sim, [(-np.inf, np.inf, -np.inf, np.inf, out, cnt)],
                                    stream=self.stream)
            n = int(cnt[0].item())
            return out[:n].cpu().numpy().view(chemo.CELL_DTYPE).reshape(n)

    def check(self):
        chemo.chemo_check(self.sim, stream=self.stream)

    def close(self):
        self.sim.close()


# ---------------------------------------------------------------------------
# Exchanges between sub-domains
# ---------------------------------------------------------------------------
class LocalExchange:
    """Every sub-domain in this process (one GPU): a message is the sender's
    buffer itself; the receiver's stream waits for an event recorded on the
    sender's stream after the buffer was written."""

    def __init__(self, subs):
        import torch
        self.torch = torch
        self.subs = subs

    def mine(self):
        return sorted(self.subs)

    def deliver(self, msgs):
        """msgs {(src, dst): tensor} -> {(src, dst): tensor} usable on dst's stream."""
        ev = {}
        for (src, _dst) in msgs:
            if src not in ev and self.subs[src].stream is not None:
                e = self.torch.cuda.Event()
                e.record(self.subs[src].stream)
                ev[src] = e
        for (src, dst) in msgs:
            if src in ev and self.subs[dst].stream is not None:
                self.subs[dst].stream.wait_event(ev[src])
        return dict(msgs)

    def counts(self, local):
        """local {(src, dst): (n, n_owned)} -> the same for every pair (all local)."""
        return dict(local)

    def cells(self, sends, recv_into):
        """sends {(src, dst): tensor of n rows}; recv_into {(src, dst): tensor slice}:
        copies on the receiver's stream (after the sender's selection)."""
        self.deliver(sends)
        for key, dst_t in recv_into.items():
            if not dst_t.shape[0]:
                continue
            st = self.subs[key[1]].stream
            if st is None:
                dst_t.copy_(sends[key])
            else:
                with self.torch.cuda.stream(st):
                    dst_t.copy_(sends[key])

    def synchronize(self):
        if self.torch.cuda.is_available() and self.torch.cuda.is_initialized():
            self.torch.cuda.synchronize()


class DistExchange:
    """One sub-domain per rank of a torch.distributed group (slab k on rank
    k): messages go point to point to the neighbouring ranks. NCCL sends
    device tensors; with the gloo backend they are staged through host
    memory (the CPU tests run the whole exchange this way)."""

    def __init__(self, subs, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.subs = subs
        self.group = group
        self.rank = dist.get_rank(group)
        self.stage = dist.get_backend(group) == "gloo"
        self.dev = "cpu" if self.stage else "cuda"  # where small host values travel
        if list(subs) != [self.rank]:
            raise ValueError("DistExchange holds exactly this rank's sub-domain")

    def mine(self):
        return [self.rank]

    def _on_stream(self):
        """Context running device work on this rank's sub-domain stream (NCCL
        orders its transfers against the current stream, and the staged
        copies must precede the sub-domain's own kernels)."""
        st = self.subs[self.rank].stream
        if st is None:
            import contextlib
            return contextlib.nullcontext()
        return self.torch.cuda.stream(st)

    def _sendrecv(self, sends, recvs):
        """sends {peer: tensor}, recvs {peer: tensor to fill} in one batch."""
        torch, dist = self.torch, self.dist
        with self._on_stream():
            ops, land = [], []
            for peer, t in sorted(sends.items()):
                src = t.cpu() if (self.stage and t.is_cuda) else t
                ops.append(dist.P2POp(dist.isend, src.contiguous(), peer, self.group))
            for peer, t in sorted(recvs.items()):
                dst = torch.empty(t.shape, dtype=t.dtype) if (self.stage and t.is_cuda) else t
                land.append((t, dst))
                ops.append(dist.P2POp(dist.irecv, dst, peer, self.group))
            if ops:
                for req in dist.batch_isend_irecv(ops):
                    req.wait()
            for t, dst in land:
                if dst is not t:
                    t.copy_(dst)

    @staticmethod
    def _recv_buffer(sub, peer, sent):
        """Receive buffer for the plane message of `peer`: the in-buffer of
        the same kind as the one sent."""
        for out_name, in_name in (("fold_buf", "fold_in_buf"), ("halo_buf", "halo_in_buf"),
                                  ("src_buf", "src_in_buf")):
            if getattr(sub, out_name)[peer] is sent:
                return getattr(sub, in_name)[peer]
        raise ValueError("unknown message buffer")

    def deliver(self, msgs):
        me = self.rank
        sub = self.subs[me]
        if sub.stream is not None:
            sub.stream.synchronize()
        sends = {dst: t for (src, dst), t in msgs.items() if src == me}
        recvs = {peer: self._recv_buffer(sub, peer, t) for peer, t in sends.items()}
        self._sendrecv(sends, recvs)
        return {(peer, me): t for peer, t in recvs.items()}

    def counts(self, local):
        me = self.rank
        sends = {dst: self.torch.tensor(list(v), dtype=self.torch.int64, device=self.dev)
                 for (src, dst), v in local.items() if src == me and dst != me}
        recvs = {peer: self.torch.zeros(2, dtype=self.torch.int64, device=self.dev) for peer in sends}
        self._sendrecv(sends, recvs)
        out = dict(local)
        for peer, t in recvs.items():
            out[(peer, me)] = (int(t[0]), int(t[1]))
        return out

    def cells(self, sends, recv_into):
        me = self.rank
        sub = self.subs[me]
        if sub.stream is not None:
            sub.stream.synchronize()
        if recv_into[(me, me)].shape[0]:
            with self._on_stream():
                recv_into[(me, me)].copy_(sends[(me, me)])
        s = {dst: t for (src, dst), t in sends.items() if src == me and dst != me and t.shape[0]}
        r = {src: t for (src, dst), t in recv_into.items() if dst == me and src != me and t.shape[0]}
        self._sendrecv(s, r)

    def synchronize(self):
        if self.torch.cuda.is_available() and self.torch.cuda.is_initialized():
            self.torch.cuda.synchronize()


# ---------------------------------------------------------------------------
# The decomposed run
# ---------------------------------------------------------------------------
class SlabRun:
    """Steps the sub-domains `subs` ({k: Subdomain}) of `layout` through
    `exchange`. total: the number of cells of the whole system (checked
    after every step: each cell owned by exactly one sub-domain)."""

    def __init__(self, layout: SlabLayout, subs: dict, exchange, total: int):
        self.layout, self.subs, self.ex, self.total = layout, subs, exchange, int(total)
        self.steps = 0

    def step(self):
        L, subs, ex = self.layout, self.subs, self.ex
        mine = ex.mine()
        for k in mine:
            subs[k].step_particles()
        got = ex.deliver({(k, j): subs[k].fold_out(j) for k in mine for j in L.neighbours(k)})
        for (j, k), t in got.items():
            subs[k].fold_in(j, t)
        if L.substeps > 1:
            got = ex.deliver({(k, j): subs[k].src_out(j) for k in mine for j in L.neighbours(k)})
            for (j, k), t in got.items():
                subs[k].src_in(j, t)
        for k in mine:
            subs[k].step_field()
        got = ex.deliver({(k, j): subs[k].halo_out(j) for k in mine for j in L.neighbours(k)})
        for (j, k), t in got.items():
            subs[k].halo_in(j, t)
        for k in mine:
            subs[k].select()
        ex.synchronize()
        local = {}
        for k in mine:
            c = subs[k].cnt.cpu().tolist()
            for i, j in enumerate(subs[k].sides):
                local[(k, j)] = (int(c[i][0]), int(c[i][1]))
                if c[i][0] > subs[k].capacity:
                    raise chemo.ChemoError(chemo.EOVERFLOW, "slab exchange",
                                           "slab %d selected %d cells for slab %d (capacity %d)"
                                           % (k, c[i][0], j, subs[k].capacity))
        counts = ex.counts(local)
        owned = self._owned_total(counts, mine)
        if owned != self.total:
            raise chemo.ChemoError(chemo.EDOMAIN, "slab exchange",
                                   "%d cells owned after the exchange, expected %d" % (owned, self.total))
        sends, recv_into, n_in = {}, {}, {}
        for k in mine:
            off = 0
            for j in [k] + L.neighbours(k):
                n = counts[(j, k)][0]
                if off + n > subs[k].capacity:
                    raise chemo.ChemoError(chemo.EOVERFLOW, "slab exchange",
                                           "slab %d would hold more than its capacity %d" % (k, subs[k].capacity))
                recv_into[(j, k)] = subs[k].inbuf[off:off + n]
                off += n
            n_in[k] = off
            for j in [k] + L.neighbours(k):
                sends[(k, j)] = subs[k].sel[j][:counts[(k, j)][0]]
        ex.cells(sends, recv_into)
        for k in mine:
            subs[k].ingest(n_in[k])
        ex.synchronize()
        self.steps += 1

    def _owned_total(self, counts, mine):
        """Cells owned by the sub-domains of this process after the exchange,
        summed over the group when distributed."""
        s = sum(counts[(j, k)][1] for k in mine for j in [k] + self.layout.neighbours(k))
        if isinstance(self.ex, DistExchange):
            t = self.ex.torch.tensor([s], dtype=self.ex.torch.int64, device=self.ex.dev)
            self.ex.dist.all_reduce(t, group=self.ex.group)
            s = int(t[0])
        return s

    def step_n(self, nsteps: int):
        for _ in range(int(nsteps)):
            self.step()
        for k in self.ex.mine():
            self.subs[k].check()


def create_local(params: dict, pos, species, nslabs: int, c0=None, planes=None, halo_planes=None,
                 capacity=None, balance=True, streams=True, max_drift=0.0):
    """All slabs of one system as sub-domains on the current GPU, each on its
    own stream (host arrays in). Returns the SlabRun; close_run closes its
    sub-domains."""
    import torch
    pos = np.asarray(pos, np.float32)
    layout = SlabLayout(params, nslabs, planes=planes, halo_planes=halo_planes,
                        z=pos[:, 2] if (balance and planes is None) else None, max_drift=max_drift)
    recs = initial_records(layout, pos, species)
    cap = int(capacity) if capacity else max(1, pos.shape[0])
    subs = {}
    try:
        for k in range(layout.K):
            st = torch.cuda.Stream() if streams else None
            subs[k] = Subdomain(layout, k, cap, stream=st)
            chemo.chemo_slab_ingest(subs[k].sim, recs[k], stream=st)
            if c0 is not None:
                q0, q1 = layout.local_planes(k)
                subs[k].write_field(np.asarray(c0, np.float32)[q0:q1 + 1])
        torch.cuda.synchronize()
    except BaseException:
        for sub in subs.values():
            sub.close()
        raise
    return SlabRun(layout, subs, LocalExchange(subs), pos.shape[0])


def gather_state(run: SlabRun):
    """(pos (N, 3), species (N,), disp (N, 3), ids (N,)) in id order, from the
    own cells of every sub-domain of this process (all of them for a local
    run)."""
    recs = np.concatenate([run.subs[k].read_own_cells() for k in run.ex.mine()])
    ids = recs["tag"] & np.uint32(chemo.GHOST_ID)
    order = np.argsort(ids, kind="stable")
    r = recs[order]
    pos = np.stack([r["x"], r["y"], r["z"]], axis=1)
    disp = np.stack([r["dx"], r["dy"], r["dz"]], axis=1)
    return pos, (r["tag"] >> np.uint32(chemo.SPECIES_SHIFT)).astype(np.uint8), disp, ids[order]


def gather_field(run: SlabRun):
    """The whole field (g[2], g[1], g[0]) from the owned planes of every
    sub-domain of this process (all of them for a local run)."""
    return np.concatenate([run.subs[k].read_own_field() for k in run.ex.mine()])


def close_run(run: SlabRun):
    for sub in run.subs.values():
        sub.close()
