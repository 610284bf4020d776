"""ctypes binding of the GB300 chemotaxis-step library (``include/chemo.h``).

Argument marshalling only: every step of the path runs in the CUDA kernels of
``libchemo_gb300.so``. The functions carry the C ABI's names. Buffers may be
CUDA torch tensors (device memory; asynchronous on the given stream) or numpy
arrays / CPU tensors (host memory; the call synchronises). ``stream`` is a
``torch.cuda.Stream``, a raw ``cudaStream_t`` integer, or None (the current
torch stream when torch is loaded, else the legacy default stream).

The library must have been built (``paper_1805_11007_gb300.build.build()`` or
``__graft_entry__.build()``); importing this module without it fails loudly.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import warnings
import weakref

import numpy as np

from . import build as _build

MAXS = 8
OK, EINVAL, ENOMEM, ECUDA, EDOMAIN, ENONFINITE, EOVERFLOW, ETIMEOUT, ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7, -8
MEM_HOST, MEM_DEVICE = 0, 1


class ChemoError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__("%s failed: %s (%d): %s" % (where, _status_text(status), status, msg))
        self.status = status


class chemo_params(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32),
        ("dim", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("diameter", ctypes.c_float * MAXS),
        ("D", ctypes.c_float * MAXS),
        ("chemotactic", ctypes.c_float * MAXS),
        ("secrete", ctypes.c_float * MAXS),
        ("consume", ctypes.c_float * MAXS),
        ("react_k0", ctypes.c_float * MAXS),
        ("react_kc", ctypes.c_float * MAXS),
        ("react_to", ctypes.c_int32 * MAXS),
        ("reactions", ctypes.c_int32),
        ("chi", ctypes.c_float),
        ("inter", ctypes.c_float),
        ("cutoff_factor", ctypes.c_float),
        ("cutoff_mode", ctypes.c_int32),
        ("chem_mode", ctypes.c_int32),
        ("fixed_grad", ctypes.c_float * 3),
        ("grid", ctypes.c_int32 * 3),
        ("Dc", ctypes.c_float),
        ("gamma", ctypes.c_float),
        ("pde_bc", ctypes.c_int32),
        ("pde_substeps", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("track_displacement", ctypes.c_int32),
        ("bin_side", ctypes.c_float),
        ("search_mode", ctypes.c_int32),
        ("bin_order", ctypes.c_int32),
        ("pde_overlap", ctypes.c_int32),
        ("warp_runs", ctypes.c_int32),
        ("move_scheme", ctypes.c_int32),
        ("hard_sphere", ctypes.c_int32),
        ("deposit_kernel", ctypes.c_int32),
        ("kde_range", ctypes.c_float),
        ("block_threads", ctypes.c_int32),
    ]


class chemo_info(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("dim", ctypes.c_int32),
        ("search_mode", ctypes.c_int32),
        ("nbins", ctypes.c_int32 * 3),
        ("bin_slots", ctypes.c_int64),
        ("bin_side", ctypes.c_float * 3),
        ("bin_pitch", ctypes.c_int32),
        ("pde_substeps", ctypes.c_int32),
        ("grid_nodes", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("launches_per_step", ctypes.c_int32),
        ("layers", ctypes.c_int32),
        ("step_ratio", ctypes.c_float),
    ]


# Sub-domains of a z-slab decomposition (include/chemo.h): a cell in transit
# is one 32-byte record, tag = id | species << 29 (id GHOST_ID for a ghost).
CELL_DTYPE = np.dtype([("x", "<f4"), ("y", "<f4"), ("z", "<f4"), ("tag", "<u4"),
                       ("dx", "<f4"), ("dy", "<f4"), ("dz", "<f4"), ("reserved", "<u4")])
CELL_FLOATS = 8
GHOST_ID = 0x1FFFFFFF
SPECIES_SHIFT = 29
OPEN_ZLO, OPEN_ZHI = 1, 2
PLANES_READ, PLANES_WRITE, PLANES_ADD = 0, 1, 2
SLAB_TARGETS = 4


class chemo_slab_target(ctypes.Structure):
    _fields_ = [
        ("z0", ctypes.c_float),
        ("z1", ctypes.c_float),
        ("own0", ctypes.c_float),
        ("own1", ctypes.c_float),
        ("out", ctypes.c_void_p),
        ("capacity", ctypes.c_int64),
        ("count", ctypes.c_void_p),
    ]


def make_params(d: dict) -> chemo_params:
    """chemo_params from a dict keyed by the field names (missing = 0 /
    library defaults; per-species lists may be shorter than 8)."""
    p = chemo_params()
    p.struct_size = ctypes.sizeof(chemo_params)
    p.dim = int(d["dim"])
    p.boundary = int(d.get("boundary", 0))
    for a in range(3):
        p.lo[a] = float(d.get("lo", [0.0] * 3)[a])
        p.hi[a] = float(d.get("hi", [1.0] * 3)[a])
    ns = int(d["n_species"])
    p.n_species = ns
    for name in ("diameter", "D", "chemotactic", "secrete", "consume", "react_k0", "react_kc"):
        vals = list(d.get(name, [0.0] * ns))
        arr = getattr(p, name)
        for s in range(MAXS):
            arr[s] = float(vals[s]) if s < len(vals) else 0.0
    rt = list(d.get("react_to", list(range(ns))))
    for s in range(MAXS):
        p.react_to[s] = int(rt[s]) if s < len(rt) else s
    p.reactions = int(d.get("reactions", 0))
    p.chi = float(d.get("chi", 0.0))
    p.inter = float(d.get("inter", 1.0))
    p.cutoff_factor = float(d.get("cutoff_factor", 1.0))
    p.cutoff_mode = int(d.get("cutoff_mode", 0))
    p.chem_mode = int(d.get("chem_mode", 0))
    fg = list(d.get("fixed_grad", [0.0] * 3))
    for a in range(3):
        p.fixed_grad[a] = float(fg[a]) if a < len(fg) else 0.0
    g = list(d.get("grid", [3, 3, 3]))
    for a in range(3):
        p.grid[a] = int(g[a]) if a < len(g) else 1
    p.Dc = float(d.get("Dc", 0.0))
    p.gamma = float(d.get("gamma", 0.0))
    p.pde_bc = int(d.get("pde_bc", 0))
    p.pde_substeps = int(d.get("pde_substeps", 0))
    p.dt = float(d["dt"])
    p.seed = int(d.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    p.track_displacement = int(d.get("track_displacement", 0))
    p.bin_side = float(d.get("bin_side", 0.0))
    p.search_mode = int(d.get("search_mode", 0))
    p.bin_order = int(d.get("bin_order", 0))
    p.pde_overlap = int(d.get("pde_overlap", 0))
    p.warp_runs = int(d.get("warp_runs", 0))
    p.block_threads = int(d.get("block_threads", 0))
    p.move_scheme = int(d.get("move_scheme", 0))
    p.hard_sphere = int(d.get("hard_sphere", 0))
    p.deposit_kernel = int(d.get("deposit_kernel", 0))
    p.kde_range = float(d.get("kde_range", 0.0))
    return p


_lib = None

# Callbacks of chemo_set_allocator: int alloc(ctx, bytes, void **ptr) and
# void release(ctx, ptr, bytes).
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p))
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t)


def lib():
    """The loaded library (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError("libchemo_gb300.so is not built (run __graft_entry__.build()): %s" % path)
        L = ctypes.CDLL(path)
        _declare(L)
        _lib = L
    return _lib


def _declare(L):
    vp, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    PP = ctypes.POINTER(chemo_params)
    sigs = {
        "chemo_create": ([PP, i64, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "chemo_create_batch": ([PP, i32, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "chemo_autotune": ([PP, i32, vp, vp, vp, ctypes.c_int, i32, vp, PP, ctypes.POINTER(ctypes.c_float)],
                           ctypes.c_int),
        "chemo_write_state": ([vp, vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_write_field": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_step": ([vp, vp], ctypes.c_int),
        "chemo_step_n": ([vp, i64, vp], ctypes.c_int),
        "chemo_read_state": ([vp, vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_read_field": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_record": ([vp, i64, i32, vp], ctypes.c_int),
        "chemo_record_stored": ([vp, i64, i32, i64, vp], ctypes.c_int),
        "chemo_observables": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_init_positions": ([vp, i64, i64, ctypes.c_float, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_histogram": ([vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_gradient": ([vp, vp, vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_set_params": ([vp, PP], ctypes.c_int),
        "chemo_step_index": ([vp], i64),
        "chemo_set_step_index": ([vp, i64, vp], ctypes.c_int),
        "chemo_check": ([vp, vp], ctypes.c_int),
        "chemo_stall_scan": ([vp, ctypes.c_uint32, vp], ctypes.c_int),
        "chemo_get_info": ([vp, ctypes.POINTER(chemo_info)], ctypes.c_int),
        "chemo_destroy": ([vp], None),
        "chemo_status_string": ([ctypes.c_int], ctypes.c_char_p),
        "chemo_last_error": ([], ctypes.c_char_p),
        "chemo_philox": ([ctypes.c_uint64, vp, vp, i64, ctypes.c_int, vp], ctypes.c_int),
        "chemo_profile_steps": ([vp, i64, vp, vp], ctypes.c_int),
        "chemo_stage_bins": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_stage_sort": ([vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_stage_forces": ([vp, vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_stage_drift": ([vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_stage_deposit": ([vp, vp, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_forces_noalloc": ([PP, i64, vp, vp, vp, vp], ctypes.c_int),
        "chemo_create_subdomain": ([PP, i64, ctypes.c_uint32, vp, ctypes.POINTER(vp)], ctypes.c_int),
        "chemo_slab_ingest": ([vp, i64, vp, ctypes.c_int, vp], ctypes.c_int),
        "chemo_slab_select": ([vp, i32, ctypes.POINTER(chemo_slab_target), vp], ctypes.c_int),
        "chemo_slab_planes": ([vp, i32, i32, i64, i64, vp, vp], ctypes.c_int),
        "chemo_step_particles": ([vp, vp], ctypes.c_int),
        "chemo_step_field": ([vp, vp], ctypes.c_int),
        "chemo_set_allocator": ([vp, vp, vp], ctypes.c_int),  # callbacks as pointers (NULL allowed)
    }
    for name, (args, res) in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res


def _status_text(status: int) -> str:
    try:
        return lib().chemo_status_string(int(status)).decode()
    except Exception:
        return "status"


def _check(status: int, where: str):
    if status != OK:
        raise ChemoError(status, where, lib().chemo_last_error().decode())


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _buf(x, dtype):
    """(pointer, mem_kind, keepalive) of an array-like for the C call."""
    if x is None:
        return None, None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                raise ValueError("tensor must be contiguous")
            want = {np.float32: torch.float32, np.uint8: torch.uint8, np.int32: torch.int32,
                    np.uint32: torch.int32, np.uint64: torch.int64}[dtype]
            if x.dtype != want and not (dtype == np.uint32 and x.dtype in (torch.int32, torch.uint32)) and \
                    not (dtype == np.uint64 and x.dtype in (torch.int64, torch.uint64)):
                raise TypeError("tensor dtype %s, expected %s" % (x.dtype, want))
            return ctypes.c_void_p(x.data_ptr()), (MEM_DEVICE if x.is_cuda else MEM_HOST), x
    except ImportError:
        pass
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("numpy buffer must be C-contiguous %s" % np.dtype(dtype))
    return a.ctypes.data_as(ctypes.c_void_p), MEM_HOST, a


def _kind(*kinds):
    ks = {k for k in kinds if k is not None}
    if len(ks) > 1:
        raise ValueError("all buffers of one call must live in the same memory (host or device)")
    return ks.pop() if ks else MEM_HOST


class Sim:
    """Owned handle of a simulation (chemo_destroy on close / garbage; the
    ones still open at interpreter exit are closed while Python callbacks
    of chemo_set_allocator can still run)."""

    def __init__(self, handle, params: dict, n: int, sizes=None):
        self.handle = handle
        _open_sims.add(self)
        self.params = dict(params)
        self.n = int(n)
        self.dim = int(params["dim"])
        # replicate sizes (one entry unless created by chemo_create_batch)
        self.sizes = [int(n)] if sizes is None else [int(v) for v in sizes]
        self.replicates = len(self.sizes)

    def close(self):
        if self.handle:
            lib().chemo_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_open_sims = weakref.WeakSet()


@atexit.register
def _close_open_sims():
    for sim in list(_open_sims):
        try:
            sim.close()
        except Exception:
            pass


def _h(sim):
    if not isinstance(sim, Sim) or not sim.handle:
        raise ValueError("not an open simulation")
    return sim.handle


def chemo_create(params: dict, pos, species, stream=None) -> Sim:
    """Creates a simulation; pos (n, dim) float32, species (n,) uint8, both
    host or both device."""
    pp, kp_, _a = _buf(pos, np.float32)
    sp, ks, _b = _buf(species, np.uint8)
    n = int(np.prod(pos.shape[:1])) if pos is not None else 0
    out = ctypes.c_void_p()
    prm = make_params(params)
    _check(lib().chemo_create(ctypes.byref(prm), n, pp, sp, _kind(kp_, ks), _stream(stream), ctypes.byref(out)),
           "chemo_create")
    sim = Sim(out, params, n)
    _warn_step(sim)
    return sim


def _warn_step(sim):
    """The paper's time-step rule (Sect. 3.2): a step should move a cell less
    than the interaction range."""
    ratio = chemo_get_info(sim)["step_ratio"]
    if ratio > 1.0:
        warnings.warn("dt is large for the interaction range: sqrt(2 (D_i + D_j) dt) / eps_ij = %.3g > 1" % ratio,
                      stacklevel=3)


def chemo_create_batch(params: dict, n_per_replicate, pos, species, stream=None) -> Sim:
    """Creates an ensemble of 2D replicates (replicate r: n_per_replicate[r]
    cells, Philox key seed + r); pos (sum n, 2) and species (sum n,) are the
    replicates' arrays concatenated in replicate order."""
    sizes = np.ascontiguousarray(np.asarray(n_per_replicate, dtype=np.int64).reshape(-1))
    pp, kp_, _a = _buf(pos, np.float32)
    sp, ks, _b = _buf(species, np.uint8)
    out = ctypes.c_void_p()
    prm = make_params(params)
    _check(lib().chemo_create_batch(ctypes.byref(prm), int(sizes.size), sizes.ctypes.data, pp, sp, _kind(kp_, ks),
                                    _stream(stream), ctypes.byref(out)), "chemo_create_batch")
    sim = Sim(out, params, int(sizes.sum()), sizes.tolist())
    _warn_step(sim)
    return sim


def chemo_autotune(params: dict, n_per_replicate, pos, species, trial_steps: int = 20, stream=None):
    """Fastest (bin_side, search_mode, warp_runs, block_threads, pde_overlap)
    for this particle set: returns (params dict with those fields set,
    device ms per step)."""
    sizes = np.ascontiguousarray(np.asarray(n_per_replicate, dtype=np.int64).reshape(-1))
    pp, kp_, _a = _buf(pos, np.float32)
    sp, ks, _b = _buf(species, np.uint8)
    prm = make_params(params)
    best = chemo_params()
    ms = ctypes.c_float(0.0)
    _check(lib().chemo_autotune(ctypes.byref(prm), int(sizes.size), sizes.ctypes.data, pp, sp, _kind(kp_, ks),
                                int(trial_steps), _stream(stream), ctypes.byref(best), ctypes.byref(ms)),
           "chemo_autotune")
    q = dict(params)
    q["bin_side"] = float(best.bin_side)
    q["search_mode"] = int(best.search_mode)
    q["pde_overlap"] = int(best.pde_overlap)
    q["warp_runs"] = int(best.warp_runs)
    q["block_threads"] = int(best.block_threads)
    return q, float(ms.value)


def chemo_write_state(sim: Sim, pos, species, disp=None, stream=None):
    pp, k1, _a = _buf(pos, np.float32)
    sp, k2, _b = _buf(species, np.uint8)
    dp, k3, _c = _buf(disp, np.float32)
    _check(lib().chemo_write_state(_h(sim), pp, sp, dp, _kind(k1, k2, k3), _stream(stream)), "chemo_write_state")


def chemo_write_field(sim: Sim, c, stream=None):
    cp, k, _a = _buf(c, np.float32)
    _check(lib().chemo_write_field(_h(sim), cp, k, _stream(stream)), "chemo_write_field")


def chemo_step(sim: Sim, stream=None):
    _check(lib().chemo_step(_h(sim), _stream(stream)), "chemo_step")


def chemo_step_n(sim: Sim, nsteps: int, stream=None):
    _check(lib().chemo_step_n(_h(sim), int(nsteps), _stream(stream)), "chemo_step_n")


def chemo_read_state(sim: Sim, pos_out=None, species_out=None, disp_out=None, stream=None):
    pp, k1, _a = _buf(pos_out, np.float32)
    sp, k2, _b = _buf(species_out, np.uint8)
    dp, k3, _c = _buf(disp_out, np.float32)
    _check(lib().chemo_read_state(_h(sim), pp, sp, dp, _kind(k1, k2, k3), _stream(stream)), "chemo_read_state")


def chemo_read_field(sim: Sim, c_out, stream=None):
    cp, k, _a = _buf(c_out, np.float32)
    _check(lib().chemo_read_field(_h(sim), cp, k, _stream(stream)), "chemo_read_field")


def chemo_record(sim: Sim, nsteps: int, every: int, stream=None, store_bytes: int = 0):
    """Recorded run for chemo_gradient, checkpoints every `every` steps; the
    latest segments whose states fit in store_bytes (< 0: all) are kept and
    not re-run by the gradient."""
    if store_bytes:
        _check(lib().chemo_record_stored(_h(sim), int(nsteps), int(every), int(store_bytes), _stream(stream)),
               "chemo_record_stored")
    else:
        _check(lib().chemo_record(_h(sim), int(nsteps), int(every), _stream(stream)), "chemo_record")


def chemo_gradient(sim: Sim, dL_dpos_final, dL_dparams, dL_dc_final=None, dL_dpos0=None, stream=None):
    a, k1, _a = _buf(dL_dpos_final, np.float32)
    b, k2, _b = _buf(dL_dc_final, np.float32)
    c, k3, _c = _buf(dL_dparams, np.float32)
    d, k4, _d = _buf(dL_dpos0, np.float32)
    _check(lib().chemo_gradient(_h(sim), a, b, c, d, _kind(k1, k2, k3, k4), _stream(stream)), "chemo_gradient")


def chemo_set_params(sim: Sim, params: dict):
    prm = make_params(params)
    _check(lib().chemo_set_params(_h(sim), ctypes.byref(prm)), "chemo_set_params")
    sim.params = dict(params)


def chemo_step_index(sim: Sim) -> int:
    return int(lib().chemo_step_index(_h(sim)))


def chemo_set_step_index(sim: Sim, step: int, stream=None):
    _check(lib().chemo_set_step_index(_h(sim), int(step), _stream(stream)), "chemo_set_step_index")


def chemo_check(sim: Sim, stream=None):
    _check(lib().chemo_check(_h(sim), _stream(stream)), "chemo_check")


def chemo_stall_scan(sim: Sim, spin_limit: int, stream=None):
    """Failure-detection test: one scan whose look-back waits on a tile that
    no block publishes and gives up after spin_limit polls (the next
    chemo_check raises ETIMEOUT); the simulation is left untouched."""
    _check(lib().chemo_stall_scan(_h(sim), int(spin_limit), _stream(stream)), "chemo_stall_scan")


def chemo_get_info(sim: Sim) -> dict:
    info = chemo_info()
    _check(lib().chemo_get_info(_h(sim), ctypes.byref(info)), "chemo_get_info")
    return {name: (list(getattr(info, name)) if hasattr(getattr(info, name), "__len__") else getattr(info, name))
            for name, _ in chemo_info._fields_}


PROF_SLOTS = 7
PROF_NAMES = ("k_step", "k_pde", "k_scan", "k_scatter", "step", "pairs_per_step", "tests_per_step")


def chemo_profile_steps(sim: Sim, nsteps: int, stream=None) -> dict:
    """Mean device ms per step of each kernel class and of a whole step, and
    the mean number of in-cutoff pair interactions per step."""
    out = (ctypes.c_float * PROF_SLOTS)()
    _check(lib().chemo_profile_steps(_h(sim), int(nsteps), out, _stream(stream)), "chemo_profile_steps")
    return {PROF_NAMES[i]: float(out[i]) for i in range(PROF_SLOTS)}


def chemo_init_positions(params: dict, n: int, n_alpha: int, sigma_frac: float = 0.1, pos_out=None,
                         species_out=None, stream=None):
    """The paper's initial state drawn on the device (alpha normal around the
    centre, beta uniform). Fills pos_out (n, dim) float32 and species_out (n,)
    uint8 (host or device); allocates host arrays when they are None."""
    dim = int(params["dim"])
    if pos_out is None:
        pos_out = np.zeros((int(n), dim), np.float32)
    if species_out is None:
        species_out = np.zeros(int(n), np.uint8)
    pp, k1, _a = _buf(pos_out, np.float32)
    sp, k2, _b = _buf(species_out, np.uint8)
    prm = make_params(params)
    _check(lib().chemo_init_positions(ctypes.byref(prm), int(n), int(n_alpha), float(sigma_frac), pp, sp,
                                      _kind(k1, k2), _stream(stream)), "chemo_init_positions")
    return pos_out, species_out


OBS_PER_LAYER = 8 * 5 + 1


def chemo_observables(sim: Sim, stream=None) -> list:
    """Observables of the current state reduced on the device, one dict per
    replicate: cells per species, mean displacement (n_species, 3) and mean
    squared displacement per species (0 unless track_displacement), and the
    chemical mass (trapezoid rule over the grid)."""
    layers = sim.replicates
    out = np.zeros(layers * OBS_PER_LAYER, np.float64)
    _check(lib().chemo_observables(_h(sim), out.ctypes.data, MEM_HOST, _stream(stream)), "chemo_observables")
    ns = int(sim.params["n_species"])
    res = []
    for layer in range(layers):
        v = out[layer * OBS_PER_LAYER:(layer + 1) * OBS_PER_LAYER]
        per = v[:40].reshape(8, 5)[:ns]
        res.append({"count": per[:, 0].copy(), "mean_disp": per[:, 1:4].copy(), "msd": per[:, 4].copy(),
                    "c_mass": float(v[40])})
    return res


def chemo_histogram(sim: Sim, shape, stream=None) -> np.ndarray:
    """Cells per part of the box cut into shape (per axis), per replicate and
    species: float32 array [replicate][species][z][y][x] (no z in 2D)."""
    dim = int(sim.dim)
    sh = [int(x) for x in shape][:dim] + [1] * (3 - dim)
    layers = sim.replicates
    ns = int(sim.params["n_species"])
    out = np.zeros([layers, ns] + list(reversed(sh[:dim])), np.float32)
    s3 = (ctypes.c_int32 * 3)(*sh)
    _check(lib().chemo_histogram(_h(sim), s3, out.ctypes.data, MEM_HOST, _stream(stream)), "chemo_histogram")
    return out


def chemo_destroy(sim: Sim):
    sim.close()


def chemo_status_string(status: int) -> str:
    return lib().chemo_status_string(int(status)).decode()


def chemo_last_error() -> str:
    return lib().chemo_last_error().decode()


def chemo_philox(seed: int, ctr, out, stream=None):
    cp, k1, _a = _buf(ctr, np.uint32)
    op, k2, _b = _buf(out, np.uint32)
    n = int(np.prod(ctr.shape)) // 4
    _check(lib().chemo_philox(int(seed) & 0xFFFFFFFFFFFFFFFF, cp, op, n, _kind(k1, k2), _stream(stream)),
           "chemo_philox")


def chemo_stage_bins(sim: Sim, cells_out, stream=None):
    cp, k, _a = _buf(cells_out, np.int32)
    _check(lib().chemo_stage_bins(_h(sim), cp, k, _stream(stream)), "chemo_stage_bins")


def chemo_stage_sort(sim: Sim, ids_out=None, bin_start_out=None, stream=None):
    ip, k1, _a = _buf(ids_out, np.uint32)
    bp, k2, _b = _buf(bin_start_out, np.uint32)
    _check(lib().chemo_stage_sort(_h(sim), ip, bp, _kind(k1, k2), _stream(stream)), "chemo_stage_sort")


def chemo_stage_forces(sim: Sim, F_out, count_out=None, idsum_out=None, stream=None):
    fp, k1, _a = _buf(F_out, np.float32)
    cp, k2, _b = _buf(count_out, np.int32)
    ip, k3, _c = _buf(idsum_out, np.uint64)
    _check(lib().chemo_stage_forces(_h(sim), fp, cp, ip, _kind(k1, k2, k3), _stream(stream)), "chemo_stage_forces")


def chemo_stage_drift(sim: Sim, drift_out, stream=None):
    dp, k, _a = _buf(drift_out, np.float32)
    _check(lib().chemo_stage_drift(_h(sim), dp, k, _stream(stream)), "chemo_stage_drift")


def chemo_stage_deposit(sim: Sim, S_out=None, R_out=None, stream=None):
    sp, k1, _a = _buf(S_out, np.float32)
    rp, k2, _b = _buf(R_out, np.float32)
    _check(lib().chemo_stage_deposit(_h(sim), sp, rp, _kind(k1, k2), _stream(stream)), "chemo_stage_deposit")


def chemo_forces_noalloc(params: dict, pos, species, F_out, stream=None):
    """Pair forces of a particle set (all CUDA tensors) without any device
    allocation (see include/chemo.h for the limits)."""
    pp, k1, _a = _buf(pos, np.float32)
    sp, k2, _b = _buf(species, np.uint8)
    fp, k3, _c = _buf(F_out, np.float32)
    if _kind(k1, k2, k3) != MEM_DEVICE:
        raise ValueError("chemo_forces_noalloc takes device buffers only")
    prm = make_params(params)
    n = int(pos.shape[0])
    _check(lib().chemo_forces_noalloc(ctypes.byref(prm), n, pp, sp, fp, _stream(stream)), "chemo_forces_noalloc")


def chemo_create_subdomain(params: dict, capacity: int, open_faces: int, stream=None) -> Sim:
    """An empty sub-domain (a z-slab with its halo) holding up to `capacity`
    cells; open_faces is a mask of OPEN_ZLO / OPEN_ZHI."""
    out = ctypes.c_void_p()
    prm = make_params(params)
    _check(lib().chemo_create_subdomain(ctypes.byref(prm), int(capacity), int(open_faces), _stream(stream),
                                        ctypes.byref(out)), "chemo_create_subdomain")
    sim = Sim(out, params, 0)
    sim.capacity = int(capacity)
    return sim


def _cells(cells):
    """(pointer, mem_kind, count, keepalive) of a cell-record buffer: a CUDA or
    CPU float32 tensor of shape (m, 8), or a numpy array of CELL_DTYPE."""
    try:
        import torch
        if isinstance(cells, torch.Tensor):
            if cells.dim() != 2 or cells.shape[1] != CELL_FLOATS or cells.dtype != torch.float32:
                raise TypeError("cell records must be a float32 tensor of shape (m, 8)")
            if not cells.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return (ctypes.c_void_p(cells.data_ptr()), MEM_DEVICE if cells.is_cuda else MEM_HOST,
                    int(cells.shape[0]), cells)
    except ImportError:
        pass
    a = np.asarray(cells)
    if a.dtype != CELL_DTYPE or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("numpy cell records must be a C-contiguous CELL_DTYPE array")
    return a.ctypes.data_as(ctypes.c_void_p), MEM_HOST, int(a.shape[0]), a


def chemo_slab_ingest(sim: Sim, cells, n=None, stream=None):
    """Replaces the sub-domain's cells by the first n records of `cells`."""
    ptr, kind, m, _k = _cells(cells)
    n = m if n is None else int(n)
    if n > m:
        raise ValueError("n = %d exceeds the %d records given" % (n, m))
    _check(lib().chemo_slab_ingest(_h(sim), n, ptr, kind, _stream(stream)), "chemo_slab_ingest")
    sim.n = n


def chemo_slab_select(sim: Sim, targets, stream=None):
    """targets: sequence of (z0, z1, own0, own1, out, count) with out a CUDA
    float32 tensor (capacity, 8) and count a CUDA int64 tensor of 2 counters
    that the call adds to."""
    import torch
    arr = (chemo_slab_target * max(len(targets), 1))()
    keep = []
    for k, (z0, z1, own0, own1, out, count) in enumerate(targets):
        if not (out.is_cuda and count.is_cuda and count.dtype == torch.int64 and count.numel() >= 2):
            raise TypeError("out and count must be CUDA tensors; count int64 with 2 entries")
        if out.dim() != 2 or out.shape[1] != CELL_FLOATS or out.dtype != torch.float32 or not out.is_contiguous():
            raise TypeError("out must be a contiguous float32 tensor of shape (capacity, 8)")
        arr[k] = chemo_slab_target(float(z0), float(z1), float(own0), float(own1), out.data_ptr(),
                                   int(out.shape[0]), count.data_ptr())
        keep.append((out, count))
    _check(lib().chemo_slab_select(_h(sim), len(targets), arr, _stream(stream)), "chemo_slab_select")


def chemo_slab_planes(sim: Sim, grid: int, op: int, plane0: int, nplanes: int, buf, stream=None):
    """Reads (op 0), writes (1) or adds (2) z-planes plane0.. of grid 0 (c),
    1 (source) or 2 (consumption) against the CUDA float32 tensor buf."""
    bp, kind, _k = _buf(buf, np.float32)
    if kind != MEM_DEVICE:
        raise ValueError("chemo_slab_planes takes a device buffer")
    need = max(int(nplanes), 0) * int(sim.params["grid"][0]) * int(sim.params["grid"][1])
    if buf.numel() < need:
        raise ValueError("buf holds %d floats, %d planes need %d" % (buf.numel(), int(nplanes), need))
    _check(lib().chemo_slab_planes(_h(sim), int(grid), int(op), int(plane0), int(nplanes), bp, _stream(stream)),
           "chemo_slab_planes")


def chemo_step_particles(sim: Sim, stream=None):
    _check(lib().chemo_step_particles(_h(sim), _stream(stream)), "chemo_step_particles")


def chemo_step_field(sim: Sim, stream=None):
    _check(lib().chemo_step_field(_h(sim), _stream(stream)), "chemo_step_field")


# ---------------------------------------------------------------------------
# Host-array conveniences (numpy in, numpy out) over the calls above.
# ---------------------------------------------------------------------------
def grid_shape(params: dict) -> tuple:
    return tuple(int(params["grid"][a]) for a in reversed(range(int(params["dim"]))))


def read_state_host(sim: Sim):
    pos = np.zeros((sim.n, sim.dim), np.float32)
    sp = np.zeros(sim.n, np.uint8)
    disp = np.zeros((sim.n, sim.dim), np.float32) if sim.params.get("track_displacement") else None
    chemo_read_state(sim, pos, sp, disp)
    return pos, sp, disp


def read_field_host(sim: Sim):
    shape = grid_shape(sim.params)
    if sim.replicates > 1:
        shape = (sim.replicates,) + shape
    c = np.zeros(shape, np.float32)
    chemo_read_field(sim, c)
    return c


_allocator = None  # the callbacks in force
_retired = []      # earlier callbacks: simulations created under them release through them


def chemo_set_allocator(alloc=None, release=None):
    """Device buffers of simulations created from now on (and the temporaries
    of chemo_philox / chemo_init_positions) come from alloc(nbytes) -> int
    device pointer (0 or an exception: failure, the call raises ENOMEM) and go
    back through release(ptr, nbytes) once the device is done with them. A
    simulation keeps the allocator it was created with. None, None restores
    cudaMalloc / cudaFree."""
    global _allocator
    if (alloc is None) != (release is None):
        raise ValueError("alloc and release are both given or both None")
    if alloc is None:
        _check(lib().chemo_set_allocator(None, None, None), "chemo_set_allocator")
        if _allocator is not None:
            _retired.append(_allocator)
        _allocator = None
        return

    def _alloc(ctx, nbytes, out):
        try:
            ptr = int(alloc(int(nbytes)) or 0)
        except Exception:
            return 1
        if ptr == 0:
            return 1
        out[0] = ptr
        return 0

    def _release(ctx, ptr, nbytes):
        if ptr:
            try:
                release(int(ptr), int(nbytes))
            except Exception:
                pass

    cb = (ALLOC_FN(_alloc), RELEASE_FN(_release))
    _check(lib().chemo_set_allocator(ctypes.cast(cb[0], ctypes.c_void_p), ctypes.cast(cb[1], ctypes.c_void_p), None),
           "chemo_set_allocator")
    if _allocator is not None:
        _retired.append(_allocator)
    _allocator = cb


def use_torch_allocator():
    """Backs the library's device buffers by PyTorch's caching allocator (on
    the current device and stream at each allocation)."""
    import torch

    chemo_set_allocator(lambda nbytes: torch.cuda.caching_allocator_alloc(nbytes),
                        lambda ptr, nbytes: torch.cuda.caching_allocator_delete(ptr))
