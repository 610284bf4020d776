"""ctypes binding of the FP64 CPU oracle (``chemo_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` import this module. The GPU
package never imports it.

Parameters are plain dicts whose keys are the model's parameter names (the
same keys the GPU binding reads); the oracle copies them into its own struct.
All arrays are numpy; positions are ``(n, dim)`` float64 and grids are C-order
``[z][y][x]`` float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "chemo_oracle.c")
_LIB = os.path.join(_HERE, "libchemo_oracle.so")
_lock = threading.Lock()
_lib = None

MAXS = 8
TAG_MOVE = 0
TAG_REACT = 2
TAG_INIT = 3


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (OpenMP when available; no FMA contraction,
    so the single-precision bin rule rounds like the GPU's)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp", "-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp, _SRC, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int32),
        ("boundary", ctypes.c_int32),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("n_species", ctypes.c_int32),
        ("diameter", ctypes.c_double * MAXS),
        ("D", ctypes.c_double * MAXS),
        ("chemotactic", ctypes.c_double * MAXS),
        ("secrete", ctypes.c_double * MAXS),
        ("consume", ctypes.c_double * MAXS),
        ("react_k0", ctypes.c_double * MAXS),
        ("react_kc", ctypes.c_double * MAXS),
        ("react_to", ctypes.c_int32 * MAXS),
        ("reactions", ctypes.c_int32),
        ("chi", ctypes.c_double),
        ("inter", ctypes.c_double),
        ("cutoff_factor", ctypes.c_double),
        ("cutoff_mode", ctypes.c_int32),
        ("chem_mode", ctypes.c_int32),
        ("fixed_grad", ctypes.c_double * 3),
        ("grid", ctypes.c_int32 * 3),
        ("Dc", ctypes.c_double),
        ("gamma", ctypes.c_double),
        ("pde_bc", ctypes.c_int32),
        ("pde_substeps", ctypes.c_int32),
        ("dt", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("move_scheme", ctypes.c_int32),
        ("hard_sphere", ctypes.c_int32),
        ("deposit_kernel", ctypes.c_int32),
        ("kde_range", ctypes.c_double),
    ]


def _f32(v) -> float:
    """Model constants are given to the GPU in single precision; the oracle
    takes the same single-precision values, widened exactly to double."""
    return float(np.float32(v))


def make_params(d: dict) -> OrcParams:
    p = OrcParams()
    p.dim = int(d["dim"])
    p.boundary = int(d.get("boundary", 0))
    for a in range(3):
        p.lo[a] = float(d.get("lo", [0.0, 0.0, 0.0])[a])
        p.hi[a] = float(d.get("hi", [1.0, 1.0, 1.0])[a])
    ns = int(d["n_species"])
    p.n_species = ns
    for name in ("diameter", "D", "chemotactic", "secrete", "consume", "react_k0", "react_kc"):
        vals = list(d.get(name, [0.0] * ns))
        arr = getattr(p, name)
        for s in range(MAXS):
            arr[s] = _f32(vals[s]) if s < len(vals) else 0.0
    rt = list(d.get("react_to", list(range(ns))))
    for s in range(MAXS):
        p.react_to[s] = int(rt[s]) if s < len(rt) else s
    p.reactions = int(d.get("reactions", 0))
    p.chi = _f32(d.get("chi", 0.0))
    p.inter = _f32(d.get("inter", 1.0))
    p.cutoff_factor = _f32(d.get("cutoff_factor", 1.0))
    p.cutoff_mode = int(d.get("cutoff_mode", 0))
    p.chem_mode = int(d.get("chem_mode", 0))
    fg = list(d.get("fixed_grad", [0.0, 0.0, 0.0]))
    for a in range(3):
        p.fixed_grad[a] = _f32(fg[a]) if a < len(fg) else 0.0
    g = list(d.get("grid", [3, 3, 3]))
    for a in range(3):
        p.grid[a] = int(g[a]) if a < len(g) else 1
    p.Dc = _f32(d.get("Dc", 0.0))
    p.gamma = _f32(d.get("gamma", 0.0))
    p.pde_bc = int(d.get("pde_bc", 0))
    p.pde_substeps = int(d.get("pde_substeps", 0))
    p.dt = float(d["dt"])
    p.seed = int(d.get("seed", 0)) & 0xFFFFFFFFFFFFFFFF
    p.move_scheme = int(d.get("move_scheme", 0))
    p.hard_sphere = int(d.get("hard_sphere", 0))
    p.deposit_kernel = int(d.get("deposit_kernel", 0))
    p.kde_range = _f32(d.get("kde_range", 0.0) or 3.0)
    return p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _declare(L):
    P = ctypes.POINTER(OrcParams)
    vp = ctypes.c_void_p
    i64 = ctypes.c_int64
    L.orc_set_threads.argtypes = [ctypes.c_int]
    L.orc_get_threads.restype = ctypes.c_int
    L.orc_philox4x32_10.argtypes = [vp, vp, vp]
    L.orc_philox_batch.argtypes = [i64, vp, ctypes.c_uint64, vp]
    L.orc_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, vp]
    L.orc_normals_batch.argtypes = [ctypes.c_uint64, i64, vp, ctypes.c_uint64, ctypes.c_uint32, vp]
    L.orc_bins_f32.argtypes = [P, ctypes.c_double, i64, vp, vp, vp]
    L.orc_pair_forces.argtypes = [P, i64, vp, vp, ctypes.c_int, vp, vp, vp, vp, vp, vp]
    L.orc_grid_h.argtypes = [P, ctypes.c_int]
    L.orc_grid_h.restype = ctypes.c_double
    L.orc_grid_size.argtypes = [P]
    L.orc_grid_size.restype = i64
    L.orc_substeps.argtypes = [P]
    L.orc_substeps.restype = ctypes.c_int
    L.orc_drift.argtypes = [P, i64, vp, vp, vp, vp]
    L.orc_conc.argtypes = [P, i64, vp, vp, vp]
    L.orc_deposit.argtypes = [P, i64, vp, vp, vp, vp]
    L.orc_kde_deposit.argtypes = [P, i64, vp, vp, vp, vp]
    L.orc_hard_sphere.argtypes = [P, i64, vp, vp, vp]
    L.orc_pde_substep.argtypes = [P, vp, vp, vp, ctypes.c_int, vp]
    L.orc_move.argtypes = [P, i64, vp, vp, vp, vp, i64, vp, vp, vp]
    L.orc_step.argtypes = [P, i64, vp, vp, vp, vp, i64, vp, vp, vp]
    L.orc_run.argtypes = [P, i64, vp, vp, vp, vp, i64, i64, vp]
    L.orc_run_tangent.argtypes = [P, i64, vp, vp, vp, vp, i64, i64, ctypes.c_int, vp, vp]
    L.orc_run_tangent.restype = ctypes.c_int


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _pos(pos, dim):
    return np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, dim))


def _u8(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint8))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def philox(ctr, seed: int) -> np.ndarray:
    """Raw Philox4x32-10 words for counters ``ctr`` ((n,4) uint32) under the
    key (seed lo, seed hi)."""
    ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    out = np.zeros_like(ctr)
    lib().orc_philox_batch(ctr.shape[0], _ptr(ctr), int(seed) & (2**64 - 1), _ptr(out))
    return out


def init_positions(params: dict, n: int, n_alpha: int, sigma_frac: float = 0.1):
    """The paper's initial state (Sect. 3: alpha cells start normal around the
    centre of the domain with sigma = 0.1 of its width, beta cells uniform),
    in FP64 from the same Philox words as the device: cell i takes the words
    of counter (i, 0, TAG_INIT, 0) under the key seed, u = (w + 1/2) 2^-32.
    Alpha (i < n_alpha, species 0): Box-Muller on (u0, u1) and (u2, u3) gives
    g, x = centre + sigma_frac L g, put inside by reflection at the walls or
    by wrapping on a periodic box. Beta (species 1): x = lo + u_a L per axis.
    Returns (pos (n, dim) float64, species (n,) uint8)."""
    dim = int(params["dim"])
    lo = np.asarray(params["lo"], np.float64)[:dim]
    hi = np.asarray(params["hi"], np.float64)[:dim]
    L = hi - lo
    periodic = int(params.get("boundary", 0)) == 1
    ctr = np.zeros((int(n), 4), np.uint32)
    ctr[:, 0] = np.arange(int(n), dtype=np.uint32)
    ctr[:, 2] = TAG_INIT
    w = philox(ctr, int(params["seed"])).astype(np.float64)
    u = (w + 0.5) / 2.0 ** 32
    r01 = np.sqrt(-2.0 * np.log(u[:, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, 2]))
    g = np.stack([r01 * np.cos(2.0 * np.pi * u[:, 1]), r01 * np.sin(2.0 * np.pi * u[:, 1]),
                  r23 * np.cos(2.0 * np.pi * u[:, 3])], axis=1)[:, :dim]
    alpha = np.arange(int(n)) < int(n_alpha)
    pos = np.where(alpha[:, None], 0.5 * (lo + hi) + sigma_frac * L * g, lo + u[:, :dim] * L)
    for a in range(dim):
        x = pos[:, a]
        if periodic:
            x = lo[a] + np.mod(x - lo[a], L[a])
        else:
            for _ in range(16):  # reflect until inside (a triangle wave)
                x = np.where(x < lo[a], 2.0 * lo[a] - x, np.where(x > hi[a], 2.0 * hi[a] - x, x))
        pos[:, a] = x
    return pos, np.where(alpha, 0, 1).astype(np.uint8)


def normals(seed: int, ids, step: int, tag: int = TAG_MOVE) -> np.ndarray:
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.uint32))
    out = np.zeros((ids.size, 4), dtype=np.float64)
    lib().orc_normals_batch(int(seed) & (2**64 - 1), ids.size, _ptr(ids), int(step), int(tag), _ptr(out))
    return out


def bins_f32(params: dict, bin_side: float, pos_f32) -> tuple[np.ndarray, tuple]:
    p = make_params(params)
    pos = np.ascontiguousarray(np.asarray(pos_f32, dtype=np.float32).reshape(-1, p.dim))
    cells = np.zeros(pos.shape, dtype=np.int32)
    nb = np.zeros(3, dtype=np.int32)
    # the bin side is a single-precision parameter of the GPU library
    lib().orc_bins_f32(ctypes.byref(p), _f32(bin_side), pos.shape[0], _ptr(pos), _ptr(cells), _ptr(nb))
    return cells, tuple(int(v) for v in nb)


def pair_forces(params: dict, pos, species, method: int = 1, extras: bool = False):
    """Pair force per particle; with extras also the per-particle sum of
    |f_ij|, the borderline magnitude, the neighbour count, and the sum / xor
    of neighbour indices."""
    p = make_params(params)
    pos = _pos(pos, p.dim)
    sp = _u8(species)
    n = pos.shape[0]
    F = np.zeros_like(pos)
    fabs = np.zeros(n)
    border = np.zeros(n)
    cnt = np.zeros(n, dtype=np.int64)
    idsum = np.zeros(n, dtype=np.uint64)
    idxor = np.zeros(n, dtype=np.uint64)
    lib().orc_pair_forces(ctypes.byref(p), n, _ptr(pos), _ptr(sp), int(method), _ptr(F), _ptr(fabs),
                          _ptr(border), _ptr(cnt), _ptr(idsum), _ptr(idxor))
    if extras:
        return F, dict(fabs=fabs, border=border, count=cnt, idsum=idsum, idxor=idxor)
    return F


def grid_shape(params: dict) -> tuple:
    """Numpy shape of the grid, C-order (z, y, x) / (y, x)."""
    g = list(params["grid"])
    return tuple(int(g[a]) for a in reversed(range(int(params["dim"]))))


def grid_h(params: dict, axis: int) -> float:
    p = make_params(params)
    return float(lib().orc_grid_h(ctypes.byref(p), int(axis)))


def substeps(params: dict) -> int:
    p = make_params(params)
    return int(lib().orc_substeps(ctypes.byref(p)))


def _grid(c, params):
    return np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(grid_shape(params)))


def drift(params: dict, pos, species, c=None) -> np.ndarray:
    p = make_params(params)
    pos = _pos(pos, p.dim)
    sp = _u8(species)
    cg = _grid(c, params) if c is not None else np.zeros(1)
    out = np.zeros_like(pos)
    lib().orc_drift(ctypes.byref(p), pos.shape[0], _ptr(pos), _ptr(sp), _ptr(cg), _ptr(out))
    return out


def conc(params: dict, pos, c=None) -> np.ndarray:
    p = make_params(params)
    pos = _pos(pos, p.dim)
    cg = _grid(c, params) if c is not None else np.zeros(1)
    out = np.zeros(pos.shape[0])
    lib().orc_conc(ctypes.byref(p), pos.shape[0], _ptr(pos), _ptr(cg), _ptr(out))
    return out


def deposit(params: dict, pos, species) -> tuple[np.ndarray, np.ndarray]:
    p = make_params(params)
    pos = _pos(pos, p.dim)
    sp = _u8(species)
    S = np.zeros(grid_shape(params))
    R = np.zeros(grid_shape(params))
    lib().orc_deposit(ctypes.byref(p), pos.shape[0], _ptr(pos), _ptr(sp), _ptr(S), _ptr(R))
    return S, R


def kde_deposit(params: dict, pos, species) -> tuple[np.ndarray, np.ndarray]:
    """Gaussian kernel density estimate at the nodes (source S, consumption R)."""
    p = make_params(params)
    pos = _pos(pos, p.dim)
    sp = _u8(species)
    S = np.zeros(grid_shape(params))
    R = np.zeros(grid_shape(params))
    lib().orc_kde_deposit(ctypes.byref(p), pos.shape[0], _ptr(pos), _ptr(sp), _ptr(S), _ptr(R))
    return S, R


def hard_sphere(params: dict, pos, species, disp=None):
    """Hard-sphere overlap correction of positions (returns new positions
    and, when given, the updated displacement)."""
    p = make_params(params)
    x = _pos(pos, p.dim).copy()
    sp = _u8(species)
    dd = None if disp is None else np.ascontiguousarray(np.asarray(disp, dtype=np.float64)).copy()
    lib().orc_hard_sphere(ctypes.byref(p), x.shape[0], _ptr(x), _ptr(sp), None if dd is None else _ptr(dd))
    return (x, dd) if disp is not None else x


def pde_substep(params: dict, c, S=None, R=None, s: int = 1) -> np.ndarray:
    p = make_params(params)
    cg = _grid(c, params)
    Sg = _grid(S, params) if S is not None else None
    Rg = _grid(R, params) if R is not None else None
    out = np.zeros_like(cg)
    lib().orc_pde_substep(ctypes.byref(p), _ptr(cg), _ptr(Sg), _ptr(Rg), int(s), _ptr(out))
    return out


def step(params: dict, pos, species, c=None, step_index: int = 0, ids=None, disp=None,
         want_terms: bool = False):
    """One full time step. Returns (pos', species', c', disp') and, with
    want_terms, the pair force and drift used."""
    p = make_params(params)
    pos = _pos(pos, p.dim).copy()
    sp = _u8(species).copy()
    n = pos.shape[0]
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
    if p.chem_mode == 0:
        cg = _grid(c if c is not None else np.zeros(grid_shape(params)), params).copy()
    else:
        cg = np.zeros(1)
    dsp = None if disp is None else _pos(disp, p.dim).copy()
    F = np.zeros_like(pos) if want_terms else None
    dr = np.zeros_like(pos) if want_terms else None
    lib().orc_step(ctypes.byref(p), n, _ptr(pos), _ptr(sp), _ptr(ids), _ptr(cg), int(step_index),
                   _ptr(dsp), _ptr(F), _ptr(dr))
    out = (pos, sp, cg if p.chem_mode == 0 else None, dsp)
    if want_terms:
        return out + (F, dr)
    return out


def run(params: dict, pos, species, c=None, step0: int = 0, nsteps: int = 1, ids=None, disp=None):
    """nsteps consecutive steps from absolute step index step0."""
    p = make_params(params)
    pos = _pos(pos, p.dim).copy()
    sp = _u8(species).copy()
    n = pos.shape[0]
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
    if p.chem_mode == 0:
        cg = _grid(c if c is not None else np.zeros(grid_shape(params)), params).copy()
    else:
        cg = np.zeros(1)
    dsp = None if disp is None else _pos(disp, p.dim).copy()
    lib().orc_run(ctypes.byref(p), n, _ptr(pos), _ptr(sp), _ptr(ids), _ptr(cg), int(step0), int(nsteps),
                  _ptr(dsp))
    return pos, sp, (cg if p.chem_mode == 0 else None), dsp


def run_tangent(params: dict, pos, species, c=None, step0: int = 0, nsteps: int = 1, ids=None,
                dpos=None, dc=None, extra: int = 0):
    """nsteps steps with their forward-mode derivative with respect to
    theta = (chi, inter, D_0 .. D_{ns-1}), the noise frozen (the tangent of
    the step written out operation by operation; see orc_step_tangent).
    Returns (pos, species, c, dpos, dc): dpos[i, a, k] = dX_ia / dtheta_k
    and dc[..., k] = dc / dtheta_k (grid shape + (P,); None without a grid).
    dpos / dc carry in a previous tangent (zero: fixed initial data). The
    positions, species and field are those of run() bit for bit. `extra`
    columns after the parameters carry no parameter: seeded through dpos
    (a direction in the initial positions) they give directional
    derivatives."""
    p = make_params(params)
    pos = _pos(pos, p.dim).copy()
    sp = _u8(species).copy()
    n = pos.shape[0]
    P = 2 + int(p.n_species) + int(extra)
    ids = np.arange(n, dtype=np.uint32) if ids is None else np.ascontiguousarray(ids, dtype=np.uint32)
    if p.chem_mode == 0:
        cg = _grid(c if c is not None else np.zeros(grid_shape(params)), params).copy()
        G = int(cg.size)
        dcg = np.zeros((G, P)) if dc is None else np.ascontiguousarray(np.asarray(dc, np.float64).reshape(G, P)).copy()
    else:
        cg = np.zeros(1)
        dcg = np.zeros((1, P))
    dp = np.zeros((n, p.dim, P)) if dpos is None else np.ascontiguousarray(np.asarray(dpos, np.float64)).copy()
    r = lib().orc_run_tangent(ctypes.byref(p), n, _ptr(pos), _ptr(sp), _ptr(ids), _ptr(cg), int(step0),
                              int(nsteps), P, _ptr(dp), _ptr(dcg))
    if r:
        raise ValueError("run_tangent: %s" % ("Euler-Maruyama with cloud-in-cell deposit only, no reactions or "
                                             "hard spheres" if r == -1 else "wrong parameter count"))
    if p.chem_mode != 0:
        return pos, sp, None, dp, None
    return pos, sp, cg, dp, dcg.reshape(tuple(grid_shape(params)) + (P,))

