"""Seeded synthetic workloads: model parameters and initial states.

This module holds no arithmetic of the method. It only draws initial particle
states and fields with numpy's seeded generator and spells out the parameter
sets of the workloads, so that the GPU library and the CPU oracle can be fed
identical inputs. It imports nothing from either side.

Parameter dicts use the model's parameter names (the C-ABI field names):

    dim, boundary (0 walls, 1 periodic), lo, hi, n_species, diameter, D,
    chemotactic, secrete, consume, react_k0, react_kc, react_to, reactions,
    chi, inter, cutoff_factor, cutoff_mode, chem_mode (0 grid, 1 fixed
    gradient), fixed_grad, grid, Dc, gamma, pde_bc (0 Neumann, 1 Dirichlet,
    2 periodic), pde_substeps (0 auto), dt, seed, track_displacement,
    bin_side (0 auto), search_mode (0 auto, 1 3^d warp, 2 2^d, 3 3^d per lane,
    4 half of the 3^d window).

Workloads (the paper's Fig. 1-3 model with the sizes of the GPU benchmarks):

* ``periodic_fixed_gradient_2d``: unit periodic square, 1,000 cells of one
  chemotactic species (diameter 0.01, D = 1), fixed gradient c = x with
  chi = 1 (the MSD set-up of Sect. 4), dt = 1e-5, 100 steps.
* ``walls_grid_2d``: unit square with walls, 100,000 cells, 50/50 species
  (diameters 0.005 / 0.01, D = 1 / 0.5), 512^2 grid, D_c = 1, gamma = 0.1,
  secretion 0.1 by species 0, c0 = 0, dt = 1e-5, 1,000 steps.
* ``clumps_grid_3d``: unit cube with walls, 1,000,000 cells (diameters 0.002 /
  0.004, D = 1 / 0.5) from 8 Gaussian clumps (sigma 0.05) at {0.25, 0.75}^3,
  256^3 grid, 7-point stencil, same chemistry, dt = 1e-6, 200 steps.
* ``ensemble_2d``: replicates of the walls_grid_2d physics with N drawn
  log-uniform in [1e3, 6.4e4], 128^2 grid each, distinct seeds.
* ``adjoint_2d``: 50,000 cells of the walls_grid_2d physics, force shifted to
  zero at the cutoff.
"""
from __future__ import annotations

import copy

import numpy as np

_BASE2 = dict(
    dim=2, boundary=0, lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0], n_species=2,
    diameter=[0.005, 0.01], D=[1.0, 0.5], chemotactic=[0.0, 1.0], secrete=[0.1, 0.0],
    consume=[0.0, 0.0], react_k0=[0.0, 0.0], react_kc=[0.0, 0.0], react_to=[1, 0], reactions=0,
    chi=1.0, inter=1.0, cutoff_factor=1.0, cutoff_mode=0, chem_mode=0, fixed_grad=[0.0, 0.0, 0.0],
    grid=[512, 512, 1], Dc=1.0, gamma=0.1, pde_bc=0, pde_substeps=0, dt=1e-5, seed=1,
    track_displacement=0, bin_side=0.0, search_mode=0,
)

WORKLOADS = {
    "periodic_fixed_gradient_2d": dict(
        params=dict(_BASE2, boundary=1, n_species=1, diameter=[0.01], D=[1.0], chemotactic=[1.0],
                    secrete=[0.0], consume=[0.0], react_k0=[0.0], react_kc=[0.0], react_to=[0],
                    chem_mode=1, fixed_grad=[1.0, 0.0, 0.0], grid=[3, 3, 1], pde_bc=2, Dc=0.0,
                    gamma=0.0, track_displacement=1),
        n=1000, init="uniform", steps=100),
    "walls_grid_2d": dict(params=dict(_BASE2), n=100_000, init="uniform", steps=1000),
    "clumps_grid_3d": dict(
        params=dict(_BASE2, dim=3, diameter=[0.002, 0.004], grid=[256, 256, 256], dt=1e-6),
        n=1_000_000, init="clumps", steps=200),
    "ensemble_2d": dict(params=dict(_BASE2, grid=[128, 128, 1]), n=None, init="uniform", steps=500,
                        replicates=256, n_min=1000, n_max=64000),
    "adjoint_2d": dict(params=dict(_BASE2, cutoff_mode=1), n=50_000, init="uniform", steps=200,
                       ckpt_every=20),
}


def params(name: str, **overrides) -> dict:
    """Parameter dict of a workload with keyword overrides."""
    p = copy.deepcopy(WORKLOADS[name]["params"])
    for k, v in overrides.items():
        p[k] = copy.deepcopy(v)
    return p


def uniform_positions(n: int, dim: int, lo, hi, seed: int) -> np.ndarray:
    """n points uniform in the box, float32 (n, dim)."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo[:dim], dtype=np.float64)
    hi = np.asarray(hi[:dim], dtype=np.float64)
    x = lo + (hi - lo) * rng.random((n, dim))
    x = x.astype(np.float32)
    # keep strictly inside [lo, hi) after rounding to float32
    top = np.nextafter(hi.astype(np.float32), np.float32(-np.inf))
    return np.minimum(x, top).astype(np.float32)


def clump_positions(n: int, dim: int, lo, hi, seed: int, sigma: float = 0.05,
                    centres=(0.25, 0.75)) -> np.ndarray:
    """n points from 2^dim Gaussian clumps (std sigma) centred at the corners
    of {0.25, 0.75}^dim (scaled to the box); point i belongs to clump i mod
    2^dim. Points that fall outside the box are drawn again."""
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo[:dim], dtype=np.float64)
    hi = np.asarray(hi[:dim], dtype=np.float64)
    ncl = 1 << dim
    cidx = np.arange(ncl)
    cen = np.array([[centres[(c >> a) & 1] for a in range(dim)] for c in cidx], dtype=np.float64)
    cen = lo + (hi - lo) * cen
    which = np.arange(n) % ncl
    x = cen[which] + sigma * (hi - lo) * rng.standard_normal((n, dim))
    top = np.nextafter(hi.astype(np.float32), np.float32(-np.inf)).astype(np.float64)
    for _ in range(1000):
        bad = np.any((x < lo) | (x > top), axis=1)
        if not bad.any():
            break
        x[bad] = cen[which[bad]] + sigma * (hi - lo) * rng.standard_normal((int(bad.sum()), dim))
    x = np.clip(x, lo, top)
    return x.astype(np.float32)


def half_species(n: int, n_species: int) -> np.ndarray:
    """Species 0 for the first half of the ids, 1 for the rest (the paper sets
    type = (i < N_alpha), Sect. 3.1); a single species gives all zeros."""
    sp = np.zeros(n, dtype=np.uint8)
    if n_species > 1:
        sp[n // 2:] = 1
    return sp


def initial_state(name: str, n: int | None = None, seed: int | None = None, **overrides):
    """(params, pos float32 (n, dim), species uint8 (n,)) of a workload; n and
    seed default to the workload's."""
    w = WORKLOADS[name]
    p = params(name, **overrides)
    n = w["n"] if n is None else n
    seed = p["seed"] if seed is None else seed
    if w["init"] == "clumps":
        pos = clump_positions(n, p["dim"], p["lo"], p["hi"], seed)
    else:
        pos = uniform_positions(n, p["dim"], p["lo"], p["hi"], seed)
    sp = half_species(n, p["n_species"])
    return p, pos, sp


def random_field(params_: dict, seed: int, scale: float = 1.0) -> np.ndarray:
    """A smooth-ish positive random field on the grid (float32, C-order),
    used as a non-zero c^n for interpolation and PDE checks."""
    rng = np.random.default_rng(seed)
    dim = params_["dim"]
    shape = tuple(int(params_["grid"][a]) for a in reversed(range(dim)))
    axes = [np.linspace(0.0, 1.0, s) for s in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    f = np.zeros(shape)
    for _ in range(4):
        k = rng.integers(1, 4, size=dim)
        ph = rng.random(dim) * 2 * np.pi
        term = np.ones(shape)
        for a in range(dim):
            term = term * np.cos(np.pi * k[a] * mesh[a] + ph[a])
        f += rng.random() * term
    f = f + 0.1 * rng.standard_normal(shape)
    f = scale * (f - f.min() + 0.5)
    return f.astype(np.float32)


def ensemble_sizes(replicates: int, n_min: int, n_max: int, seed: int) -> np.ndarray:
    """Replicate sizes drawn log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=replicates))).astype(np.int64)


def ensemble_state(name: str = "ensemble_2d", replicates: int | None = None, seed: int | None = None,
                   sizes=None, **overrides):
    """(params, sizes int64 (R,), pos float32 (sum n, 2), species uint8
    (sum n,)) of an ensemble workload: replicate r has sizes[r] cells drawn
    uniform in the box with seed + 1000 + r, species split in halves. The
    replicates' arrays are concatenated in replicate order (the layout of
    chemo_create_batch); replicate r runs with Philox key params['seed'] + r."""
    w = WORKLOADS[name]
    p = params(name, **overrides)
    seed = p["seed"] if seed is None else seed
    if sizes is None:
        R = w["replicates"] if replicates is None else replicates
        sizes = ensemble_sizes(R, w["n_min"], w["n_max"], seed)
    sizes = np.asarray(sizes, dtype=np.int64).reshape(-1)
    pos = [uniform_positions(int(m), p["dim"], p["lo"], p["hi"], seed + 1000 + r) for r, m in enumerate(sizes)]
    sp = [half_species(int(m), p["n_species"]) for m in sizes]
    pos = np.concatenate(pos, axis=0) if len(pos) else np.zeros((0, p["dim"]), np.float32)
    sp = np.concatenate(sp) if len(sp) else np.zeros(0, np.uint8)
    return p, sizes, np.ascontiguousarray(pos, dtype=np.float32), np.ascontiguousarray(sp)


def replicate_params(params_: dict, r: int) -> dict:
    """Parameters of replicate r of an ensemble run on its own (seed + r)."""
    q = copy.deepcopy(params_)
    q["seed"] = int(params_.get("seed", 0)) + int(r)
    return q
