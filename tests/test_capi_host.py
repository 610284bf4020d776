"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/chemo.h declares, its struct layouts match the ctypes
binding, and parameter validation rejects bad input before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1805_11007_gb300 import build as gb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "chemo.h")


@pytest.fixture(scope="module")
def chemo():
    gb.build()
    from paper_1805_11007_gb300 import chemo as c
    return c


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chemo_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_function_is_exported(chemo):
    names = _declared()
    assert len(names) >= 20
    out = subprocess.run(["nm", "-D", "--defined-only", gb.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (chemo_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    L = chemo.lib()
    for n in names:
        assert hasattr(L, n)


def test_binding_declares_every_function_of_the_header(chemo):
    """The Python binding sets argument and result types for exactly the
    functions the header declares (no call goes through ctypes' defaults)."""
    import inspect
    bound = set(re.findall(r'"(chemo_[a-z_0-9]+)"', inspect.getsource(chemo._declare)))
    assert bound == set(_declared())


def test_struct_layouts_match_ctypes(chemo, tmp_path):
    prog = tmp_path / "layout.c"
    fields_p = [f for f, _ in chemo.chemo_params._fields_]
    fields_i = [f for f, _ in chemo.chemo_info._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chemo.h"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(chemo_params), sizeof(chemo_info));']
    for f in fields_p:
        lines.append('printf("p %s %%zu\\n", offsetof(chemo_params, %s));' % (f, f))
    for f in fields_i:
        lines.append('printf("i %s %%zu\\n", offsetof(chemo_info, %s));' % (f, f))
    lines.append("return 0;}")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    sp, si = map(int, out[0].split())
    assert sp == ctypes.sizeof(chemo.chemo_params)
    assert si == ctypes.sizeof(chemo.chemo_info)
    for line in out[1:]:
        if not line:
            continue
        kind, name, off = line.split()
        cls = chemo.chemo_params if kind == "p" else chemo.chemo_info
        assert getattr(cls, name).offset == int(off), name


def test_allocator_setting_checks_its_arguments(chemo):
    """chemo_set_allocator takes both callbacks or neither, and touches no
    GPU (the setting is read at the next allocation)."""
    L = chemo.lib()
    fa = chemo.ALLOC_FN(lambda ctx, nbytes, out: 1)
    fr = chemo.RELEASE_FN(lambda ctx, ptr, nbytes: None)
    only_alloc, only_release = ctypes.cast(fa, ctypes.c_void_p), ctypes.cast(fr, ctypes.c_void_p)
    assert L.chemo_set_allocator(only_alloc, None, None) == chemo.EINVAL
    assert "both" in L.chemo_last_error().decode()
    assert L.chemo_set_allocator(None, only_release, None) == chemo.EINVAL
    with pytest.raises(ValueError):
        chemo.chemo_set_allocator(lambda nbytes: 0, None)
    chemo.chemo_set_allocator(lambda nbytes: 0, lambda ptr, nbytes: None)
    chemo.chemo_set_allocator(None, None)
    assert L.chemo_set_allocator(None, None, None) == chemo.OK


def test_status_strings(chemo):
    assert chemo.chemo_status_string(0) == "ok"
    assert "invalid" in chemo.chemo_status_string(chemo.EINVAL)
    assert chemo.chemo_status_string(12345) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(dim=4), dict(n_species=0), dict(n_species=9), dict(dt=0.0), dict(grid=[2, 64, 1]),
    dict(boundary=1, pde_bc=0), dict(boundary=0, pde_bc=2), dict(cutoff_mode=3), dict(search_mode=5),
    dict(hi=[0.0, 1.0, 1.0]), dict(react_to=[5, 0]), dict(warp_runs=33), dict(move_scheme=2),
    dict(hard_sphere=2), dict(deposit_kernel=2), dict(kde_range=-1.0),
    dict(deposit_kernel=1, chem_mode=1), dict(deposit_kernel=1, diameter=[0.0, 0.01]),
])
def test_invalid_parameters_rejected_on_host(chemo, bad):
    from paper_1805_11007_gb300 import workloads as wl
    p = wl.params("walls_grid_2d", grid=[64, 64, 1])
    p.update(bad)
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_create(p, np.zeros((0, p["dim"] if p["dim"] in (2, 3) else 2), np.float32),
                           np.zeros(0, np.uint8))
    assert ei.value.status == chemo.EINVAL


def test_struct_size_mismatch_rejected(chemo):
    from paper_1805_11007_gb300 import workloads as wl
    prm = chemo.make_params(wl.params("walls_grid_2d"))
    prm.struct_size = 12
    out = ctypes.c_void_p()
    st = chemo.lib().chemo_create(ctypes.byref(prm), 0, None, None, 0, None, ctypes.byref(out))
    assert st == chemo.EINVAL
    assert "struct_size" in chemo.chemo_last_error()


def test_plain_c_program_uses_the_library(chemo, tmp_path):
    """The ABI needs no Python: a C program built against include/chemo.h
    and linked to the library gets status strings, sets and resets an
    allocator, and sees a bad parameter set rejected before any GPU work."""
    prog = tmp_path / "use.c"
    prog.write_text(r"""
#include <stdio.h>
#include <string.h>
#include "chemo.h"
static int my_alloc(void *ctx, size_t bytes, void **ptr) { (void)ctx; (void)bytes; *ptr = 0; return 1; }
static void my_release(void *ctx, void *ptr, size_t bytes) { (void)ctx; (void)ptr; (void)bytes; }
int main(void) {
    chemo_params p;
    chemo_sim *sim = 0;
    int st;
    memset(&p, 0, sizeof p);
    p.struct_size = sizeof p;
    p.dim = 4; /* invalid */
    p.n_species = 1;
    p.hi[0] = p.hi[1] = p.hi[2] = 1.0;
    p.dt = 1e-5;
    st = chemo_create(&p, 0, 0, 0, CHEMO_MEM_HOST, 0, &sim);
    printf("%d %s|%s|%d\n", st, chemo_status_string(st), chemo_last_error(), sim == 0);
    printf("%d %d %d\n", chemo_set_allocator(my_alloc, 0, 0), chemo_set_allocator(my_alloc, my_release, 0),
           chemo_set_allocator(0, 0, 0));
    chemo_destroy(0);
    return 0;
}
""")
    exe = tmp_path / "use"
    libdir = os.path.dirname(gb.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(prog), "-o",
                    str(exe), "-L", libdir, "-lchemo_gb300", "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    st, rest = out[0].split(" ", 1)
    assert int(st) == chemo.EINVAL
    text, msg, null_out = rest.split("|")
    assert "invalid" in text and "dim" in msg and null_out == "1"
    assert out[1].split() == [str(chemo.EINVAL), "0", "0"]


def test_gradient_needs_a_simulation(chemo):
    st = chemo.lib().chemo_gradient(None, None, None, None, None, 0, None)
    assert st == chemo.EINVAL
    st = chemo.lib().chemo_record(None, 1, 1, None)
    assert st == chemo.EINVAL


@pytest.mark.parametrize("case", ["dim3", "zero", "negative", "too_many"])
def test_batch_arguments_rejected_on_host(chemo, case):
    """chemo_create_batch validates its replicate arguments before touching
    the device: 3D ensembles, no replicates, negative sizes, > 65535."""
    from paper_1805_11007_gb300 import workloads as wl
    p = wl.params("ensemble_2d")
    sizes = [0, 0]
    if case == "dim3":
        p = wl.params("clumps_grid_3d", grid=[8, 8, 8])
    elif case == "zero":
        sizes = []
    elif case == "negative":
        sizes = [3, -1]
    else:
        sizes = [0] * 65536
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_create_batch(p, sizes, np.zeros((0, p["dim"]), np.float32), np.zeros(0, np.uint8))
    assert ei.value.status == chemo.EINVAL


def test_autotune_needs_trial_steps(chemo):
    from paper_1805_11007_gb300 import workloads as wl
    p = wl.params("ensemble_2d")
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_autotune(p, [0], np.zeros((0, 2), np.float32), np.zeros(0, np.uint8), trial_steps=0)
    assert ei.value.status == chemo.EINVAL


def test_slab_structs_match_the_binding(chemo, tmp_path):
    """chemo_cell is 32 bytes laid out as CELL_DTYPE; chemo_slab_target as
    the ctypes structure."""
    prog = tmp_path / "slab.c"
    cell = list(chemo.CELL_DTYPE.names)
    tgt = [f for f, _ in chemo.chemo_slab_target._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "chemo.h"', "int main(void){",
             'printf("%zu %zu\\n", sizeof(chemo_cell), sizeof(chemo_slab_target));']
    lines += ['printf("c %s %%zu\\n", offsetof(chemo_cell, %s));' % (f, f) for f in cell]
    lines += ['printf("t %s %%zu\\n", offsetof(chemo_slab_target, %s));' % (f, f) for f in tgt]
    lines += ['printf("g %u %u %u\\n", CHEMO_GHOST_ID, CHEMO_OPEN_ZLO, CHEMO_OPEN_ZHI);', "return 0;}"]
    prog.write_text("\n".join(lines))
    exe = tmp_path / "slab"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()
    sc, st = map(int, out[0].split())
    assert sc == chemo.CELL_DTYPE.itemsize == 32
    assert st == ctypes.sizeof(chemo.chemo_slab_target)
    for line in out[1:]:
        f = line.split()
        if f[0] == "c":
            assert chemo.CELL_DTYPE.fields[f[1]][1] == int(f[2]), f[1]
        elif f[0] == "t":
            assert getattr(chemo.chemo_slab_target, f[1]).offset == int(f[2]), f[1]
        else:
            assert [int(v) for v in f[1:]] == [chemo.GHOST_ID, chemo.OPEN_ZLO, chemo.OPEN_ZHI]


@pytest.mark.parametrize("case,status", [("dim2", "EINVAL"), ("periodic", "ENOTSUP"), ("hard_sphere", "ENOTSUP"),
                                         ("kde", "ENOTSUP"), ("fixed_gradient", "ENOTSUP"),
                                         ("capacity", "EINVAL"), ("faces", "EINVAL")])
def test_subdomain_arguments_rejected_on_host(chemo, case, status):
    """chemo_create_subdomain checks its arguments before touching the
    device: 3D walls with a grid, no hard spheres or kernel density, a
    capacity of 1 .. 2^29 - 1, face bits 0 and 1 only."""
    from paper_1805_11007_gb300 import workloads as wl
    p = wl.params("clumps_grid_3d", grid=[8, 8, 8])
    cap, faces = 100, chemo.OPEN_ZLO | chemo.OPEN_ZHI
    if case == "dim2":
        p = wl.params("walls_grid_2d")
    elif case == "periodic":
        p = dict(p, boundary=1, pde_bc=2)
    elif case == "hard_sphere":
        p = dict(p, hard_sphere=1)
    elif case == "kde":
        p = dict(p, deposit_kernel=1)
    elif case == "fixed_gradient":
        p = dict(p, chem_mode=1)
    elif case == "capacity":
        cap = 0
    else:
        faces = 4
    with pytest.raises(chemo.ChemoError) as ei:
        chemo.chemo_create_subdomain(p, cap, faces)
    assert ei.value.status == getattr(chemo, status)


def test_slab_calls_need_a_subdomain(chemo):
    L = chemo.lib()
    assert L.chemo_slab_ingest(None, 0, None, chemo.MEM_HOST, None) == chemo.EINVAL
    assert L.chemo_slab_select(None, 0, None, None) == chemo.EINVAL
    assert L.chemo_slab_planes(None, 0, 0, 0, 0, None, None) == chemo.EINVAL
    assert L.chemo_step_particles(None, None) == chemo.EINVAL
    assert L.chemo_step_field(None, None) == chemo.EINVAL
