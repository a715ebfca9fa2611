"""The C ABI library loads, exports every declared entry point and rejects
invalid arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2501_02317_gb300 import build as kbuild
from paper_2501_02317_gb300 import khydro
from paper_2501_02317_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    kbuild.build()
    return khydro.lib()


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(khy_\w+)\s*\(", src, flags=re.M):
                names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["khy_create", "khy_destroy", "khy_set_boundary", "khy_set_primitive", "khy_set_conserved",
                 "khy_step_to", "khy_get_conserved", "khy_totals", "khy_last_error"]:
        assert want in names


def test_library_exports_every_declared_symbol(L):
    names = declared_functions()
    assert names
    for n in names:
        assert hasattr(L, n), "libkhydro.so does not export %s" % n
    assert set(khydro.EXPORTS) <= set(names)


def test_version(L):
    assert khydro.khy_version() >= 100


@pytest.mark.parametrize("bad", [
    dict(ndim=4),
    dict(ndim=0),
    dict(n=(1, 1, 1)),
    dict(n=(8, 2, 1)),          # ndim = 1 but n[1] != 1
    dict(gamma=1.0),
    dict(cfl=0.0),
    dict(cfl=1.5),
    dict(prec=7),
    dict(hi=(0.0, 1.0, 1.0)),
    dict(bc=((9, 0), (0, 0), (0, 0))),
    dict(rho_floor=-1.0),
    dict(ndim=3, n=(1 << 30, 1 << 30, 1 << 30)),   # the cell count's product would overflow
    dict(ndim=2, n=(1 << 16, 1 << 16, 1)),         # 2^32 cells
    dict(hi=(float("inf"), 1.0, 1.0)),
    dict(lo=(float("nan"), 0.0, 0.0)),
])
def test_create_rejects_invalid_descriptors(L, bad):
    base = dict(ndim=1, n=(8, 1, 1))
    base.update(bad)
    mesh = wl.Mesh(**base)
    with pytest.raises(khydro.KhydroError) as ei:
        khydro.khy_create(mesh)
    assert ei.value.status == -1
    assert khydro.lib().khy_last_error()


def test_null_arguments_rejected(L):
    assert L.khy_create(None, None, None) == -1
    assert L.khy_set_boundary(None, 0, 0, 0) == -1
    assert L.khy_step_to(None, 1.0, 1, None, None) == -1
    assert L.khy_totals(None, None) == -1
    L.khy_destroy(None)  # no-op


def test_desc_struct_layout_matches_header():
    # the ctypes mirror must have the C layout: offsets of the fields
    d = khydro.khy_mesh_desc
    assert d.ndim.offset == 0 and d.n.offset == 4 and d.lo.offset == 16
    assert d.hi.offset == 40 and d.gamma.offset == 64 and d.cfl.offset == 72 and d.prec.offset == 80
    assert d.bc.offset == 84 and d.integrator.offset == 108
    assert d.rho_floor.offset == 112 and d.p_floor.offset == 120
    assert ctypes.sizeof(d) == 128


def test_noalloc_scratch_limit_refused_on_the_host(L):
    # the size check of khy_step_noalloc runs before any CUDA call: meshes
    # one cell row or layer beyond the fixed scratch are refused with
    # KHY_ERR_ARG (the pointers are never touched on this path)
    src = open(os.path.join(ROOT, "include", "khydro.h")).read()
    m = re.search(r"#define KHY_NOALLOC_SCRATCH_BYTES \((\d+)u \* (\d+)u \* (\d+)u\)", src)
    assert m and int(m.group(1)) * int(m.group(2)) * int(m.group(3)) == khydro.KHY_NOALLOC_SCRATCH_BYTES
    for n in ((1024, 1025, 1), (95, 95, 95), (96, 96, 96)):
        mesh = wl.Mesh(ndim=2 if n[2] == 1 else 3, n=n, prec=wl.PREC_MIXED)
        assert mesh.nvar * mesh.ncell * 8 > khydro.KHY_NOALLOC_SCRATCH_BYTES
        with pytest.raises(khydro.KhydroError) as ei:
            khydro.khy_step_noalloc(mesh, 16, 0.0, 1.0, 16)
        assert ei.value.status == -1 and "no-allocation limit" in str(ei.value)
    for n in ((1024, 1024, 1), (94, 94, 94)):  # at or under the limit
        mesh = wl.Mesh(ndim=2 if n[2] == 1 else 3, n=n, prec=wl.PREC_MIXED)
        assert mesh.nvar * mesh.ncell * 8 <= khydro.KHY_NOALLOC_SCRATCH_BYTES
