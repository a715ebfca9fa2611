"""The smallest grids the library accepts, against the FP64 oracle.

An active axis needs two cells; with the two-cell ghost zones of Sec. 3.1.1
a grid of two or three cells is narrower than its halo, so every ghost cell
maps back into the grid -- periodic wrap onto the other side, a reflecting
wall onto a mirrored cell that is also the far wall's neighbour, outflow
onto the edge cell -- and every tile is ragged (a few active lanes of a
32-wide tile row).  Thin slabs (one axis of two cells in an otherwise
larger grid) and cells-in-a-row shapes are covered too.  All-FP64 path:
bitwise equal to the oracle; mixed path: within the stated gates; both with
every integrator.
"""
import numpy as np
import pytest

import oracle
from hydro_util import check_fields, gpu_run, oracle_run
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    oracle.set_threads(0)


P, R, O, F = wl.BC_PERIODIC, wl.BC_REFLECT, wl.BC_OUTFLOW, wl.BC_FREE

CASES = [
    (1, (2, 1, 1), ((P, P),)),
    (1, (3, 1, 1), ((R, O),)),
    (1, (2, 1, 1), ((F, R),)),
    (2, (2, 2, 1), ((P, P), (R, R))),
    (2, (3, 2, 1), ((O, F), (P, P))),
    (2, (2, 37, 1), ((R, O), (P, P))),
    (2, (45, 3, 1), ((P, P), (O, R))),
    (3, (2, 2, 2), ((P, P), (P, P), (P, P))),
    (3, (3, 2, 3), ((R, R), (O, F), (P, P))),
    (3, (2, 19, 35), ((P, P), (R, O), (P, P))),
    (3, (37, 2, 11), ((O, O), (P, P), (R, F))),
    (3, (33, 9, 2), ((P, P), (F, R), (P, P))),
]


@pytest.mark.parametrize("integrator", [wl.INT_HEUN, wl.INT_HEUN_LEAN, wl.INT_VL2])
@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_smallest_grids_against_oracle(case, prec, integrator):
    ndim, n, bc = CASES[case]
    bcs = tuple(bc) + ((P, P),) * (3 - ndim)
    mesh = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3, prec=prec, bc=bcs, integrator=integrator)
    W = wl.random_smooth(mesh, seed=10 + case)
    Uo, to, so, _ = oracle_run(mesh, W, max_steps=6)
    U, t, s, _ = gpu_run(mesh, W, max_steps=6)
    assert s == so == 6
    if prec == wl.PREC_FP64:
        np.testing.assert_array_equal(U, Uo)
        assert t == to
    check_fields(mesh, U, Uo, prec == wl.PREC_FP64)
