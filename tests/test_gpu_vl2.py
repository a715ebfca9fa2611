"""Parity of the CUDA van Leer integrator (Sec. 3.3, memory-optimized
predictor-corrector) with the FP64 CPU oracle, through the C ABI.

Gates as for the Heun path: all-FP64 bitwise (relative L1 <= 1e-12 as the
written bound), mixed <= 1e-5 in density and <= 1e-4 in pressure, all-FP32
<= 1e-4; conservation <= 1e-14 relative per step (FP64 state).  The
half-step primitives are stored in FP32 in the mixed path, which the mixed
gate covers.
"""
import numpy as np
import pytest

import oracle
from hydro_util import check_fields, field_errors, gpu_run, oracle_run, step_with_totals
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
SINGLE_TOL = 1e-4
VL = wl.INT_VL2
PRECS = [wl.PREC_FP64, wl.PREC_MIXED, wl.PREC_FP32]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    oracle.set_threads(0)


def check(mesh, U, Uo, prec):
    errs = field_errors(mesh, U, Uo)
    if prec == wl.PREC_FP64:
        np.testing.assert_array_equal(U, Uo)
        assert max(errs) <= FP64_TOL, errs
    elif prec == wl.PREC_MIXED:
        check_fields(mesh, U, Uo, False)
    else:
        check_fields(mesh, U, Uo, False, gates=[SINGLE_TOL] * (mesh.nvar + 1))
    return errs


@pytest.mark.parametrize("prec", PRECS)
def test_vl2_sod_512_full_run(prec):
    mesh, W = wl.sod(512, prec=prec)
    mesh = mesh.replace(integrator=VL)
    Uo, to, so, _ = oracle_run(mesh, W, 0.2)
    U, t, s, _ = gpu_run(mesh, W, 0.2)
    assert t == to == 0.2
    if prec == wl.PREC_FP64:
        assert s == so
    errs = field_errors(mesh, U, Uo)
    tol = 1e-3 if prec == wl.PREC_FP32 else None  # FP32 state over ~600 steps
    if tol:
        assert errs[0] <= tol and errs[-1] <= tol, errs
    else:
        check(mesh, U, Uo, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [(64, 64), (130, 70), (257, 33), (5, 9), (2, 2)])
def test_vl2_2d_random_state_periodic(prec, n):
    mesh = wl.Mesh(ndim=2, n=(n[0], n[1], 1), gamma=1.4, cfl=0.4, prec=prec, integrator=VL)
    W = wl.random_jumpy(mesh, seed=n[0] * 7 + n[1])
    Uo, _, so, _ = oracle_run(mesh, W, max_steps=6)
    U, _, s, _ = gpu_run(mesh, W, max_steps=6)
    assert s == so == 6
    check(mesh, U, Uo, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [(32, 16, 40), (37, 11, 9), (2, 3, 2), (66, 10, 35)])
def test_vl2_3d_random_state_periodic(prec, n):
    mesh = wl.Mesh(ndim=3, n=n, gamma=5.0 / 3.0, cfl=0.3, prec=prec, integrator=VL)
    W = wl.random_jumpy(mesh, seed=sum(n))
    Uo, _, so, _ = oracle_run(mesh, W, max_steps=4)
    U, _, s, _ = gpu_run(mesh, W, max_steps=4)
    assert s == so == 4
    check(mesh, U, Uo, prec)


BCS = [
    ((wl.BC_OUTFLOW, wl.BC_REFLECT), (wl.BC_FREE, wl.BC_OUTFLOW), (wl.BC_REFLECT, wl.BC_FREE)),
    ((wl.BC_REFLECT, wl.BC_REFLECT), (wl.BC_PERIODIC, wl.BC_PERIODIC), (wl.BC_OUTFLOW, wl.BC_OUTFLOW)),
]


@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_vl2_boundaries(prec, bc, ndim):
    n = {1: (67, 1, 1), 2: (45, 38, 1), 3: (21, 14, 17)}[ndim]
    mesh = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3, prec=prec, bc=bc, integrator=VL)
    W = wl.random_smooth(mesh, seed=ndim)
    Uo, _, so, _ = oracle_run(mesh, W, max_steps=8)
    U, _, s, _ = gpu_run(mesh, W, max_steps=8)
    assert s == so
    check(mesh, U, Uo, prec)


@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
def test_vl2_turbulence_48(prec):
    mesh, W = wl.turbulence(48, prec=prec)
    mesh = mesh.replace(integrator=VL)
    Uo, _, so, _ = oracle_run(mesh, W, max_steps=20)
    U, _, s, _ = gpu_run(mesh, W, max_steps=20)
    assert s == so == 20
    check(mesh, U, Uo, prec)


@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
def test_vl2_implosion_reflecting(prec):
    mesh, W = wl.liska_wendroff(64, prec=prec)
    mesh = mesh.replace(integrator=VL)
    Uo, _, _, _ = oracle_run(mesh, W, max_steps=40)
    U, _, _, _ = gpu_run(mesh, W, max_steps=40)
    check(mesh, U, Uo, prec)
    if prec == wl.PREC_FP64:
        np.testing.assert_array_equal(U[0, 0], U[0, 0].T)


@pytest.mark.parametrize("prec", [wl.PREC_MIXED, wl.PREC_FP64])
def test_vl2_turbulence_256_full_size(prec):
    mesh, W = wl.turbulence(256, prec=prec)
    mesh = mesh.replace(integrator=VL)
    Uo, _, _, _ = oracle_run(mesh, W, max_steps=2)
    U, _, s, _ = gpu_run(mesh, W, max_steps=2)
    assert s == 2
    check(mesh, U, Uo, prec)


@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_vl2_conservation_per_step(prec, ndim):
    from paper_2501_02317_gb300 import khydro
    n = {1: (300, 1, 1), 2: (96, 80, 1), 3: (40, 24, 36)}[ndim]
    mesh = wl.Mesh(ndim=ndim, n=n, gamma=5.0 / 3.0, cfl=0.3, prec=prec, integrator=VL)
    W = wl.random_jumpy(mesh, seed=4)
    with khydro.Sim(mesh) as sim:
        sim.set_primitive(W)
        step_with_totals(sim, mesh, 10, drift_tol=1e-14)


def test_vl2_uniform_state_and_axis_interchange():
    for prec in (wl.PREC_FP64, wl.PREC_MIXED):
        m = wl.Mesh(ndim=3, n=(20, 9, 7), gamma=5.0 / 3.0, cfl=0.3, prec=prec, integrator=VL)
        W = wl.uniform(m)
        U, _, _, _ = gpu_run(m, W, max_steps=12)
        np.testing.assert_array_equal(U, oracle.prim_to_cons(m, W))
    m1, W1 = wl.sod(96, axis=0, ndim=1)
    U1, _, s1, _ = gpu_run(m1.replace(integrator=VL), W1, 0.2)
    for ndim, axis in [(2, 1), (3, 2), (3, 0)]:
        m, W = wl.sod(96, axis=axis, ndim=ndim, ntrans=5)
        U, _, s, _ = gpu_run(m.replace(integrator=VL), W, 0.2)
        assert s == s1
        for row in np.moveaxis(U[0], 2 - axis, -1).reshape(-1, 96):
            np.testing.assert_array_equal(row, U1[0].ravel())


def test_vl2_split_run_equals_straight_run():
    from paper_2501_02317_gb300 import khydro
    for prec in (wl.PREC_MIXED, wl.PREC_FP64):
        mesh, W = wl.kelvin_helmholtz(96, prec=prec)
        mesh = mesh.replace(integrator=VL)
        Ua, ta, _, _ = gpu_run(mesh, W, max_steps=20)
        with khydro.Sim(mesh) as sim:
            sim.set_primitive(W)
            sim.step_to(1e30, 8)
            Umid = sim.conserved()
            tmid, _, _ = sim.time()
        with khydro.Sim(mesh) as sim2:
            sim2.set_conserved(Umid)
            sim2.set_time(tmid)
            s2, t2 = sim2.step_to(1e30, 12)
            Ub = sim2.conserved()
        assert s2 == 12 and t2 == ta
        np.testing.assert_array_equal(Ua, Ub)


def test_vl2_holds_less_device_memory():
    # the second state array becomes primitives in the flux precision:
    # mixed 40 + 20 bytes per 3D cell instead of 40 + 40 for the lean Heun
    # step (FP64: unchanged); the default Heun step also stores the
    # primitives of U^n and U^1
    from paper_2501_02317_gb300 import khydro
    m = wl.Mesh(ndim=3, n=(16, 12, 10), prec=wl.PREC_MIXED)
    sizes = {}
    for prec in (wl.PREC_FP64, wl.PREC_MIXED, wl.PREC_FP32):
        for integ in (wl.INT_HEUN, wl.INT_HEUN_LEAN, VL):
            with khydro.Sim(m.replace(prec=prec, integrator=integ)) as sim:
                sizes[prec, integ] = sim.device_bytes()[0]
    cb = 5 * 8 * 16 * 12 * 10  # one FP64 state
    assert sizes[wl.PREC_MIXED, wl.INT_HEUN_LEAN] == 2 * cb
    assert sizes[wl.PREC_MIXED, wl.INT_HEUN] == 3 * cb
    assert sizes[wl.PREC_MIXED, VL] == cb + cb // 2
    assert sizes[wl.PREC_FP64, VL] == sizes[wl.PREC_FP64, wl.INT_HEUN_LEAN] == 2 * cb
    assert sizes[wl.PREC_FP64, wl.INT_HEUN] == 4 * cb
    assert sizes[wl.PREC_FP32, VL] < sizes[wl.PREC_FP32, wl.INT_HEUN_LEAN]


def test_vl2_profile_and_dt_match_heun_dt():
    # the first dt of both integrators comes from the same CFL condition
    from paper_2501_02317_gb300 import khydro
    mesh, W = wl.kelvin_helmholtz(80, prec=wl.PREC_FP64)
    _, _, _, dt_h = gpu_run(mesh, W, max_steps=1)
    _, _, _, dt_v = gpu_run(mesh.replace(integrator=VL), W, max_steps=1)
    assert dt_h == dt_v
    with khydro.Sim(mesh.replace(integrator=VL, prec=wl.PREC_MIXED)) as sim:
        sim.set_primitive(W)
        ms = sim.profile_steps(1e30, 3)
        assert all(x > 0 for x in ms)
        assert sim.time()[1] == 3


def test_vl2_fp32_state_round_trip():
    # the FP32 state is converted field by field through the (smaller)
    # second array: set/get must still give the FP32-rounded values
    from paper_2501_02317_gb300 import khydro
    m = wl.Mesh(ndim=3, n=(9, 8, 7), prec=wl.PREC_FP32, integrator=VL)
    W = wl.random_jumpy(m)
    U = oracle.prim_to_cons(m, W)
    with khydro.Sim(m) as sim:
        sim.set_conserved(U)
        np.testing.assert_array_equal(sim.conserved(), U.astype(np.float32).astype(np.float64))
        sim.set_primitive(W)
        np.testing.assert_array_equal(sim.conserved(), U.astype(np.float32).astype(np.float64))
        np.testing.assert_allclose(sim.totals(), U.astype(np.float32).astype(np.float64).reshape(5, -1).sum(1),
                                   rtol=1e-12)


def test_vl2_rejected_where_unsupported():
    from paper_2501_02317_gb300 import khydro
    m = wl.Mesh(ndim=2, n=(16, 16, 1), prec=wl.PREC_MIXED, integrator=VL)
    with pytest.raises(khydro.KhydroError):
        khydro.Batch([m, m])
