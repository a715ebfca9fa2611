"""The CUDA path against the bounds and behaviour the paper prints
(tests/golden/paper_setups.json, each entry cited):

* Sec. 3.2.2: the mixed-precision flux stays within 1e-3 relative of the
  double-precision one -- checked on the one-step update U1 - Un (the flux
  divergence times dt) of the mixed path against the all-FP64 path, on
  shock, shear-layer, implosion and random states in 1D, 2D and 3D;
* Sec. 4.1: with A = 0.1 the contact and shear wave errors of the mixed
  path are almost those of the FP64 path; with A = 1e-4 the mixed and FP32
  sound waves still converge up to N ~ 10^2.
"""
import json
import math
import os

import numpy as np
import pytest

from hydro_util import gpu_run, rel_l1
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PAPER = json.load(open(os.path.join(GOLDEN, "paper_setups.json")))
WAVE = PAPER["wave_tests"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()


def _cases():
    m3 = wl.Mesh(ndim=3, n=(24, 20, 16), gamma=1.4, cfl=0.3)
    m2 = wl.Mesh(ndim=2, n=(70, 66, 1), gamma=5.0 / 3.0, cfl=0.4)
    yield "sod", wl.sod(512)
    yield "kelvin_helmholtz", wl.kelvin_helmholtz(128)
    yield "implosion", wl.liska_wendroff(96)
    yield "random_2d", (m2, wl.random_jumpy(m2))
    yield "random_3d", (m3, wl.random_jumpy(m3))
    yield "turbulence", wl.turbulence(32)


@pytest.mark.parametrize("name", ["sod", "kelvin_helmholtz", "implosion", "random_2d", "random_3d", "turbulence"])
def test_mixed_update_within_paper_bound(name):
    mesh, W = dict(_cases())[name]
    bound = PAPER["hllc_mixed_vs_fp64"]["relative_error_below"]
    dU = {}
    for prec in (wl.PREC_FP64, wl.PREC_MIXED):
        m = mesh.replace(prec=prec)
        from paper_2501_02317_gb300 import khydro
        with khydro.Sim(m) as sim:
            sim.set_primitive(np.ascontiguousarray(W))
            U0 = sim.conserved()
            s, _ = sim.step_to(1e30, 1)
            assert s == 1
            dU[prec] = sim.conserved() - U0
    for q in range(mesh.nvar):
        ref = dU[wl.PREC_FP64][q]
        if np.abs(ref).sum() == 0.0:  # e.g. a velocity component nothing moves
            assert np.abs(dU[wl.PREC_MIXED][q]).max() == 0.0
            continue
        assert rel_l1(dU[wl.PREC_MIXED][q], ref) < bound, (name, q)


def _wave_l1(kind, n, prec):
    mesh, W = wl.advection_wave(n, kind, "sine", amp=WAVE["amp_contact_shear"], v=WAVE["background_speeds"][0],
                                rho0=WAVE["rho0"], p0=WAVE["p0"], gamma=WAVE["gamma"], prec=prec)
    U, t, s, _ = gpu_run(mesh, W, WAVE["t_end"])
    assert t == WAVE["t_end"]
    q = 0 if kind == "contact" else 2
    qf = U[0] if kind == "contact" else U[2] / U[0]
    return float(np.abs(qf - W[q]).sum() / (W[q].size * (W[q].max() - W[q].min())))


@pytest.mark.parametrize("kind", ["contact", "shear"])
def test_mixed_wave_errors_match_fp64(kind):
    for n in (64, 256):
        e64, emx = _wave_l1(kind, n, wl.PREC_FP64), _wave_l1(kind, n, wl.PREC_MIXED)
        assert abs(emx - e64) <= 1e-3 * e64, (kind, n, e64, emx)


@pytest.mark.parametrize("prec", [wl.PREC_MIXED, wl.PREC_FP32])
def test_reduced_precision_sound_wave_converges_to_a_hundred_cells(prec):
    # Sec. 4.1: with A = 1e-4 the mixed and FP32 errors fall with resolution
    # up to N ~ 10^2 and stop falling beyond; below that they are the
    # discretisation error of the scheme, i.e. the FP64 oracle's at the same
    # amplitude
    import oracle
    amp = WAVE["amp_sound_reduced_precision"]
    cs = wl.sound_speed(WAVE["p0"], WAVE["rho0"], WAVE["gamma"])
    ns = (32, 64, 128)
    assert ns[-1] >= WAVE["sound_reduced_precision_stalls_beyond_n"]
    errs, ref = [], []
    for n in ns:
        mesh, W = wl.sound_wave(n, amp=amp, p0=WAVE["p0"], rho0=WAVE["rho0"], gamma=WAVE["gamma"], prec=prec)
        x = (np.arange(n) + 0.5) / n
        exact = WAVE["rho0"] + amp * np.sin(2.0 * np.pi * (x - cs * WAVE["t_end"]))
        span = n * (W[0].max() - W[0].min())
        U, t, s, _ = gpu_run(mesh, W, WAVE["t_end"])
        assert t == WAVE["t_end"]
        errs.append(np.abs(U[0].ravel() - exact).sum() / span)
        Uo, to, so, fo = oracle.run(mesh.replace(prec=wl.PREC_FP64), oracle.prim_to_cons(mesh, W), 0.0, WAVE["t_end"])
        ref.append(np.abs(Uo[0].ravel() - exact).sum() / span)
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert all(sl >= 1.0 for sl in slopes), (errs, slopes)
    for i, n in enumerate(ns):
        if n <= 64:
            assert abs(errs[i] - ref[i]) <= 0.05 * ref[i], (n, errs[i], ref[i])
