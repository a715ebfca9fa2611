"""The oracle and the input recipes against what the paper prints
(tests/golden/paper_setups.json, each entry cited), and the oracle against
its own stored states (tests/golden/oracle_regression.json, written by
tests/golden/make_oracle_fixtures.py from the oracle alone).

* Sec. 4.1 wave tests at the paper's parameters (rho0 = 1, p0 = 5/3,
  gamma = 5/3, unit periodic box, t = 0 .. 1): sinusoidal contact and shear
  waves (A = 0.1, carried once around the box by v = 1) converge as N^-2 in
  the Eq. 6 L1 norm, the top-hat more slowly than N^-1, and v = -1 gives the
  same errors; the FP64 sound wave (A = 1e-6) keeps converging as N^-2 beyond
  N = 10^3, measured against the linear solution translated by c_s t.
* Sec. 4.4, Eq. 7: the implosion's initial state.
* Regression: two oracle runs reproduce the stored exact doubles.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2501_02317_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PAPER = json.load(open(os.path.join(GOLDEN, "paper_setups.json")))
WAVE = PAPER["wave_tests"]


def l1_eq6(q, q0):
    """Eq. 6: sum |q - q0| / (N (max q0 - min q0))."""
    return float(np.abs(q - q0).sum() / (q0.size * (q0.max() - q0.min())))


def test_every_golden_entry_is_cited():
    for key, entry in PAPER.items():
        if key != "about":
            assert entry.get("cite"), key


def _wave_error(kind, profile, n, v):
    mesh, W = wl.advection_wave(n, kind, profile, amp=WAVE["amp_contact_shear"], v=v, rho0=WAVE["rho0"],
                                p0=WAVE["p0"], gamma=WAVE["gamma"])
    assert mesh.hi[0] - mesh.lo[0] == WAVE["l_box"]
    U, t, s, f = oracle.run(mesh, oracle.prim_to_cons(mesh, W), WAVE["t_start"], WAVE["t_end"])
    assert t == WAVE["t_end"] and f == 0
    Wf, _ = oracle.cons_to_prim(mesh, U)
    q = 0 if kind == "contact" else 2
    # one full period: the exact solution is the initial state
    return l1_eq6(Wf[q], W[q])


@pytest.mark.parametrize("kind", ["contact", "shear"])
def test_wave_convergence_at_paper_setup(kind):
    ns = (128, 256, 512)
    sine = [_wave_error(kind, "sine", n, 1.0) for n in ns]
    top = [_wave_error(kind, "tophat", n, 1.0) for n in ns]
    s_sine = [math.log2(sine[i] / sine[i + 1]) for i in range(2)]
    s_top = [math.log2(top[i] / top[i + 1]) for i in range(2)]
    # L1 ~ N^-2 for the sinusoid (minmod clips the extrema: the slope
    # approaches 2 from below), slower than N^-1 for the top-hat
    assert all(1.8 < s < 2.1 for s in s_sine), (sine, s_sine)
    assert all(0.3 < s < -WAVE["tophat_l1_slope_slower_than"] for s in s_top), (top, s_top)


@pytest.mark.parametrize("profile", ["sine", "tophat"])
def test_wave_background_speed_sign_gives_same_error(profile):
    ea, eb = (_wave_error("contact", profile, 128, v) for v in WAVE["background_speeds"])
    assert ea == pytest.approx(eb, rel=1e-10)


def test_sound_wave_fp64_converges_beyond_a_thousand_cells():
    errs = []
    ns = (256, 512, 1024)
    assert ns[-1] > WAVE["sound_fp64_converges_beyond_n"]
    for n in ns:
        mesh, W = wl.sound_wave(n, amp=WAVE["amp_sound_fp64"], p0=WAVE["p0"], rho0=WAVE["rho0"],
                                gamma=WAVE["gamma"])
        cs = wl.sound_speed(WAVE["p0"], WAVE["rho0"], WAVE["gamma"])
        U, t, s, f = oracle.run(mesh, oracle.prim_to_cons(mesh, W), WAVE["t_start"], WAVE["t_end"])
        assert t == WAVE["t_end"]
        x = (np.arange(n) + 0.5) / n
        exact = WAVE["rho0"] + WAVE["amp_sound_fp64"] * np.sin(2.0 * np.pi * (x - cs * t))
        errs.append(np.abs(U[0].ravel() - exact).sum() / (n * (W[0].max() - W[0].min())))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(ns) - 1)]
    assert all(s > 1.8 for s in slopes), (errs, slopes)


def test_implosion_initial_state_is_eq7():
    lw = PAPER["liska_wendroff"]
    mesh, W = wl.liska_wendroff(40)
    assert mesh.gamma == lw["gamma"]
    for d in range(2):
        assert mesh.bc[d] == (wl.BC_REFLECT, wl.BC_REFLECT)
    x, y, _ = (np.broadcast_to(c, mesh.shape[1:]) for c in wl._grids(mesh))
    inner = x + y < 0.15
    assert inner.any() and (~inner).any()
    for region, mask in (("inner", inner), ("outer", ~inner)):
        v = lw[region]
        assert np.all(W[0][mask] == v["rho"])
        assert np.all(W[3][mask] == v["p"])
        assert np.all(W[1][mask] == v["v"]) and np.all(W[2][mask] == v["v"])


@pytest.mark.parametrize("name", ["sod_512_t0.2", "implosion_48_60_steps"])
def test_oracle_reproduces_stored_states(name):
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_oracle_fixtures", os.path.join(GOLDEN, "make_oracle_fixtures.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored = json.load(open(os.path.join(GOLDEN, "oracle_regression.json")))[name]
    assert mk.compute(name) == stored
