"""Pins for the oracle's time integrators (Sec. 3.3), fixed by the mathematics.

* Contact advection: with uniform velocity and pressure the Euler equations
  reduce to linear advection of the density, the HLLC flux resolves the
  contact exactly (upwind mass flux), and both integrators must reduce to the
  textbook scalar schemes written out independently below: the Heun
  (RK2) method-of-lines PLM scheme, and the van Leer predictor-corrector
  (first-order half step, PLM full step from the half-step values).
* Van Leer integrator on the whole scheme: conservation to round-off, a
  uniform state stays uniform, second-order convergence on the sound wave
  (Sec. 4.1, Eq. 6), Sod against the exact solution (Sec. 4.2), bitwise axis
  interchange (Sec. 4.2) and the diagonal symmetry of the implosion (Sec. 4.4).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact_riemann as er
from paper_2501_02317_gb300 import workloads as wl

import test_oracle_pins as pins


# ------------------------------------------------ scalar advection schemes

def _minmod(a, b):
    same = ((a > 0) & (b > 0)) | ((a < 0) & (b < 0))
    return np.where(same, np.where(np.abs(a) < np.abs(b), a, b), 0.0)


def _face_states(r, order):
    """(left, right) states at face i+1/2 of a periodic row: left from cell
    i, right from cell i+1; piecewise constant (order 1) or minmod PLM."""
    if order == 1:
        return r, np.roll(r, -1)
    s = _minmod(r - np.roll(r, 1), np.roll(r, -1) - r)
    return r + 0.5 * s, np.roll(r - 0.5 * s, -1)


def _advect_rhs(r, u, dtdx, order):
    left, right = _face_states(r, order)
    F = u * (left if u > 0 else right)  # upwind flux at face i+1/2
    return -dtdx * (F - np.roll(F, 1))


def _advection_setup(u, n=64):
    m = wl.Mesh(ndim=1, n=(n, 1, 1), gamma=1.4, cfl=0.4)
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.4 * np.sin(2 * math.pi * x) + 0.5 * ((x > 0.3) & (x < 0.55))
    W = np.zeros(m.shape)
    W[0, 0, 0] = rho
    W[1, 0, 0] = u
    W[2, 0, 0] = 1.0
    return m, W


@pytest.mark.parametrize("integrator", [wl.INT_HEUN, wl.INT_VL2])
@pytest.mark.parametrize("u", [0.5, -0.35, 2.5])
def test_contact_advection_reduces_to_scalar_scheme(integrator, u):
    m, W = _advection_setup(u)
    U = oracle.prim_to_cons(m, W)
    r = W[0, 0, 0].copy()
    dx = 1.0 / m.n[0]
    step = oracle.vl2_step if integrator == wl.INT_VL2 else oracle.heun_step
    t = 0.0
    for _ in range(30):
        U, t, dt, f = step(m, U, t, 100.0)
        assert f == 0
        c = dt / dx
        if integrator == wl.INT_VL2:
            rh = r + _advect_rhs(r, u, 0.5 * c, 1)
            r = r + _advect_rhs(rh, u, c, 2)
        else:
            r1 = r + _advect_rhs(r, u, c, 2)
            r = 0.5 * (r + (r1 + _advect_rhs(r1, u, c, 2)))
    np.testing.assert_allclose(U[0, 0, 0], r, rtol=0, atol=1e-12)
    Wf, _ = oracle.cons_to_prim(m, U)
    np.testing.assert_allclose(Wf[1, 0, 0], u, rtol=1e-12)
    np.testing.assert_allclose(Wf[2, 0, 0], 1.0, rtol=1e-12)


def test_integrators_differ():
    # the two integrators are different schemes: same dt, different states
    m, W = _advection_setup(0.5)
    U0 = oracle.prim_to_cons(m, W)
    Ua, _, dta, _ = oracle.heun_step(m, U0, 0.0, 1.0)
    Ub, _, dtb, _ = oracle.vl2_step(m, U0, 0.0, 1.0)
    assert dta == dtb
    assert np.abs(Ua - Ub).max() > 1e-6


# ------------------------------------------------ van Leer, whole scheme

VL = wl.INT_VL2


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_vl2_conservation_periodic(ndim):
    n = {1: (64, 1, 1), 2: (24, 20, 1), 3: (12, 10, 8)}[ndim]
    m = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3, integrator=VL)
    W = wl.random_jumpy(m)
    U = oracle.prim_to_cons(m, W)
    t = 0.0
    for _ in range(5):
        Un, t, dt, f = oracle.vl2_step(m, U, t, 10.0)
        assert f == 0
        assert np.all(pins._rel_drift(m, U, Un) <= 1e-14)
        U = Un


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_vl2_uniform_state_stays_uniform(ndim):
    n = {1: (16, 1, 1), 2: (8, 6, 1), 3: (6, 5, 4)}[ndim]
    m = wl.Mesh(ndim=ndim, n=n, gamma=5.0 / 3.0, cfl=0.4, integrator=VL)
    U0 = oracle.prim_to_cons(m, wl.uniform(m))
    U, t, s, f = oracle.run(m, U0, 0.0, 1.0, 20)
    assert s == 20
    np.testing.assert_array_equal(U, U0)


def test_vl2_sound_wave_second_order():
    errs = []
    Ns = [64, 128, 256, 512]
    p0 = 3.0 / 5.0
    for n in Ns:
        m, W = wl.sound_wave(n, amp=1e-6, p0=p0)
        m = m.replace(integrator=VL)
        cs = wl.sound_speed(p0, 1.0, m.gamma)
        U0 = oracle.prim_to_cons(m, W)
        U, t, s, f = oracle.run(m, U0, 0.0, 1.0 / cs)
        errs.append(pins.l1_eq6(U[0], U0[0]))
    slopes = [math.log(errs[i + 1] / errs[i]) / math.log(2.0) for i in range(len(Ns) - 1)]
    assert slopes[-1] < -1.8 and slopes[-2] < -1.8, (errs, slopes)


def test_vl2_sod_against_exact_solution():
    m, W = wl.sod(512)
    m = m.replace(integrator=VL)
    U, t, s, f = oracle.run(m, oracle.prim_to_cons(m, W), 0.0, 0.2)
    assert t == 0.2 and f == 0
    Wf, _ = oracle.cons_to_prim(m, U)
    ex = er.cell_averages(pins.SOD_L, pins.SOD_R, 1.4, 0.5, 0.2, np.linspace(0.0, 1.0, 513))
    errs = [float(np.mean(np.abs(Wf[q].ravel() - ex[q]))) for q in range(3)]
    assert errs[0] < 3e-3 and errs[1] < 4e-3 and errs[2] < 2e-3, errs


def test_vl2_axis_interchange_identical():
    m1, W1 = wl.sod(96, axis=0, ndim=1)
    m1 = m1.replace(integrator=VL)
    U1, t1, s1, _ = oracle.run(m1, oracle.prim_to_cons(m1, W1), 0.0, 0.2)
    for ndim, axis in [(2, 1), (3, 2), (3, 0)]:
        m, W = wl.sod(96, axis=axis, ndim=ndim, ntrans=3)
        m = m.replace(integrator=VL)
        U, t, s, _ = oracle.run(m, oracle.prim_to_cons(m, W), 0.0, 0.2)
        assert s == s1 and t == t1
        rho = np.moveaxis(U[0], 2 - axis, -1).reshape(-1, 96)
        E = np.moveaxis(U[-1], 2 - axis, -1).reshape(-1, 96)
        for row in range(rho.shape[0]):
            np.testing.assert_array_equal(rho[row], U1[0].ravel())
            np.testing.assert_array_equal(E[row], U1[2].ravel())


def test_vl2_implosion_diagonal_symmetry():
    m, W = wl.liska_wendroff(48)
    m = m.replace(integrator=VL)
    U, t, s, f = oracle.run(m, oracle.prim_to_cons(m, W), 0.0, 0.2, 60)
    np.testing.assert_array_equal(U[0, 0], U[0, 0].T)
    np.testing.assert_array_equal(U[1, 0], U[2, 0].T)
    np.testing.assert_array_equal(U[3, 0], U[3, 0].T)
