"""Shock tubes beyond Sod (Sec. 4.2: the scheme follows the exact solution
across a range of Riemann problems): a strong shock (pressure ratio 2.5e4),
a double rarefaction close to vacuum, colliding streams, a moving contact and
a shock running into gas at rest.  The oracle against the exact solution
(oracle/exact_riemann.py, itself pinned by Newton vs bisection and the
Rankine-Hugoniot jumps): first-order-at-discontinuity errors below fixed
bounds at 512 cells and falling with resolution; the moving contact keeps
v and p to round-off (HLLC resolves an isolated contact exactly)."""
import numpy as np
import pytest

import oracle
from hydro_util import SHOCK_TUBES, tube_errors
from paper_2501_02317_gb300 import workloads as wl

# bounds on (rho, v, p) errors at 512 cells, about twice the measured values
BOUNDS = {
    "strong_shock": (1.5e-2, 1.1e-2, 4.1e-3),
    "double_rarefaction": (8.3e-3, 1.4e-2, 8.0e-3),
    "colliding_streams": (1.3e-3, 1.8e-3, 9.3e-4),
    "moving_contact": (2.8e-3, 1e-13, 1e-13),
    "shock_into_rest": (2.5e-3, 4.0e-3, 2.3e-3),
}


def _run(name, n):
    left, right, x0, t = SHOCK_TUBES[name]
    mesh, W = wl.shock_tube(n, left, right, x0)
    U, tt, s, f = oracle.run(mesh, oracle.prim_to_cons(mesh, W), 0.0, t)
    assert tt == t and f == 0
    Wf, _ = oracle.cons_to_prim(mesh, U)
    return tube_errors(left, right, x0, t, mesh.gamma, Wf)


@pytest.mark.parametrize("name", sorted(SHOCK_TUBES))
def test_shock_tube_against_exact_solution(name):
    e512 = _run(name, 512)
    assert all(e <= b for e, b in zip(e512, BOUNDS[name])), (name, e512)
    e256 = _run(name, 256)
    assert e512[0] < e256[0], (name, e256, e512)  # the density error falls with resolution


def test_moving_contact_keeps_velocity_and_pressure():
    left, right, x0, t = SHOCK_TUBES["moving_contact"]
    mesh, W = wl.shock_tube(512, left, right, x0)
    U, _, _, _ = oracle.run(mesh, oracle.prim_to_cons(mesh, W), 0.0, t)
    Wf, _ = oracle.cons_to_prim(mesh, U)
    np.testing.assert_allclose(Wf[1].ravel(), 0.15, rtol=1e-13)
    np.testing.assert_allclose(Wf[2].ravel(), 1.0, rtol=1e-13)
