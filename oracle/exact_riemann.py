"""Exact solution of the 1D Riemann problem for an ideal gas (test oracle).

The shock tubes of Sec. 4.2 are compared with the exact (semi-analytic)
solution.  The solution is the textbook one (e.g. Toro, *Riemann Solvers and
Numerical Methods for Fluid Dynamics*, ch. 4), restated here from the
mathematics:

* Across a shock into state K (pressure p > p_K) the velocity jump follows
  from the Rankine-Hugoniot conditions,
  f_K(p) = (p - p_K) sqrt(A_K / (p + B_K)),  A_K = 2 / ((g+1) rho_K),
  B_K = (g-1)/(g+1) p_K.
* Across a rarefaction (p <= p_K) the isentrope and the Riemann invariant give
  f_K(p) = 2 c_K/(g-1) ((p/p_K)^((g-1)/(2g)) - 1).
* The star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0 and the star
  velocity is u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2.

``star_state`` finds p* by Newton iteration; ``star_pressure_bisect`` finds it
independently by bisection, so the two can pin each other.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def _fk(p: float, rho: float, pk: float, g: float) -> Tuple[float, float]:
    """f_K(p) and its derivative."""
    ck = math.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    r = p / pk
    e = (g - 1.0) / (2.0 * g)
    return 2.0 * ck / (g - 1.0) * (r ** e - 1.0), (1.0 / (rho * ck)) * r ** (-(g + 1.0) / (2.0 * g))


def star_state(left, right, g: float, tol: float = 1e-15, maxit: int = 200) -> Tuple[float, float]:
    """(p*, u*) by Newton iteration on the pressure function."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    if 2.0 * (cl + cr) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum is generated; not handled")
    p = max(0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr), 1e-8)
    for _ in range(maxit):
        fl, dl = _fk(p, rl, pl, g)
        fr, dr = _fk(p, rr, pr, g)
        pn = p - (fl + fr + ur - ul) / (dl + dr)
        if pn <= 0.0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, g)
    fr, _ = _fk(p, rr, pr, g)
    return p, 0.5 * (ul + ur) + 0.5 * (fr - fl)


def star_pressure_bisect(left, right, g: float) -> float:
    """p* by bisection on f_L + f_R + du (independent of the Newton path)."""
    rl, ul, pl = left
    rr, ur, pr = right

    def F(p):
        return _fk(p, rl, pl, g)[0] + _fk(p, rr, pr, g)[0] + (ur - ul)

    a, b = 1e-14, 1.0
    while F(b) < 0.0:
        b *= 2.0
    for _ in range(400):
        m = 0.5 * (a + b)
        if F(m) > 0.0:
            b = m
        else:
            a = m
        if b - a <= 4e-16 * b:
            break
    return 0.5 * (a + b)


def sample(left, right, g: float, xi: np.ndarray) -> np.ndarray:
    """Exact (rho, u, p) at similarity coordinates xi = (x - x0)/t.
    Returns an array of shape (3, len(xi))."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    gm1, gp1 = g - 1.0, g + 1.0
    out = np.zeros((3, len(xi)))
    for i, s in enumerate(np.asarray(xi, dtype=np.float64)):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt(gp1 / (2 * g) * ps / pl + gm1 / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + gm1 / gp1) / (gm1 / gp1 * ps / pl + 1.0)
                    w = (r, us, ps)
            else:  # left rarefaction
                csl = cl * (ps / pl) ** (gm1 / (2 * g))
                head, tail = ul - cl, us - csl
                if s <= head:
                    w = (rl, ul, pl)
                elif s >= tail:
                    w = (rl * (ps / pl) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / gp1 * (cl + gm1 / 2.0 * ul + s)
                    c = 2.0 / gp1 * (cl + gm1 / 2.0 * (ul - s))
                    r = rl * (c / cl) ** (2.0 / gm1)
                    w = (r, u, pl * (c / cl) ** (2.0 * g / gm1))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt(gp1 / (2 * g) * ps / pr + gm1 / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + gm1 / gp1) / (gm1 / gp1 * ps / pr + 1.0)
                    w = (r, us, ps)
            else:  # right rarefaction
                csr = cr * (ps / pr) ** (gm1 / (2 * g))
                head, tail = ur + cr, us + csr
                if s >= head:
                    w = (rr, ur, pr)
                elif s <= tail:
                    w = (rr * (ps / pr) ** (1.0 / g), us, ps)
                else:
                    u = 2.0 / gp1 * (-cr + gm1 / 2.0 * ur + s)
                    c = 2.0 / gp1 * (cr - gm1 / 2.0 * (ur - s))
                    r = rr * (c / cr) ** (2.0 / gm1)
                    w = (r, u, pr * (c / cr) ** (2.0 * g / gm1))
        out[:, i] = w
    return out


def cell_averages(left, right, g: float, x0: float, t: float, edges: np.ndarray, sub: int = 64) -> np.ndarray:
    """Exact solution averaged over each cell [edges[i], edges[i+1]] with
    ``sub`` midpoint samples per cell (the discontinuities make point values
    at centres a poor comparison)."""
    n = len(edges) - 1
    xs = (edges[:-1, None] + (np.arange(sub)[None, :] + 0.5) / sub * np.diff(edges)[:, None]).ravel()
    w = sample(left, right, g, (xs - x0) / t)
    return w.reshape(3, n, sub).mean(axis=2)
