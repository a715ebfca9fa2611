"""The seeded input generators follow the recipes of the benchmark configs
(no GPU): the shapes, sizes, value distributions and structure the parity
tests and the benchmark rely on.  Each check restates the recipe, not the
generator's code: values inside and outside the structures, the spectrum's
support and normalisation, the distributions of sizes and arrival gaps."""
import math

import numpy as np
import pytest

from paper_2501_02317_gb300 import workloads as wl


def _centres(n):
    return (np.arange(n) + 0.5) / n


def test_sod_tube():
    # 512 cells on [0, 1], gamma 1.4, (1, 0, 1) left of 0.5, (0.125, 0, 0.1)
    # right of it, outflow ends, CFL 0.4
    mesh, W = wl.sod(512)
    assert mesh.ndim == 1 and mesh.n == (512, 1, 1) and mesh.gamma == 1.4 and mesh.cfl == 0.4
    assert mesh.bc[0] == (wl.BC_OUTFLOW, wl.BC_OUTFLOW)
    left = _centres(512) < 0.5
    rho, v, p = W[0, 0, 0], W[1, 0, 0], W[2, 0, 0]
    assert np.all(rho[left] == 1.0) and np.all(rho[~left] == 0.125)
    assert np.all(p[left] == 1.0) and np.all(p[~left] == 0.1) and np.all(v == 0.0)
    assert left.sum() == 256


def test_kelvin_helmholtz_layer():
    # periodic unit square, gamma 5/3: rho 2 and vx +0.5 where |y - 0.5| <
    # 0.25, else rho 1 and vx -0.5; p 2.5; vy seeded uniform noise of
    # amplitude 0.01
    n = 256
    mesh, W = wl.kelvin_helmholtz(n, seed=1)
    assert mesh.ndim == 2 and mesh.n == (n, n, 1) and mesh.gamma == 5.0 / 3.0
    assert all(b == (wl.BC_PERIODIC, wl.BC_PERIODIC) for b in mesh.bc[:2])
    band = np.abs(_centres(n) - 0.5) < 0.25          # along y (axis 1 of the (ny, nx) plane)
    rho, vx, vy, p = W[0, 0], W[1, 0], W[2, 0], W[3, 0]
    assert np.all(rho[band, :] == 2.0) and np.all(rho[~band, :] == 1.0)
    assert np.all(vx[band, :] == 0.5) and np.all(vx[~band, :] == -0.5)
    assert np.all(p == 2.5)
    assert np.abs(vy).max() <= 0.01 and np.abs(vy).max() > 0.0099
    assert abs(vy.mean()) < 3 * 0.01 / math.sqrt(3 * n * n)   # uniform on [-0.01, 0.01]
    assert abs(vy.std() - 0.01 / math.sqrt(3.0)) < 0.01 * 0.02
    # seeded: the same seed gives the same noise, another seed another
    assert np.array_equal(wl.kelvin_helmholtz(n, seed=1)[1], W)
    assert not np.array_equal(wl.kelvin_helmholtz(n, seed=2)[1][2], vy[None])


def test_turbulence_box():
    # periodic cube, gamma 5/3, rho 1, p 0.6 (sound speed 1); velocity with
    # zero mean and rms |v| = 1 (rms Mach 1), its power only on integer
    # wavevectors 1 <= |k| <= 4
    n = 48
    mesh, W = wl.turbulence(n, seed=2)
    assert mesh.ndim == 3 and mesh.n == (n, n, n) and mesh.gamma == 5.0 / 3.0 and mesh.cfl == 0.3
    assert np.all(W[0] == 1.0) and np.all(W[4] == 0.6)
    assert math.sqrt(mesh.gamma * 0.6 / 1.0) == pytest.approx(1.0)
    v = W[1:4]
    assert np.abs(v.mean(axis=(1, 2, 3))).max() < 1e-12
    assert math.sqrt(float(np.mean((v * v).sum(axis=0)))) == pytest.approx(1.0, abs=1e-12)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kk = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + k1[None, None, :] ** 2)
    inside = (kk >= 1.0) & (kk <= 4.0)
    for d in range(3):
        P = np.abs(np.fft.fftn(v[d])) ** 2
        assert P[~inside].sum() <= 1e-20 * P.sum()
        # every component carries power (independent fields, none empty)
        assert P[inside].sum() > 0.1 * sum(np.mean(v[e] ** 2) for e in range(3)) * n ** 6 / 3.0
    # the shell spectrum falls with k: the power of the k in [3, 4] shell is
    # well below that of the k in [1, 2) shell (k^-4 by construction)
    P = sum(np.abs(np.fft.fftn(v[d])) ** 2 for d in range(3))
    lo = P[(kk >= 1.0) & (kk < 2.0)].sum()
    hi = P[(kk >= 3.0) & (kk <= 4.0)].sum()
    assert hi < 0.2 * lo


def test_batch_of_blasts():
    # 4096 square periodic 2D grids, sides log-uniform in [32, 256], each a
    # blast: rho 1, v 0, p 0.1 with p 10 within periodic distance 0.1 of a
    # seeded centre
    sides = wl.batch_sides(4096)
    assert sides.min() >= 32 and sides.max() <= 256
    ls = np.log(sides)
    assert abs(ls.mean() - 0.5 * (math.log(32) + math.log(256))) < 0.05
    # log-uniform: each third of [ln 32, ln 256] holds about a third of the grids
    edges = np.linspace(math.log(32), math.log(256), 4)
    counts = np.histogram(ls, bins=edges)[0]
    assert np.all(np.abs(counts / 4096.0 - 1.0 / 3.0) < 0.03)
    grids = wl.batch_blasts(64)                    # the first grids of the same stream
    assert [m.n[0] for m, _ in grids] == list(wl.batch_sides(64))
    for mesh, W in grids:
        assert mesh.ndim == 2 and mesh.n[0] == mesh.n[1] and mesh.gamma == 5.0 / 3.0
        assert np.all(W[0] == 1.0) and np.all(W[1:3] == 0.0)
        p = W[3, 0]
        assert set(np.unique(p)) <= {0.1, 10.0}
        frac = (p == 10.0).mean()
        assert 0.0 < frac <= math.pi * 0.1 ** 2 * 1.6       # a disc of radius 0.1


def test_serving_stream():
    # Poisson arrivals at 200 jobs/s; half 2D grids of sides 64-512, half 3D
    # grids of sides 32-128; initial conditions KH, blast or turbulence;
    # t_end uniform in [0.05, 0.5]
    jobs = wl.serving_stream(2000, seed=4)
    t = np.array([j.arrival for j in jobs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0.0)
    assert abs(gaps.mean() - 1.0 / 200.0) < 0.1 / 200.0
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1          # exponential gaps
    nd = np.array([j.ndim for j in jobs])
    assert set(nd) == {2, 3} and abs((nd == 2).mean() - 0.5) < 0.05
    for j in jobs:
        lo, hi = (64, 512) if j.ndim == 2 else (32, 128)
        assert lo <= j.side <= hi
        assert 0.05 <= j.t_end <= 0.5
        assert j.kind in ("kh", "blast", "turb")
    assert {j.kind for j in jobs} == {"kh", "blast", "turb"}
    assert [j.arrival for j in wl.serving_stream(2000, seed=4)] == list(t)   # seeded
