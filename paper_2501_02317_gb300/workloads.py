"""Seeded synthetic inputs: mesh descriptors and primitive initial states.

This module only draws random numbers and lays out initial primitive fields
(density, velocity, pressure).  It holds none of the finite-volume method's
arithmetic (no conserved-variable conversion, no fluxes), so the CUDA library
and the CPU oracle can both start from exactly the same FP64 arrays.

Every generator returns ``(mesh, W)`` where ``W`` is a float64 array of shape
``(2 + ndim, nz, ny, nx)`` (x fastest) holding ``(rho, v_1..v_ndim, p)`` on the
interior cells, and ``mesh`` is a :class:`Mesh`.

Workloads (the paper's own test problems need inputs it does not print, so
these seeded problems of the same kind stand in for them):
  * Sod shock tube, 1D (Sec. 4.2), also rotated onto y or z (axis interchange)
  * linear sound wave, 1D periodic (Sec. 4.1, Eq. 6 setup)
  * Kelvin-Helmholtz shear layer, 2D periodic (sharp layer, seeded noise)
  * random-phase turbulence box, 3D periodic, shell spectrum ~ k^-4, rms Mach 1
  * blast wave, 2D periodic (batched small grids)
  * Liska-Wendroff implosion, 2D reflecting (Sec. 4.4, Eq. 7)
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

BC_PERIODIC = 0
BC_OUTFLOW = 1
BC_FREE = 2
BC_REFLECT = 3

PREC_FP64 = 0
PREC_MIXED = 1
PREC_FP32 = 2

# time integrators (Sec. 3.3): Heun, memory-optimized van Leer, and Heun
# without stored primitives (the same step, less device memory)
INT_HEUN = 0
INT_VL2 = 1
INT_HEUN_LEAN = 2

DEFAULT_FLOOR = 1e-10


@dataclasses.dataclass
class Mesh:
    """Uniform Cartesian mesh descriptor (mirrors ``khy_mesh_desc``)."""

    ndim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    hi: Tuple[float, float, float] = (1.0, 1.0, 1.0)
    gamma: float = 1.4
    cfl: float = 0.4
    bc: Tuple[Tuple[int, int], Tuple[int, int], Tuple[int, int]] = (
        (BC_PERIODIC, BC_PERIODIC),
        (BC_PERIODIC, BC_PERIODIC),
        (BC_PERIODIC, BC_PERIODIC),
    )
    prec: int = PREC_FP64
    rho_floor: float = DEFAULT_FLOOR
    p_floor: float = DEFAULT_FLOOR
    integrator: int = INT_HEUN

    @property
    def nvar(self) -> int:
        return 2 + self.ndim

    @property
    def ncell(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    @property
    def shape(self) -> Tuple[int, int, int, int]:
        return (self.nvar, self.n[2], self.n[1], self.n[0])

    def replace(self, **kw) -> "Mesh":
        return dataclasses.replace(self, **kw)


def _centres(mesh: Mesh, d: int) -> np.ndarray:
    n = mesh.n[d]
    lo, hi = mesh.lo[d], mesh.hi[d]
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * ((hi - lo) / n)


def _grids(mesh: Mesh):
    """Cell-centre coordinates broadcast to (nz, ny, nx)."""
    x = _centres(mesh, 0)[None, None, :]
    y = _centres(mesh, 1)[None, :, None]
    z = _centres(mesh, 2)[:, None, None]
    return x, y, z


def _empty(mesh: Mesh) -> np.ndarray:
    return np.zeros(mesh.shape, dtype=np.float64)


def _all_bc(b: int):
    return ((b, b), (b, b), (b, b))


# --------------------------------------------------------------- Sec. 4.2 Sod


def sod(n: int = 512, axis: int = 0, ndim: int = 1, ntrans: int = 4, prec: int = PREC_FP64,
        gamma: float = 1.4, cfl: float = 0.4) -> Tuple[Mesh, np.ndarray]:
    """Sod tube along ``axis``: (rho, v, p) = (1, 0, 1) left of 0.5, else
    (0.125, 0, 0.1); outflow on the tube axis, periodic across it.
    ``ntrans`` cells on the transverse axes when ndim > axis-only."""
    assert 0 <= axis < ndim <= 3
    nn = [1, 1, 1]
    for d in range(ndim):
        nn[d] = n if d == axis else ntrans
    bc = [[BC_PERIODIC, BC_PERIODIC] for _ in range(3)]
    bc[axis] = [BC_OUTFLOW, BC_OUTFLOW]
    mesh = Mesh(ndim=ndim, n=tuple(nn), gamma=gamma, cfl=cfl,
                bc=tuple(tuple(b) for b in bc), prec=prec)
    W = _empty(mesh)
    c = _grids(mesh)[axis]
    left = np.broadcast_to(c < 0.5, mesh.shape[1:])
    W[0] = np.where(left, 1.0, 0.125)
    W[mesh.nvar - 1] = np.where(left, 1.0, 0.1)
    return mesh, W


def shock_tube(n: int, left: Sequence[float], right: Sequence[float], x0: float = 0.5, gamma: float = 1.4,
               prec: int = PREC_FP64, cfl: float = 0.4, bc: int = BC_FREE) -> Tuple[Mesh, np.ndarray]:
    """1D Riemann problem on [0, 1] (Sec. 4.2): primitive states (rho, v, p)
    left and right of x0.  Zero-gradient ("free") ends by default: the
    outflow rule of Sec. 3.1.1 refuses inflow, which would launch a wave from
    an end where the state moves into the tube."""
    mesh = Mesh(ndim=1, n=(n, 1, 1), gamma=gamma, cfl=cfl,
                bc=((bc, bc), (BC_PERIODIC, BC_PERIODIC), (BC_PERIODIC, BC_PERIODIC)), prec=prec)
    W = _empty(mesh)
    lft = _grids(mesh)[0] < x0
    for q in range(3):
        W[q] = np.broadcast_to(np.where(lft, left[q], right[q]), mesh.shape[1:])
    return mesh, W


# ------------------------------------------------ Sec. 4.1 linear sound wave


def sound_wave(n: int, amp: float = 1e-6, p0: float = 5.0 / 3.0, rho0: float = 1.0,
               gamma: float = 5.0 / 3.0, cfl: float = 0.4, prec: int = PREC_FP64,
               ndim: int = 1, axis: int = 0, ntrans: int = 4) -> Tuple[Mesh, np.ndarray]:
    """Right-moving linearised sound wave on a periodic unit box:
    drho = A sin(2 pi x), dv = (c_s/rho0) drho, dp = c_s^2 drho."""
    nn = [1, 1, 1]
    for d in range(ndim):
        nn[d] = n if d == axis else ntrans
    mesh = Mesh(ndim=ndim, n=tuple(nn), gamma=gamma, cfl=cfl, bc=_all_bc(BC_PERIODIC), prec=prec)
    cs = math.sqrt(gamma * p0 / rho0)
    c = _grids(mesh)[axis]
    drho = np.broadcast_to(amp * np.sin(2.0 * np.pi * c), mesh.shape[1:])
    W = _empty(mesh)
    W[0] = rho0 + drho
    W[1 + axis] = (cs / rho0) * drho
    W[mesh.nvar - 1] = p0 + cs * cs * drho
    return mesh, W


def advection_wave(n: int, kind: str = "contact", profile: str = "sine", amp: float = 0.1,
                   v: float = 1.0, rho0: float = 1.0, p0: float = 5.0 / 3.0, gamma: float = 5.0 / 3.0,
                   cfl: float = 0.4, prec: int = PREC_FP64) -> Tuple[Mesh, np.ndarray]:
    """Sec. 4.1 wave tests on a periodic unit box, background (rho0, p0) moving
    with v along x: a contact wave (drho) or a shear wave (dv_y; a 2D grid n x 2),
    the perturbation A sin(2 pi x) ("sine") or A where x < 0.5 ("tophat")."""
    if kind not in ("contact", "shear") or profile not in ("sine", "tophat"):
        raise ValueError("kind is contact or shear, profile is sine or tophat")
    ndim = 1 if kind == "contact" else 2
    mesh = Mesh(ndim=ndim, n=(n, 1 if ndim == 1 else 2, 1), gamma=gamma, cfl=cfl,
                bc=_all_bc(BC_PERIODIC), prec=prec)
    x = _grids(mesh)[0]
    d = amp * np.sin(2.0 * np.pi * x) if profile == "sine" else np.where(x < 0.5, amp, 0.0)
    d = np.broadcast_to(d, mesh.shape[1:])
    W = _empty(mesh)
    W[0] = rho0 + d if kind == "contact" else rho0
    W[1] = v
    if kind == "shear":
        W[2] = d
    W[mesh.nvar - 1] = p0
    return mesh, W


def sound_speed(p0: float, rho0: float, gamma: float) -> float:
    return math.sqrt(gamma * p0 / rho0)


# ------------------------------------------------------ 2D Kelvin-Helmholtz


def kelvin_helmholtz(n: int = 1024, seed: int = 1, prec: int = PREC_MIXED, cfl: float = 0.4,
                     ny: int | None = None) -> Tuple[Mesh, np.ndarray]:
    """Sharp shear layer on the periodic unit square, gamma = 5/3:
    rho = 2, vx = +0.5 for |y - 0.5| < 0.25, else rho = 1, vx = -0.5;
    p = 2.5; vy = 0.01 (2u - 1), u ~ U[0,1) per cell (seeded)."""
    ny = n if ny is None else ny
    mesh = Mesh(ndim=2, n=(n, ny, 1), gamma=5.0 / 3.0, cfl=cfl, bc=_all_bc(BC_PERIODIC), prec=prec)
    rng = np.random.default_rng(seed)
    _, y, _ = _grids(mesh)
    band = np.broadcast_to(np.abs(y - 0.5) < 0.25, mesh.shape[1:])
    W = _empty(mesh)
    W[0] = np.where(band, 2.0, 1.0)
    W[1] = np.where(band, 0.5, -0.5)
    W[2] = 0.01 * (2.0 * rng.random(mesh.shape[1:]) - 1.0)
    W[3] = 2.5
    return mesh, W


# -------------------------------------------------------- 3D turbulence box


def turbulence(n: int = 256, seed: int = 2, prec: int = PREC_MIXED, cfl: float = 0.3,
               kmin: float = 1.0, kmax: float = 4.0, mach: float = 1.0) -> Tuple[Mesh, np.ndarray]:
    """Periodic unit cube, gamma = 5/3, rho = 1, p = 0.6 (c_s = 1).  Each
    velocity component is an independent Gaussian random field with random
    phases over integer wavevectors kmin <= |k| <= kmax (units 2 pi / L),
    mode power ~ k^-4 / (4 pi k^2) so the shell spectrum goes as k^-4; mean
    removed; scaled to rms |v| = mach (no solenoidal projection)."""
    mesh = Mesh(ndim=3, n=(n, n, n), gamma=5.0 / 3.0, cfl=cfl, bc=_all_bc(BC_PERIODIC), prec=prec)
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz = k1[:, None, None]
    ky = k1[None, :, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    shell = (kk >= kmin) & (kk <= kmax)
    amp = np.zeros_like(kk)
    amp[shell] = np.sqrt(kk[shell] ** -4.0 / (4.0 * np.pi * kk[shell] ** 2))
    W = _empty(mesh)
    W[0] = 1.0
    W[4] = 0.6
    vel = []
    for _ in range(3):
        coef = amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape))
        v = np.fft.irfftn(coef, s=(n, n, n), axes=(0, 1, 2))
        v -= v.mean()
        vel.append(v)
    rms = math.sqrt(float(np.mean(vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)))
    for d in range(3):
        W[1 + d] = vel[d] * (mach / rms)
    return mesh, W


# ------------------------------------------------------------ 2D blast wave


def blast(n: int, centre: Sequence[float], prec: int = PREC_MIXED, cfl: float = 0.4,
          radius: float = 0.1, p_in: float = 10.0, p_out: float = 0.1,
          ndim: int = 2) -> Tuple[Mesh, np.ndarray]:
    """rho = 1, v = 0, p = p_out except p = p_in within periodic distance
    ``radius`` of ``centre``; periodic unit box, gamma = 5/3."""
    nn = [n if d < ndim else 1 for d in range(3)]
    mesh = Mesh(ndim=ndim, n=tuple(nn), gamma=5.0 / 3.0, cfl=cfl, bc=_all_bc(BC_PERIODIC), prec=prec)
    g = _grids(mesh)
    r2 = 0.0
    for d in range(ndim):
        dd = np.abs(g[d] - centre[d])
        dd = np.minimum(dd, 1.0 - dd)
        r2 = r2 + dd * dd
    inside = np.broadcast_to(r2 < radius * radius, mesh.shape[1:])
    W = _empty(mesh)
    W[0] = 1.0
    W[mesh.nvar - 1] = np.where(inside, p_in, p_out)
    return mesh, W


def batch_blasts(ngrids: int = 4096, seed: int = 3, lo: int = 32, hi: int = 256,
                 prec: int = PREC_MIXED) -> List[Tuple[Mesh, np.ndarray]]:
    """Independent square 2D blast grids with sides round(exp(U[ln lo, ln hi]))
    and centres ~ U[0,1)^2, all from one seeded stream."""
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=ngrids))).astype(int)
    centres = rng.random((ngrids, 2))
    return [blast(int(s), c, prec=prec) for s, c in zip(sides, centres)]


def batch_sides(ngrids: int = 4096, seed: int = 3, lo: int = 32, hi: int = 256) -> np.ndarray:
    """Only the side lengths of :func:`batch_blasts` (same stream)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=ngrids))).astype(int)


# ------------------------------------------ Sec. 4.4 Liska-Wendroff implosion


def liska_wendroff(n: int = 400, size: float = 0.3, prec: int = PREC_FP64,
                   cfl: float = 0.4) -> Tuple[Mesh, np.ndarray]:
    """Eq. 7: (rho, p, v) = (0.125, 0.14, 0) where x + y < 0.15, else (1, 1, 0);
    gamma = 1.4; reflecting on all sides.  The paper does not state the domain;
    a square [0, size]^2 is used."""
    mesh = Mesh(ndim=2, n=(n, n, 1), hi=(size, size, 1.0), gamma=1.4, cfl=cfl,
                bc=_all_bc(BC_REFLECT), prec=prec)
    x, y, _ = _grids(mesh)
    inner = np.broadcast_to(x + y < 0.15, mesh.shape[1:])
    W = _empty(mesh)
    W[0] = np.where(inner, 0.125, 1.0)
    W[3] = np.where(inner, 0.14, 1.0)
    return mesh, W


# ---------------------------------------------------------- uniform state


def cold_fast_state(ndim: int, n: Tuple[int, int, int], seed: int = 13,
                    prec: int = PREC_MIXED) -> Tuple[Mesh, np.ndarray]:
    """Fast, cold gas: rho in [0.5, 2], velocity components in [5, 10] with
    random signs, pressure 1e-4 x [0.2, 2] (gamma 1.4): the kinetic energy is
    ~2e5 times the internal energy; with a pressure floor of 1e-4 about half
    of the cells are floored.  A stress state for the conserved-to-primitive
    recovery (Sec. 3.1)."""
    mesh = Mesh(ndim=ndim, n=tuple(n), gamma=1.4, cfl=0.4 if ndim < 3 else 0.3, prec=prec,
                bc=_all_bc(BC_PERIODIC), p_floor=1e-4)
    rng = np.random.default_rng(seed)
    W = _empty(mesh)
    sh = mesh.shape[1:]
    W[0] = rng.uniform(0.5, 2.0, size=sh)
    for d in range(ndim):
        W[1 + d] = rng.uniform(5.0, 10.0, size=sh) * rng.choice([-1.0, 1.0], size=sh)
    W[mesh.nvar - 1] = 1e-4 * rng.uniform(0.2, 2.0, size=sh)
    return mesh, W


def uniform(mesh: Mesh, rho: float = 1.0, v: Sequence[float] = (0.3, -0.2, 0.1), p: float = 0.7) -> np.ndarray:
    W = _empty(mesh)
    W[0] = rho
    for d in range(mesh.ndim):
        W[1 + d] = v[d]
    W[mesh.nvar - 1] = p
    return W


def random_smooth(mesh: Mesh, seed: int = 7, amp: float = 0.2) -> np.ndarray:
    """Smooth positive random state (a few low Fourier modes per field), used
    for parity cases that must exercise every flux branch."""
    rng = np.random.default_rng(seed)
    g = _grids(mesh)
    W = _empty(mesh)
    for q in range(mesh.nvar):
        f = np.zeros(mesh.shape[1:])
        for _ in range(3):
            phase = rng.random(3) * 2 * np.pi
            kv = rng.integers(1, 3, size=3)
            term = 1.0
            for d in range(mesh.ndim):
                term = term * np.cos(2 * np.pi * kv[d] * g[d] + phase[d])
            f = f + term
        W[q] = f
    W[0] = 1.0 + amp * W[0]
    for d in range(mesh.ndim):
        W[1 + d] = 0.8 * W[1 + d]
    W[mesh.nvar - 1] = 1.0 + amp * W[mesh.nvar - 1]
    return W


def random_jumpy(mesh: Mesh, seed: int = 11) -> np.ndarray:
    """Piecewise-random positive state with jumps in every field: exercises
    supersonic, subsonic and both star-state flux branches and the limiter."""
    rng = np.random.default_rng(seed)
    W = _empty(mesh)
    s = mesh.shape[1:]
    W[0] = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=s))
    for d in range(mesh.ndim):
        W[1 + d] = rng.uniform(-1.0, 1.0, size=s)
    W[mesh.nvar - 1] = np.exp(rng.uniform(np.log(0.3), np.log(3.0), size=s))
    return W


# ------------------------------------------------------ serving arrivals


@dataclasses.dataclass
class Job:
    arrival: float
    kind: str          # "kh" | "blast" | "turb"
    ndim: int
    side: int
    t_end: float
    seed: int


def serving_stream(njobs: int = 2000, rate: float = 200.0, seed: int = 4,
                   side2d: Tuple[int, int] = (64, 512), side3d: Tuple[int, int] = (32, 128),
                   t_end: Tuple[float, float] = (0.05, 0.5)) -> List[Job]:
    """Poisson arrivals (mean ``rate`` per second); half 2D, half 3D grids with
    log-uniform sides; initial condition drawn from {kh, blast, turb};
    t_end ~ U[t_end]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for i in range(njobs):
        t += float(rng.exponential(1.0 / rate))
        ndim = 2 if rng.random() < 0.5 else 3
        lo, hi = side2d if ndim == 2 else side3d
        side = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        kind = ["kh", "blast", "turb"][int(rng.integers(0, 3))]
        te = float(rng.uniform(*t_end))
        jobs.append(Job(arrival=t, kind=kind, ndim=ndim, side=side, t_end=te, seed=int(rng.integers(0, 2**31))))
    return jobs


def job_initial_state(job: Job, prec: int = PREC_MIXED) -> Tuple[Mesh, np.ndarray]:
    """Initial state of a serving job: the job's kind at the job's size."""
    if job.kind == "blast":
        rng = np.random.default_rng(job.seed)
        return blast(job.side, rng.random(3), prec=prec, ndim=job.ndim, cfl=0.4 if job.ndim == 2 else 0.3)
    if job.kind == "kh":
        if job.ndim == 2:
            return kelvin_helmholtz(job.side, seed=job.seed, prec=prec)
        # 3D shear layer: the 2D layer extruded along z with 3D noise
        mesh = Mesh(ndim=3, n=(job.side,) * 3, gamma=5.0 / 3.0, cfl=0.3, bc=_all_bc(BC_PERIODIC), prec=prec)
        rng = np.random.default_rng(job.seed)
        _, y, _ = _grids(mesh)
        band = np.broadcast_to(np.abs(y - 0.5) < 0.25, mesh.shape[1:])
        W = _empty(mesh)
        W[0] = np.where(band, 2.0, 1.0)
        W[1] = np.where(band, 0.5, -0.5)
        W[2] = 0.01 * (2.0 * rng.random(mesh.shape[1:]) - 1.0)
        W[4] = 2.5
        return mesh, W
    # turbulence
    if job.ndim == 3:
        return turbulence(job.side, seed=job.seed, prec=prec)
    mesh = Mesh(ndim=2, n=(job.side, job.side, 1), gamma=5.0 / 3.0, cfl=0.4, bc=_all_bc(BC_PERIODIC), prec=prec)
    rng = np.random.default_rng(job.seed)
    n = job.side
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    ky = k1[:, None]
    kx = np.fft.rfftfreq(n, d=1.0 / n)[None, :]
    kk = np.sqrt(kx * kx + ky * ky)
    shell = (kk >= 1) & (kk <= 4)
    amp = np.zeros_like(kk)
    amp[shell] = np.sqrt(kk[shell] ** -4.0 / (2.0 * np.pi * kk[shell]))
    W = _empty(mesh)
    W[0] = 1.0
    W[3] = 0.6
    vs = []
    for _ in range(2):
        coef = amp * (rng.standard_normal(kk.shape) + 1j * rng.standard_normal(kk.shape))
        v = np.fft.irfftn(coef, s=(n, n), axes=(0, 1))
        vs.append(v - v.mean())
    rms = math.sqrt(float(np.mean(vs[0] ** 2 + vs[1] ** 2)))
    W[1, 0] = vs[0] / rms
    W[2, 0] = vs[1] / rms
    return mesh, W
