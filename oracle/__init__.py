"""CPU oracle for the Godunov hydro step (test infrastructure only).

Plain FP64 C (``khydro_oracle.c``) behind ctypes, plus the exact Riemann
solver (``exact_riemann.py``).  Only the tests, the package smoke check and
the benchmark's CPU-baseline leg use this package; the CUDA library never
does, and this package never imports the CUDA library.

Arrays are float64 with shape ``(nvar, nz, ny, nx)`` as produced by
``paper_2501_02317_gb300.workloads``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "khydro_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")

FLAG_NONPHYSICAL = 1
FLAG_FLOOR = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no FMA contraction, no fast-math."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _OrcMesh(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double),
        ("bc", (ctypes.c_int * 2) * 3),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER
        d, vp = ctypes.c_double, ctypes.c_void_p
        L.orc_prim_to_cons.argtypes = [P(_OrcMesh), vp, vp]
        L.orc_cons_to_prim.argtypes = [P(_OrcMesh), vp, vp, P(ctypes.c_uint)]
        L.orc_cfl_dt.argtypes = [P(_OrcMesh), vp, P(ctypes.c_uint)]
        L.orc_cfl_dt.restype = d
        L.orc_minmod.argtypes = [d, d]
        L.orc_minmod.restype = d
        L.orc_hllc.argtypes = [d, vp, vp, vp]
        L.orc_rhs.argtypes = [P(_OrcMesh), vp, d, vp, P(ctypes.c_uint)]
        L.orc_heun_step.argtypes = [P(_OrcMesh), vp, P(d), d, P(ctypes.c_uint)]
        L.orc_heun_step.restype = d
        L.orc_run.argtypes = [P(_OrcMesh), vp, P(d), d, ctypes.c_long, P(ctypes.c_uint)]
        L.orc_run.restype = ctypes.c_long
        L.orc_vl2_step.argtypes = [P(_OrcMesh), vp, P(d), d, P(ctypes.c_uint)]
        L.orc_vl2_step.restype = d
        L.orc_run_with.argtypes = [P(_OrcMesh), vp, P(d), d, ctypes.c_long, ctypes.c_int, P(ctypes.c_uint)]
        L.orc_run_with.restype = ctypes.c_long
        L.orc_totals.argtypes = [P(_OrcMesh), vp, vp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_set_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _mesh(m) -> _OrcMesh:
    o = _OrcMesh()
    o.ndim = m.ndim
    for d in range(3):
        o.n[d] = int(m.n[d])
        o.lo[d] = float(m.lo[d])
        o.hi[d] = float(m.hi[d])
        o.bc[d][0] = int(m.bc[d][0])
        o.bc[d][1] = int(m.bc[d][1])
    o.gamma = float(m.gamma)
    o.cfl = float(m.cfl)
    o.rho_floor = float(m.rho_floor)
    o.p_floor = float(m.p_floor)
    return o


def _arr(a: np.ndarray, shape) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == tuple(shape), (a.shape, shape)
    return a


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> int:
    return lib().orc_set_threads(int(n))


def prim_to_cons(mesh, W: np.ndarray) -> np.ndarray:
    W = _arr(W, mesh.shape)
    U = np.empty_like(W)
    lib().orc_prim_to_cons(ctypes.byref(_mesh(mesh)), _p(W), _p(U))
    return U


def cons_to_prim(mesh, U: np.ndarray) -> Tuple[np.ndarray, int]:
    U = _arr(U, mesh.shape)
    W = np.empty_like(U)
    f = ctypes.c_uint(0)
    lib().orc_cons_to_prim(ctypes.byref(_mesh(mesh)), _p(U), _p(W), ctypes.byref(f))
    return W, f.value


def cfl_dt(mesh, U: np.ndarray) -> float:
    U = _arr(U, mesh.shape)
    f = ctypes.c_uint(0)
    return lib().orc_cfl_dt(ctypes.byref(_mesh(mesh)), _p(U), ctypes.byref(f))


def minmod(a: float, b: float) -> float:
    return lib().orc_minmod(float(a), float(b))


def hllc(gamma: float, wl, wr) -> np.ndarray:
    """HLLC flux for rotated primitive states (rho, u_n, u_t1, u_t2, p)."""
    a = np.ascontiguousarray(wl, dtype=np.float64)
    b = np.ascontiguousarray(wr, dtype=np.float64)
    assert a.shape == (5,) and b.shape == (5,)
    F = np.zeros(5)
    lib().orc_hllc(float(gamma), _p(a), _p(b), _p(F))
    return F


def rhs(mesh, U: np.ndarray, dt: float) -> Tuple[np.ndarray, int]:
    U = _arr(U, mesh.shape)
    dU = np.empty_like(U)
    f = ctypes.c_uint(0)
    lib().orc_rhs(ctypes.byref(_mesh(mesh)), _p(U), float(dt), _p(dU), ctypes.byref(f))
    return dU, f.value


def heun_step(mesh, U: np.ndarray, t: float, t_end: float):
    """One Heun step in place on a copy; returns (U_new, t_new, dt, flags)."""
    U = _arr(U, mesh.shape).copy()
    tt = ctypes.c_double(t)
    f = ctypes.c_uint(0)
    dt = lib().orc_heun_step(ctypes.byref(_mesh(mesh)), _p(U), ctypes.byref(tt), float(t_end), ctypes.byref(f))
    return U, tt.value, dt, f.value


def vl2_step(mesh, U: np.ndarray, t: float, t_end: float):
    """One memory-optimized van Leer step on a copy; returns (U_new, t_new, dt, flags)."""
    U = _arr(U, mesh.shape).copy()
    tt = ctypes.c_double(t)
    f = ctypes.c_uint(0)
    dt = lib().orc_vl2_step(ctypes.byref(_mesh(mesh)), _p(U), ctypes.byref(tt), float(t_end), ctypes.byref(f))
    return U, tt.value, dt, f.value


def run(mesh, U: np.ndarray, t: float, t_end: float, max_steps: int = 1 << 40, integrator=None):
    """Steps from t to t_end (or max_steps) with the mesh's integrator (0 Heun,
    1 van Leer) unless one is given; returns (U, t, steps, flags)."""
    if integrator is None:
        integrator = getattr(mesh, "integrator", 0)
    U = _arr(U, mesh.shape).copy()
    tt = ctypes.c_double(t)
    f = ctypes.c_uint(0)
    s = lib().orc_run_with(ctypes.byref(_mesh(mesh)), _p(U), ctypes.byref(tt), float(t_end), int(max_steps),
                           int(integrator), ctypes.byref(f))
    return U, tt.value, s, f.value


def totals(mesh, U: np.ndarray) -> np.ndarray:
    U = _arr(U, mesh.shape)
    out = np.zeros(5)
    lib().orc_totals(ctypes.byref(_mesh(mesh)), _p(U), _p(out))
    return out[: mesh.nvar]


def pressure(mesh, U: np.ndarray) -> np.ndarray:
    W, _ = cons_to_prim(mesh, U)
    return W[mesh.nvar - 1]
