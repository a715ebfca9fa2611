"""Thin ctypes binding of libkhydro.so (include/khydro.h).

Argument marshalling only: every step of the method runs in the CUDA
library.  The module-level functions carry the C names (``khy_create``,
``khy_step_to`` ...); :class:`Sim` is a small convenience wrapper over them.
Host arrays are numpy float64; device arrays may be torch CUDA tensors (their
``data_ptr()`` is passed to the ``*_dev`` calls).

Loading fails loudly if the library has not been built: there is no CPU or
Python fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

from .workloads import Mesh

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkhydro.so")

KHY_OK = 0
STATUS_NAMES = {0: "KHY_OK", -1: "KHY_ERR_ARG", -2: "KHY_ERR_OOM", -3: "KHY_ERR_CUDA",
                -4: "KHY_ERR_NONPHYSICAL", -5: "KHY_ERR_DT_UNDERFLOW", -6: "KHY_ERR_TIMEOUT",
                -7: "KHY_ERR_BUDGET"}

# capacity of khy_step_noalloc's fixed scratch state (KHY_NOALLOC_SCRATCH_BYTES
# of include/khydro.h; a CPU test checks that the two agree)
KHY_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024

# public symbols of include/khydro.h (checked by the CPU tests)
EXPORTS = [
    "khy_create", "khy_destroy", "khy_set_boundary", "khy_set_conserved", "khy_set_primitive",
    "khy_set_conserved_dev", "khy_set_primitive_dev", "khy_set_time", "khy_step_to",
    "khy_enqueue_steps", "khy_get_conserved", "khy_get_conserved_dev", "khy_get_time", "khy_totals",
    "khy_get_flags", "khy_last_error", "khy_version", "khy_profile_steps", "khy_step_noalloc",
    "khy_get_primitive",
    "khy_device_bytes",
    "khy_batch_create", "khy_batch_destroy", "khy_batch_set_primitive", "khy_batch_set_conserved",
    "khy_batch_get_conserved", "khy_batch_set_target", "khy_batch_enqueue_steps", "khy_batch_run",
    "khy_batch_get_clock", "khy_batch_autotune", "khy_batch_set_variant", "khy_batch_profile_steps",
    "khy_batch_set_schedule", "khy_batch_get_schedule",
    "khy_batch_info", "khy_server_create", "khy_server_destroy", "khy_server_submit", "khy_server_poll",
    "khy_server_wait", "khy_server_result", "khy_server_stats",
]


class KhydroError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class khy_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("hi", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("prec", ctypes.c_int),
        ("bc", (ctypes.c_int * 2) * 3),
        ("integrator", ctypes.c_int),
        ("rho_floor", ctypes.c_double),
        ("p_floor", ctypes.c_double),
    ]


def desc_of(mesh: Mesh) -> khy_mesh_desc:
    d = khy_mesh_desc()
    d.ndim = int(mesh.ndim)
    for a in range(3):
        d.n[a] = int(mesh.n[a])
        d.lo[a] = float(mesh.lo[a])
        d.hi[a] = float(mesh.hi[a])
        d.bc[a][0] = int(mesh.bc[a][0])
        d.bc[a][1] = int(mesh.bc[a][1])
    d.gamma = float(mesh.gamma)
    d.cfl = float(mesh.cfl)
    d.prec = int(mesh.prec)
    d.integrator = int(getattr(mesh, "integrator", 0))
    d.rho_floor = float(mesh.rho_floor)
    d.p_floor = float(mesh.p_floor)
    return d


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libkhydro.so; raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libkhydro.so is not built (run __graft_entry__.build() or "
                          "python -m paper_2501_02317_gb300.build); there is no fallback")
    L = ctypes.CDLL(LIB_PATH)
    P, vp, st = ctypes.POINTER, ctypes.c_void_p, ctypes.c_size_t
    i, d, l = ctypes.c_int, ctypes.c_double, ctypes.c_long
    sig = {
        "khy_create": [P(khy_mesh_desc), vp, P(vp)],
        "khy_set_boundary": [vp, i, i, i],
        "khy_set_conserved": [vp, vp, st],
        "khy_set_primitive": [vp, vp, st],
        "khy_set_conserved_dev": [vp, vp, st],
        "khy_set_primitive_dev": [vp, vp, st],
        "khy_set_time": [vp, d],
        "khy_step_to": [vp, d, l, P(l), P(d)],
        "khy_enqueue_steps": [vp, d, l],
        "khy_get_conserved": [vp, vp, st],
        "khy_get_conserved_dev": [vp, vp, st],
        "khy_get_primitive": [vp, vp, st],
        "khy_get_time": [vp, P(d), P(l), P(d)],
        "khy_totals": [vp, vp],
        "khy_get_flags": [vp, P(ctypes.c_uint), P(ctypes.c_ulonglong), i],
        "khy_profile_steps": [vp, d, l, P(ctypes.c_float)],
        "khy_device_bytes": [vp, P(st), P(st)],
        "khy_step_noalloc": [P(khy_mesh_desc), vp, d, d, vp, vp],
        "khy_batch_create": [P(khy_mesh_desc), i, vp, P(vp)],
        "khy_batch_set_primitive": [vp, vp, st],
        "khy_batch_set_conserved": [vp, vp, st],
        "khy_batch_get_conserved": [vp, vp, st],
        "khy_batch_set_target": [vp, i, d, l],
        "khy_batch_enqueue_steps": [vp, l],
        "khy_batch_run": [vp, P(l)],
        "khy_batch_get_clock": [vp, i, P(d), P(l), P(d)],
        "khy_batch_autotune": [vp, i, P(i), P(ctypes.c_float)],
        "khy_batch_set_variant": [vp, i],
        "khy_batch_set_schedule": [vp, i, i],
        "khy_batch_get_schedule": [vp, P(i), P(i)],
        "khy_batch_profile_steps": [vp, l, P(ctypes.c_float)],
        "khy_batch_info": [vp, P(ctypes.c_longlong), P(st), P(i), P(i)],
        "khy_server_create": [st, i, vp, P(vp)],
        "khy_server_submit": [vp, P(khy_mesh_desc), vp, st, d, P(l)],
        "khy_server_poll": [vp, l, P(i), P(d), P(l)],
        "khy_server_wait": [vp, l, d],
        "khy_server_result": [vp, l, vp, st, i],
        "khy_server_stats": [vp, P(l), P(i), P(i), P(ctypes.c_ulonglong), P(d)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.khy_destroy.argtypes = [vp]
    L.khy_destroy.restype = None
    L.khy_batch_destroy.argtypes = [vp]
    L.khy_batch_destroy.restype = None
    L.khy_server_destroy.argtypes = [vp]
    L.khy_server_destroy.restype = None
    L.khy_last_error.argtypes = []
    L.khy_last_error.restype = ctypes.c_char_p
    L.khy_version.argtypes = []
    L.khy_version.restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int) -> None:
    if status != KHY_OK:
        raise KhydroError(status, lib().khy_last_error().decode(errors="replace"))


def _host(a: np.ndarray) -> Tuple[np.ndarray, ctypes.c_void_p]:
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise TypeError("host arrays must be C-contiguous float64 numpy arrays")
    return a, ctypes.c_void_p(a.ctypes.data)


def _is_device_tensor(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _dev_ptr(t) -> ctypes.c_void_p:
    import torch
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("device tensors must be contiguous float64")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------ C-named calls

def khy_version() -> int:
    return lib().khy_version()


def khy_create(mesh: Mesh, stream: Optional[int] = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    desc = desc_of(mesh)
    _check(lib().khy_create(ctypes.byref(desc), ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def khy_destroy(h) -> None:
    lib().khy_destroy(h)


def khy_set_boundary(h, axis: int, side: int, bc: int) -> None:
    _check(lib().khy_set_boundary(h, axis, side, bc))


def khy_set_primitive(h, W) -> None:
    if _is_device_tensor(W):
        _check(lib().khy_set_primitive_dev(h, _dev_ptr(W), W.numel()))
    else:
        W, p = _host(W)
        _check(lib().khy_set_primitive(h, p, W.size))


def khy_set_conserved(h, U) -> None:
    if _is_device_tensor(U):
        _check(lib().khy_set_conserved_dev(h, _dev_ptr(U), U.numel()))
    else:
        U, p = _host(U)
        _check(lib().khy_set_conserved(h, p, U.size))


def khy_set_time(h, t: float) -> None:
    _check(lib().khy_set_time(h, float(t)))


def khy_step_to(h, t_end: float, max_steps: int = -1) -> Tuple[int, float]:
    s = ctypes.c_long(0)
    t = ctypes.c_double(0.0)
    _check(lib().khy_step_to(h, float(t_end), int(max_steps), ctypes.byref(s), ctypes.byref(t)))
    return s.value, t.value


def khy_enqueue_steps(h, t_end: float, nsteps: int) -> None:
    _check(lib().khy_enqueue_steps(h, float(t_end), int(nsteps)))


def khy_get_conserved(h, out) -> None:
    if _is_device_tensor(out):
        _check(lib().khy_get_conserved_dev(h, _dev_ptr(out), out.numel()))
    else:
        out, p = _host(out)
        _check(lib().khy_get_conserved(h, p, out.size))


def khy_get_primitive(h, out) -> None:
    out, p = _host(out)
    _check(lib().khy_get_primitive(h, p, out.size))


def khy_profile_steps(h, t_end: float, nsteps: int) -> Tuple[float, float, float]:
    ms = (ctypes.c_float * 3)()
    _check(lib().khy_profile_steps(h, float(t_end), int(nsteps), ms))
    return ms[0], ms[1], ms[2]


def khy_step_noalloc(mesh: Mesh, U_dev_ptr: int, t: float, t_end: float, out_dev_ptr: int,
                     stream: Optional[int] = None) -> None:
    """One allocation-free Heun step on a caller-owned device state (raw
    device pointers: U_dev_ptr holds nvar*ncell doubles, out_dev_ptr 3)."""
    desc = desc_of(mesh)
    _check(lib().khy_step_noalloc(ctypes.byref(desc), ctypes.c_void_p(U_dev_ptr), float(t), float(t_end),
                                  ctypes.c_void_p(out_dev_ptr), ctypes.c_void_p(stream or 0)))


def khy_get_time(h) -> Tuple[float, int, float]:
    t, s, dt = ctypes.c_double(), ctypes.c_long(), ctypes.c_double()
    _check(lib().khy_get_time(h, ctypes.byref(t), ctypes.byref(s), ctypes.byref(dt)))
    return t.value, s.value, dt.value


def khy_totals(h, nvar: int) -> np.ndarray:
    out = np.zeros(5)
    _check(lib().khy_totals(h, ctypes.c_void_p(out.ctypes.data)))
    return out[:nvar]


def khy_get_flags(h, clear: bool = False) -> Tuple[int, int]:
    f = ctypes.c_uint()
    n = ctypes.c_ulonglong()
    _check(lib().khy_get_flags(h, ctypes.byref(f), ctypes.byref(n), int(clear)))
    return f.value, n.value


def khy_device_bytes(h) -> Tuple[int, int]:
    """(state bytes, total bytes) of device memory held by a simulation."""
    a = ctypes.c_size_t()
    b = ctypes.c_size_t()
    _check(lib().khy_device_bytes(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


# ------------------------------------------------------------ wrapper

class Sim:
    """One simulation on the current CUDA device (owns its device state)."""

    def __init__(self, mesh: Mesh, stream: Optional[int] = None):
        self.mesh = mesh
        self.h = khy_create(mesh, stream)

    def close(self) -> None:
        if self.h:
            khy_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_primitive(self, W) -> None:
        khy_set_primitive(self.h, W)

    def set_conserved(self, U) -> None:
        khy_set_conserved(self.h, U)

    def set_boundary(self, axis: int, side: int, bc: int) -> None:
        khy_set_boundary(self.h, axis, side, bc)

    def set_time(self, t: float) -> None:
        khy_set_time(self.h, t)

    def step_to(self, t_end: float, max_steps: int = -1) -> Tuple[int, float]:
        return khy_step_to(self.h, t_end, max_steps)

    def enqueue_steps(self, t_end: float, nsteps: int) -> None:
        khy_enqueue_steps(self.h, t_end, nsteps)

    def profile_steps(self, t_end: float, nsteps: int) -> Tuple[float, float, float]:
        return khy_profile_steps(self.h, t_end, nsteps)

    def conserved(self, out=None):
        if out is None:
            out = np.empty(self.mesh.shape, dtype=np.float64)
        khy_get_conserved(self.h, out)
        return out

    def primitive(self, out=None):
        """(rho, v.., p) as the library recovers them (flux precision, widened)."""
        if out is None:
            out = np.empty(self.mesh.shape, dtype=np.float64)
        khy_get_primitive(self.h, out)
        return out

    def time(self) -> Tuple[float, int, float]:
        return khy_get_time(self.h)

    def totals(self) -> np.ndarray:
        return khy_totals(self.h, self.mesh.nvar)

    def flags(self, clear: bool = False) -> Tuple[int, int]:
        return khy_get_flags(self.h, clear)

    def device_bytes(self) -> Tuple[int, int]:
        return khy_device_bytes(self.h)


# ------------------------------------------------------------ many grids

class Batch:
    """Many independent grids (one ndim, one precision) stepped together."""

    def __init__(self, meshes, stream: Optional[int] = None):
        self.meshes = list(meshes)
        arr = (khy_mesh_desc * len(self.meshes))()
        for k, m in enumerate(self.meshes):
            arr[k] = desc_of(m)
        self.h = ctypes.c_void_p()
        _check(lib().khy_batch_create(arr, len(self.meshes), ctypes.c_void_p(stream or 0), ctypes.byref(self.h)))
        self.sizes = [m.nvar * m.ncell for m in self.meshes]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)

    def close(self) -> None:
        if self.h:
            lib().khy_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _concat(self, arrays) -> np.ndarray:
        flat = np.concatenate([np.ascontiguousarray(a, dtype=np.float64).ravel() for a in arrays])
        assert flat.size == self.offsets[-1]
        return flat

    def set_primitive(self, Ws) -> None:
        flat = self._concat(Ws)
        _check(lib().khy_batch_set_primitive(self.h, ctypes.c_void_p(flat.ctypes.data), flat.size))

    def set_conserved(self, Us) -> None:
        flat = self._concat(Us)
        _check(lib().khy_batch_set_conserved(self.h, ctypes.c_void_p(flat.ctypes.data), flat.size))

    def conserved_flat(self, out: Optional[np.ndarray] = None) -> np.ndarray:
        if out is None:
            out = np.empty(int(self.offsets[-1]), dtype=np.float64)
        _check(lib().khy_batch_get_conserved(self.h, ctypes.c_void_p(out.ctypes.data), out.size))
        return out

    def conserved(self):
        flat = self.conserved_flat()
        return [flat[self.offsets[k]:self.offsets[k + 1]].reshape(m.shape) for k, m in enumerate(self.meshes)]

    def set_target(self, t_end: float, max_steps: int = -1, grid: int = -1) -> None:
        _check(lib().khy_batch_set_target(self.h, int(grid), float(t_end), int(max_steps)))

    def enqueue_steps(self, nsteps: int) -> None:
        _check(lib().khy_batch_enqueue_steps(self.h, int(nsteps)))

    def run(self) -> int:
        n = ctypes.c_long(0)
        _check(lib().khy_batch_run(self.h, ctypes.byref(n)))
        return n.value

    def clock(self, grid: int) -> Tuple[float, int, float]:
        t, s, dt = ctypes.c_double(), ctypes.c_long(), ctypes.c_double()
        _check(lib().khy_batch_get_clock(self.h, int(grid), ctypes.byref(t), ctypes.byref(s), ctypes.byref(dt)))
        return t.value, s.value, dt.value

    def autotune(self, trial_steps: int = 2) -> Tuple[int, float]:
        v, ms = ctypes.c_int(), ctypes.c_float()
        _check(lib().khy_batch_autotune(self.h, int(trial_steps), ctypes.byref(v), ctypes.byref(ms)))
        return v.value, ms.value

    def set_variant(self, v: int) -> None:
        _check(lib().khy_batch_set_variant(self.h, int(v)))

    def set_schedule(self, variant: int, ctas_per_slot: int) -> None:
        _check(lib().khy_batch_set_schedule(self.h, int(variant), int(ctas_per_slot)))

    def schedule(self) -> Tuple[int, int]:
        v, c = ctypes.c_int(0), ctypes.c_int(0)
        _check(lib().khy_batch_get_schedule(self.h, ctypes.byref(v), ctypes.byref(c)))
        return v.value, c.value

    def profile_steps(self, nsteps: int) -> Tuple[float, float, float]:
        ms = (ctypes.c_float * 3)()
        _check(lib().khy_batch_profile_steps(self.h, int(nsteps), ms))
        return ms[0], ms[1], ms[2]

    def info(self):
        cells, pool, v, nb = ctypes.c_longlong(), ctypes.c_size_t(), ctypes.c_int(), ctypes.c_int()
        _check(lib().khy_batch_info(self.h, ctypes.byref(cells), ctypes.byref(pool), ctypes.byref(v), ctypes.byref(nb)))
        return {"cells": cells.value, "pool_doubles": pool.value, "variant": v.value, "nblocks": nb.value}


# ------------------------------------------------------------ serving

JOB_QUEUED, JOB_ACTIVE, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


class Server:
    """Continuous-batching job server (a thread of libkhydro.so)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 256, stream: Optional[int] = None):
        self.h = ctypes.c_void_p()
        _check(lib().khy_server_create(int(hbm_budget_bytes), int(max_slots), ctypes.c_void_p(stream or 0),
                                       ctypes.byref(self.h)))
        self.meshes = {}

    def close(self) -> None:
        if self.h:
            lib().khy_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, mesh: Mesh, W: np.ndarray, t_end: float) -> int:
        W = np.ascontiguousarray(W, dtype=np.float64)
        desc = desc_of(mesh)
        jid = ctypes.c_long()
        _check(lib().khy_server_submit(self.h, ctypes.byref(desc), ctypes.c_void_p(W.ctypes.data), W.size,
                                       float(t_end), ctypes.byref(jid)))
        self.meshes[jid.value] = mesh
        return jid.value

    def poll(self, job: int):
        st, steps = ctypes.c_int(), ctypes.c_long()
        times = (ctypes.c_double * 3)()
        _check(lib().khy_server_poll(self.h, int(job), ctypes.byref(st), times, ctypes.byref(steps)))
        return st.value, (times[0], times[1], times[2]), steps.value

    def wait(self, job: int, timeout_s: float = 600.0) -> None:
        _check(lib().khy_server_wait(self.h, int(job), float(timeout_s)))

    def result(self, job: int, release: bool = False) -> np.ndarray:
        mesh = self.meshes[job]
        out = np.empty(mesh.shape, dtype=np.float64)
        _check(lib().khy_server_result(self.h, int(job), ctypes.c_void_p(out.ctypes.data), out.size, int(release)))
        if release:
            self.meshes.pop(job, None)
        return out

    def stats(self):
        c, a, q, cu, el = ctypes.c_long(), ctypes.c_int(), ctypes.c_int(), ctypes.c_ulonglong(), ctypes.c_double()
        _check(lib().khy_server_stats(self.h, ctypes.byref(c), ctypes.byref(a), ctypes.byref(q), ctypes.byref(cu),
                                      ctypes.byref(el)))
        return {"completed": c.value, "active": a.value, "queued": q.value, "cell_updates": cu.value,
                "elapsed_s": el.value}
