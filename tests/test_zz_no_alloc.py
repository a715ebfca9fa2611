"""khy_step_noalloc: the one-step entry point for callers that cannot
allocate device memory when they step (a host program that reserves all
device memory for its own pool, a real-time loop that cannot take the
synchronisation an allocation may cause, a plug-in whose host owns every
allocation).  Its scratch is a fixed file-scope device array, so the caller
only passes the state and an output buffer.

Checked through the C ABI against the allocating entry point (khy_create +
khy_step_to): two calls in a row, within the parity tolerances of the GPU
tests (all-FP64 1e-12 relative L1 per field; mixed 1e-5 density, momenta
and energy, 1e-4 pressure), and in FP64 bit for bit against the CPU
oracle's Heun step.  The caller's buffers here come from torch; the entry point itself
allocates nothing.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from hydro_util import field_errors, gate_errors, mixed_gates
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    return khydro


def reference_steps(khydro, mesh, U0, nsteps, t_end):
    """The allocating path, one step at a time."""
    out = []
    with khydro.Sim(mesh) as sim:
        sim.set_conserved(U0)
        for _ in range(nsteps):
            sim.step_to(t_end, 1)
            t, _, dt = sim.time()
            out.append((sim.conserved(), t, dt))
    return out


def within_tolerance(mesh, U, Uref):
    errs = field_errors(mesh, U, Uref)
    if mesh.prec == wl.PREC_FP64:
        return max(errs) <= 1e-12, errs
    return all(e <= g for e, g in zip(gate_errors(mesh, U, Uref), mixed_gates(mesh.nvar))), errs


CASES = [
    ("kh2d-mixed", lambda: wl.kelvin_helmholtz(128, prec=wl.PREC_MIXED)),
    ("turb3d-fp64", lambda: wl.turbulence(32, prec=wl.PREC_FP64)),
    ("sod1d-fp64", lambda: wl.sod(512, prec=wl.PREC_FP64)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point_two_calls(kh, name, make):
    import torch
    import oracle
    mesh, W = make()
    U0 = oracle.prim_to_cons(mesh, W)  # initial conserved state (input only)
    t_end = 10.0
    ref = reference_steps(kh, mesh, U0, 2, t_end)
    torch.cuda.synchronize()
    U_dev = torch.from_numpy(U0.copy()).cuda()
    out_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    t = 0.0
    for call in range(2):
        kh.khy_step_noalloc(mesh, U_dev.data_ptr(), t, t_end, out_dev.data_ptr(), stream)
        torch.cuda.synchronize()
        t_new, dt, status = out_dev.cpu().tolist()
        Uref, tref, dtref = ref[call]
        ok, errs = within_tolerance(mesh, U_dev.cpu().numpy(), Uref)
        assert ok, (call, errs)
        assert status == 0.0
        assert abs(dt - dtref) <= 1e-12 * dtref and abs(t_new - tref) <= 1e-12 * tref
        t = t_new
    if mesh.prec == wl.PREC_FP64:
        # the FP64 step follows the oracle's operation order: same bits
        Uo, to = U0, 0.0
        for _ in range(2):
            Uo, to, _, _ = oracle.heun_step(mesh, Uo, to, t_end)
        np.testing.assert_array_equal(U_dev.cpu().numpy(), Uo)
        assert t == to


def test_noalloc_clips_to_t_end_and_rejects_oversized(kh):
    import torch
    mesh, W = wl.kelvin_helmholtz(64, prec=wl.PREC_MIXED)
    import oracle
    U_dev = torch.from_numpy(oracle.prim_to_cons(mesh, W)).cuda()
    out_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    # a step that would overshoot lands exactly on t_end
    kh.khy_step_noalloc(mesh, U_dev.data_ptr(), 0.0, 1e-6, out_dev.data_ptr())
    torch.cuda.synchronize()
    t_new, dt, _ = out_dev.cpu().tolist()
    assert t_new == 1e-6 and dt == 1e-6
    # no step past t_end
    before = U_dev.clone()
    kh.khy_step_noalloc(mesh, U_dev.data_ptr(), 1e-6, 1e-6, out_dev.data_ptr())
    torch.cuda.synchronize()
    assert out_dev[1].item() == 0.0 and torch.equal(before, U_dev)
    # a state beyond the fixed scratch is refused before any launch
    big = wl.Mesh(ndim=3, n=(128, 128, 128))
    with pytest.raises(kh.KhydroError) as ei:
        kh.khy_step_noalloc(big, U_dev.data_ptr(), 0.0, 1.0, out_dev.data_ptr())
    assert ei.value.status == -1 and "no-allocation limit" in str(ei.value)
    assert np.isfinite(U_dev.cpu().numpy()).all()


def test_noalloc_at_the_size_limit(kh):
    # 1024^2 cells in 2D need exactly the scratch size (4 x 1024^2 x 8 bytes)
    # and are stepped; one more row is refused; 94^3 fits in 3D, 95^3 does not
    import torch
    import oracle
    mesh, W = wl.kelvin_helmholtz(1024, prec=wl.PREC_MIXED)
    assert mesh.nvar * mesh.ncell * 8 == kh.KHY_NOALLOC_SCRATCH_BYTES
    U0 = oracle.prim_to_cons(mesh, W)
    Uref, tref, _ = reference_steps(kh, mesh, U0, 1, 10.0)[0]
    U_dev = torch.from_numpy(U0.copy()).cuda()
    out_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    kh.khy_step_noalloc(mesh, U_dev.data_ptr(), 0.0, 10.0, out_dev.data_ptr())
    torch.cuda.synchronize()
    ok, errs = within_tolerance(mesh, U_dev.cpu().numpy(), Uref)
    assert ok, errs
    assert out_dev[2].item() == 0.0 and abs(out_dev[0].item() - tref) <= 1e-6 * tref
    for n, refused in (((1024, 1025, 1), True), ((94, 94, 94), False), ((95, 95, 95), True)):
        m = wl.Mesh(ndim=2 if n[2] == 1 else 3, n=n, prec=wl.PREC_FP64)
        if refused:
            with pytest.raises(kh.KhydroError) as ei:
                kh.khy_step_noalloc(m, U_dev.data_ptr(), 0.0, 1.0, out_dev.data_ptr())
            assert ei.value.status == -1 and "no-allocation limit" in str(ei.value)
        else:
            Wm = wl.uniform(m)
            Um = torch.from_numpy(oracle.prim_to_cons(m, Wm)).cuda()
            kh.khy_step_noalloc(m, Um.data_ptr(), 0.0, 1.0, out_dev.data_ptr())
            torch.cuda.synchronize()
            assert out_dev[1].item() > 0.0 and out_dev[2].item() == 0.0
            np.testing.assert_array_equal(Um.cpu().numpy(), oracle.prim_to_cons(m, Wm))  # uniform stays uniform


def test_noalloc_reports_step_underflow(kh):
    # a remaining interval t_end - t below 1e-300 cannot be stepped: status
    # bit 4, dt 0, time and state unchanged (a caller looping to t_end stops
    # on the bit)
    import torch
    import oracle
    mesh, W = wl.kelvin_helmholtz(64, prec=wl.PREC_FP64)
    U0 = oracle.prim_to_cons(mesh, W)
    U_dev = torch.from_numpy(U0.copy()).cuda()
    out_dev = torch.zeros(3, dtype=torch.float64, device="cuda")
    kh.khy_step_noalloc(mesh, U_dev.data_ptr(), 0.0, 1e-305, out_dev.data_ptr())
    torch.cuda.synchronize()
    t_new, dt, status = out_dev.cpu().tolist()
    assert int(status) & 4 and dt == 0.0 and t_new == 0.0
    np.testing.assert_array_equal(U_dev.cpu().numpy(), U0)
