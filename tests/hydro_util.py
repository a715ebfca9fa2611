"""Shared helpers of the tests (no method arithmetic beyond diagnostics)."""
import numpy as np

import oracle


def rel_l1(a, b):
    """Sum |a - b| / sum |b| (b is the reference)."""
    den = float(np.abs(b).sum())
    return float(np.abs(a - b).sum()) / den if den > 0 else float(np.abs(a - b).sum())


def pressure_np(mesh, U):
    """Pressure of a conserved state, plain numpy (diagnostic only)."""
    rho = U[0]
    ke = 0.5 * sum(U[1 + d] ** 2 for d in range(mesh.ndim)) / rho
    return (mesh.gamma - 1.0) * (U[mesh.nvar - 1] - ke)


def oracle_run(mesh, W, t_end=1e30, max_steps=1 << 40, allow_flags=False):
    """Oracle run from primitive W; a parity case must stay physical (no
    floor, no negative pressure) unless allow_flags."""
    U0 = oracle.prim_to_cons(mesh, W)
    U, t, s, f = oracle.run(mesh, U0, 0.0, t_end, max_steps)
    if not allow_flags:
        assert f == 0, "oracle flags %d: the parity input is not a valid physical case" % f
    return U, t, s, f


def gpu_run(mesh, W, t_end=1e30, max_steps=-1):
    from paper_2501_02317_gb300 import khydro
    with khydro.Sim(mesh) as sim:
        sim.set_primitive(np.ascontiguousarray(W))
        s, t = sim.step_to(t_end, max_steps)
        U = sim.conserved()
        _, _, dt = sim.time()
    return U, t, s, dt


def field_errors(mesh, U, Uref):
    errs = [rel_l1(U[q], Uref[q]) for q in range(mesh.nvar)]
    errs.append(rel_l1(pressure_np(mesh, U), pressure_np(mesh, Uref)))
    return errs


FP64_TOL = 1e-12


def gate_errors(mesh, U, Uref):
    """The errors the gates apply to, in the order of field_errors (rho,
    momenta, E, p): relative L1 of rho, E and p; for each momentum
    component m_d, sum |m_d - m_d,ref| / sum |m_ref| with |m_ref| the
    magnitude of the reference momentum vector.  A component's own sum can
    be a tiny fraction of the momentum the fluxes carry (the seeded
    transverse velocity of the shear layer is 1/50 of the streaming one),
    and its plain relative L1 then measures that fraction, not the
    precision of the step."""
    nd = mesh.ndim
    errs = [rel_l1(U[0], Uref[0])]
    mag = float(np.sqrt(sum(Uref[1 + d] ** 2 for d in range(nd))).sum())
    for d in range(nd):
        diff = float(np.abs(U[1 + d] - Uref[1 + d]).sum())
        errs.append(diff / mag if mag > 0 else diff)
    errs.append(rel_l1(U[nd + 1], Uref[nd + 1]))
    errs.append(rel_l1(pressure_np(mesh, U), pressure_np(mesh, Uref)))
    return errs


def mixed_gates(nvar):
    """Gates of the mixed path against the FP64 oracle, in the order of
    gate_errors (rho, momenta, E, p): the density and pressure gates are the
    method's stated accuracy targets (1e-5, 1e-4); the momenta and the
    energy, flux-summed conserved fields like the density, take the
    density's."""
    return [1e-5] * nvar + [1e-4]


def field_names(ndim):
    return ["rho"] + ["m_%s" % "xyz"[d] for d in range(ndim)] + ["E", "p"]


def check_fields(mesh, U, Uref, fp64, gates=None):
    """Assert every field's gate (all-FP64 path: FP64_TOL on the plain
    relative L1 of every field; otherwise `gates`, default mixed_gates, on
    gate_errors) and return the plain relative L1 of each field by name
    (the per-field errors the results state)."""
    errs = field_errors(mesh, U, Uref)
    if fp64:
        checked, gates = errs, [FP64_TOL] * len(errs)
    else:
        checked = gate_errors(mesh, U, Uref)
        gates = gates if gates is not None else mixed_gates(mesh.nvar)
    names = field_names(mesh.ndim)
    bad = [(n, e, g) for n, e, g in zip(names, checked, gates) if not e <= g]
    assert not bad, bad
    return dict(zip(names, errs))


# Riemann problems for the Sec. 4.2 shock-tube checks (values chosen here,
# not a published suite): (left (rho, v, p), right, x0, t_end)
SHOCK_TUBES = {
    "strong_shock": ((1.0, 0.0, 500.0), (1.0, 0.0, 0.02), 0.5, 0.012),
    "double_rarefaction": ((1.0, -1.8, 0.5), (1.0, 1.8, 0.5), 0.5, 0.12),
    "colliding_streams": ((1.2, 2.4, 1.5), (0.9, -2.1, 0.9), 0.5, 0.06),
    "moving_contact": ((1.3, 0.15, 1.0), (0.8, 0.15, 1.0), 0.5, 0.5),
    "shock_into_rest": ((2.5, 1.2, 4.0), (1.0, 0.0, 1.0), 0.4, 0.08),
}


def tube_errors(left, right, x0, t, gamma, W):
    """Mean |W - exact cell average| per primitive, over max |exact|."""
    from oracle import exact_riemann as er
    n = W.shape[-1]
    ex = er.cell_averages(left, right, gamma, x0, t, np.linspace(0.0, 1.0, n + 1))
    return [float(np.mean(np.abs(W[q].ravel() - ex[q]))) / float(np.abs(ex[q]).max()) for q in range(3)]


def step_with_totals(sim, mesh, nsteps, drift_tol=None, agree_tol=1e-15):
    """Steps `sim` one step at a time.  After every step the library's
    compensated totals (khy_totals) must equal the oracle's compensated
    totals of the state the library holds to agree_tol x sum |q| (an
    independent sum: a totals kernel that dropped a field or returned a
    stale value fails here whenever the totals move), and, when drift_tol
    is given, the oracle's totals of consecutive states must differ by at
    most drift_tol x sum |q| of the earlier state.  Returns the largest
    drift and disagreement per field."""
    nv = mesh.nvar
    U = sim.conserved()
    scale = np.abs(U).reshape(nv, -1).sum(axis=1)
    prev = oracle.totals(mesh, U)
    agree_max = np.abs(sim.totals() - prev) / scale
    assert np.all(agree_max <= agree_tol), agree_max
    drift_max = np.zeros(nv)
    for _ in range(nsteps):
        sim.step_to(1e30, 1)
        U = sim.conserved()
        ref = oracle.totals(mesh, U)
        agree = np.abs(sim.totals() - ref) / scale
        assert np.all(agree <= agree_tol), agree
        drift = np.abs(ref - prev) / scale
        if drift_tol is not None:
            assert np.all(drift <= drift_tol), drift
        agree_max = np.maximum(agree_max, agree)
        drift_max = np.maximum(drift_max, drift)
        prev = ref
        scale = np.abs(U).reshape(nv, -1).sum(axis=1)
    return drift_max, agree_max
