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
