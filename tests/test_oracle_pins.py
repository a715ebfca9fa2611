"""Pins for the CPU oracle: each check is fixed by the paper or by the
mathematics, not by the oracle itself.

* minmod truth table (Eq. 3)
* HLLC: consistency with the physical flux of Eq. 2, exact resolution of
  isolated contacts, supersonic upwinding, mirror symmetry
* exact Riemann solver: Newton vs bisection, Rankine-Hugoniot jumps at the
  shock, Riemann invariants through the rarefaction
* whole scheme: Sod tube vs the exact solution (Sec. 4.2), sound-wave
  convergence ~ N^-2 (Sec. 4.1, Eq. 6), conservation to round-off with
  periodic boundaries, axis interchange gives identical results (Sec. 4.2),
  uniform state stays uniform, outflow-boundary momentum budget, reflecting
  walls conserve mass and energy, diagonal symmetry of the implosion (Sec. 4.4)
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exact_riemann as er
from paper_2501_02317_gb300 import workloads as wl


# ------------------------------------------------------------ Eq. 3 minmod

@pytest.mark.parametrize("a,b,want", [
    (1.0, 2.0, 1.0),      # |a| < |b|, ab > 0 -> a
    (2.0, 1.0, 1.0),      # |a| >= |b|, ab > 0 -> b
    (-1.0, -3.0, -1.0),
    (-3.0, -1.0, -1.0),
    (2.0, 2.0, 2.0),      # |a| == |b| -> b
    (1.0, -1.0, 0.0),     # ab < 0 -> 0
    (-5.0, 0.5, 0.0),
    (0.0, 3.0, 0.0),      # ab == 0 -> 0 (reading)
    (3.0, 0.0, 0.0),
    (1e-200, 1e-200, 1e-200),  # the product would underflow; the signs decide
])
def test_minmod_truth_table(a, b, want):
    assert oracle.minmod(a, b) == want


# ------------------------------------------------------------ HLLC pins

def physical_flux(gamma, w):
    """Normal flux of Eq. 2 for w = (rho, u, t1, t2, p)."""
    rho, u, t1, t2, p = w
    E = p / (gamma - 1.0) + 0.5 * rho * (u * u + t1 * t1 + t2 * t2)
    return np.array([rho * u, rho * u * u + p, rho * u * t1, rho * u * t2, (E + p) * u])


def _rand_state(rng, umax=2.0):
    return np.array([math.exp(rng.uniform(-2, 2)), rng.uniform(-umax, umax), rng.uniform(-1, 1),
                     rng.uniform(-1, 1), math.exp(rng.uniform(-2, 2))])


def test_hllc_consistency():
    rng = np.random.default_rng(0)
    for gamma in (1.4, 5.0 / 3.0):
        for _ in range(200):
            w = _rand_state(rng, umax=5.0)
            F = oracle.hllc(gamma, w, w)
            ref = physical_flux(gamma, w)
            np.testing.assert_allclose(F, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_hllc_stationary_contact_exact():
    # equal pressure, zero velocity, density jump: no mass or energy flux
    for rl, rr in [(1.0, 0.125), (0.3, 7.0), (2.0, 2.0)]:
        wl_ = np.array([rl, 0.0, 0.2, -0.4, 0.9])
        wr_ = np.array([rr, 0.0, -0.3, 0.1, 0.9])
        F = oracle.hllc(1.4, wl_, wr_)
        assert F[0] == 0.0 and F[4] == 0.0 and F[2] == 0.0 and F[3] == 0.0
        assert F[1] == 0.9


@pytest.mark.parametrize("u", [0.7, -0.7, 1e-3, -2.5])
def test_hllc_moving_contact_is_upwind(u):
    # same u and p on both sides: HLLC resolves the contact exactly and the
    # flux is the physical flux of the upwind state
    wl_ = np.array([1.0, u, 0.3, -0.2, 1.0])
    wr_ = np.array([0.1, u, -0.5, 0.6, 1.0])
    F = oracle.hllc(5.0 / 3.0, wl_, wr_)
    ref = physical_flux(5.0 / 3.0, wl_ if u > 0 else wr_)
    np.testing.assert_allclose(F, ref, rtol=1e-14, atol=1e-15)


def test_hllc_supersonic_upwinding():
    g = 1.4
    rng = np.random.default_rng(1)
    for _ in range(50):
        a, b = _rand_state(rng), _rand_state(rng)
        ca = math.sqrt(g * a[4] / a[0]); cb = math.sqrt(g * b[4] / b[0])
        shift = 10.0 * (ca + cb) + 20.0
        a[1] += shift; b[1] += shift      # everything moves right, supersonic
        np.testing.assert_allclose(oracle.hllc(g, a, b), physical_flux(g, a), rtol=1e-13)
        a[1] -= 2 * shift; b[1] -= 2 * shift  # everything moves left
        np.testing.assert_allclose(oracle.hllc(g, a, b), physical_flux(g, b), rtol=1e-13)


def test_hllc_mirror_symmetry():
    # reflecting x -> -x swaps the states and flips the normal velocity: mass,
    # transverse momentum and energy fluxes change sign, normal momentum does not
    rng = np.random.default_rng(2)
    M = np.array([1.0, -1.0, 1.0, 1.0, 1.0])
    for _ in range(200):
        a, b = _rand_state(rng, 3.0), _rand_state(rng, 3.0)
        F = oracle.hllc(1.4, a, b)
        G = oracle.hllc(1.4, b * M, a * M)
        np.testing.assert_allclose(F * np.array([-1, 1, -1, -1, -1]), G, rtol=1e-12,
                                   atol=1e-12 * np.abs(F).max())


def test_hllc_flux_between_hll_bounds_for_mass():
    # The HLLC mass flux of a strong 1D shock state pair lies between the
    # physical fluxes' range extended by the HLL average (sanity of branch choice)
    wl_ = np.array([1.0, 0.0, 0.0, 0.0, 1.0])
    wr_ = np.array([0.125, 0.0, 0.0, 0.0, 0.1])
    F = oracle.hllc(1.4, wl_, wr_)
    assert F[0] > 0.0 and F[4] > 0.0 and F[1] > 0.1


# ------------------------------------------------ exact Riemann solver pins

SOD_L, SOD_R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def test_exact_riemann_newton_vs_bisection():
    for L, R, g in [(SOD_L, SOD_R, 1.4), ((1.0, -2.0, 0.4), (1.0, 2.0, 0.4), 1.4),
                    ((1.0, 0.0, 1000.0), (1.0, 0.0, 0.01), 1.4), ((5.99924, 19.5975, 460.894), (5.99242, -6.19633, 46.095), 1.4)]:
        p_newton, _ = er.star_state(L, R, g)
        p_bis = er.star_pressure_bisect(L, R, g)
        assert abs(p_newton - p_bis) <= 1e-12 * p_bis


def test_exact_riemann_rankine_hugoniot_and_invariants():
    g = 1.4
    ps, us = er.star_state(SOD_L, SOD_R, g)
    # right-moving shock: sample just behind and ahead of it
    xi = np.linspace(-2.0, 2.0, 40001)
    w = er.sample(SOD_L, SOD_R, g, xi)
    rho, u, p = w
    jump = np.where(np.abs(np.diff(p)) > 1e-3)[0]
    k = jump[-1]  # the shock is the right-most pressure jump
    S = 0.5 * (xi[k] + xi[k + 1])
    r1, u1, p1 = rho[k], u[k], p[k]
    r0, u0, p0 = rho[k + 1], u[k + 1], p[k + 1]
    E = lambda r, uu, pp: pp / (g - 1) + 0.5 * r * uu * uu
    # Rankine-Hugoniot: F(U1) - F(U0) = S (U1 - U0) for the exact shock speed
    Sx = (r1 * u1 - r0 * u0) / (r1 - r0)
    assert abs(Sx - S) < 1e-3
    np.testing.assert_allclose(r1 * u1 * u1 + p1 - (r0 * u0 * u0 + p0), Sx * (r1 * u1 - r0 * u0), rtol=1e-10)
    np.testing.assert_allclose((E(r1, u1, p1) + p1) * u1 - (E(r0, u0, p0) + p0) * u0,
                               Sx * (E(r1, u1, p1) - E(r0, u0, p0)), rtol=1e-10)
    # left rarefaction: entropy p/rho^g and the invariant u + 2c/(g-1) are constant
    fan = (xi > -math.sqrt(g) + 1e-6) & (xi < us - math.sqrt(g * ps / (1.0 * (ps / 1.0) ** (1 / g))) - 1e-6)
    assert fan.sum() > 100
    c = np.sqrt(g * p[fan] / rho[fan])
    np.testing.assert_allclose(p[fan] / rho[fan] ** g, 1.0, rtol=1e-12)
    np.testing.assert_allclose(u[fan] + 2 * c / (g - 1), 2 * math.sqrt(g) / (g - 1), rtol=1e-12)
    # the pressure and velocity are continuous across the contact
    assert abs(p[np.searchsorted(xi, us) - 1] - p[np.searchsorted(xi, us) + 1]) < 1e-12


# ------------------------------------------------- whole-scheme pins

def _run(mesh, W, t_end, max_steps=1 << 40):
    U0 = oracle.prim_to_cons(mesh, W)
    U, t, s, f = oracle.run(mesh, U0, 0.0, t_end, max_steps)
    return U0, U, t, s, f


def sod_errors(n):
    m, W = wl.sod(n)
    _, U, t, s, f = _run(m, W, 0.2)
    assert t == 0.2 and f == 0
    Wf, _ = oracle.cons_to_prim(m, U)
    ex = er.cell_averages(SOD_L, SOD_R, 1.4, 0.5, 0.2, np.linspace(0.0, 1.0, n + 1))
    return [float(np.mean(np.abs(Wf[q].ravel() - ex[q]))) for q in range(3)], s


def test_sod_against_exact_solution():
    errs, steps = sod_errors(512)
    # a second-order Godunov scheme on 512 cells: L1 of a few 1e-3 at most
    assert errs[0] < 3e-3 and errs[1] < 4e-3 and errs[2] < 2e-3, errs
    assert 450 < steps < 700


def test_sod_converges():
    e128, _ = sod_errors(128)
    e1024, _ = sod_errors(1024)
    order = math.log(e128[0] / e1024[0]) / math.log(8.0)
    # discontinuous solution: first order at best, ~0.6-0.9 observed in practice
    assert 0.55 < order < 1.2, order


def l1_eq6(q, q0):
    """Normalised L1 error of Eq. 6."""
    return float(np.sum(np.abs(q - q0)) / (q0.size * (q0.max() - q0.min())))


@pytest.mark.parametrize("p0,amp", [(5.0 / 3.0, 1e-6), (3.0 / 5.0, 1e-6)])
def test_sound_wave_second_order(p0, amp):
    errs = []
    Ns = [64, 128, 256, 512]
    for n in Ns:
        m, W = wl.sound_wave(n, amp=amp, p0=p0)
        cs = wl.sound_speed(p0, 1.0, m.gamma)
        U0, U, t, s, f = _run(m, W, 1.0 / cs)   # one period: L / c_s
        errs.append(l1_eq6(U[0], U0[0]))
    slopes = [math.log(errs[i + 1] / errs[i]) / math.log(2.0) for i in range(len(Ns) - 1)]
    assert slopes[-1] < -1.8 and slopes[-2] < -1.8, (errs, slopes)


def _rel_drift(mesh, Ua, Ub):
    ta, tb = oracle.totals(mesh, Ua), oracle.totals(mesh, Ub)
    scale = np.abs(Ua).reshape(mesh.nvar, -1).sum(axis=1)
    return np.abs(tb - ta) / scale


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_conservation_periodic(ndim):
    n = {1: (64, 1, 1), 2: (24, 20, 1), 3: (12, 10, 8)}[ndim]
    m = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3)
    W = wl.random_jumpy(m)
    U = oracle.prim_to_cons(m, W)
    t = 0.0
    for _ in range(5):
        Un, t, dt, f = oracle.heun_step(m, U, t, 10.0)
        assert f == 0
        assert np.all(_rel_drift(m, U, Un) <= 1e-14)
        U = Un


def test_axis_interchange_identical():
    # Sec. 4.2: Sod along x, y or z gives identical results
    m1, W1 = wl.sod(128, axis=0, ndim=1)
    _, U1, t1, s1, _ = _run(m1, W1, 0.2)
    for ndim, axis in [(2, 1), (2, 0), (3, 2), (3, 0)]:
        m, W = wl.sod(128, axis=axis, ndim=ndim, ntrans=3)
        _, U, t, s, _ = _run(m, W, 0.2)
        assert s == s1 and t == t1
        rho = np.moveaxis(U[0], 2 - axis, -1).reshape(-1, 128)
        mom = np.moveaxis(U[1 + axis], 2 - axis, -1).reshape(-1, 128)
        E = np.moveaxis(U[-1], 2 - axis, -1).reshape(-1, 128)
        for row in range(rho.shape[0]):
            np.testing.assert_array_equal(rho[row], U1[0].ravel())
            np.testing.assert_array_equal(mom[row], U1[1].ravel())
            np.testing.assert_array_equal(E[row], U1[2].ravel())
        for d in range(ndim):
            if d != axis:
                assert np.all(U[1 + d] == 0.0)


@pytest.mark.parametrize("ndim", [1, 2, 3])
def test_uniform_state_stays_uniform(ndim):
    n = {1: (16, 1, 1), 2: (8, 6, 1), 3: (6, 5, 4)}[ndim]
    m = wl.Mesh(ndim=ndim, n=n, gamma=5.0 / 3.0, cfl=0.4)
    W = wl.uniform(m)
    U0 = oracle.prim_to_cons(m, W)
    U, t, s, f = oracle.run(m, U0, 0.0, 1.0, 20)
    np.testing.assert_array_equal(U, U0)


def test_uniform_dt_closed_form():
    m = wl.Mesh(ndim=3, n=(8, 4, 2), hi=(1.0, 2.0, 0.5), gamma=1.4, cfl=0.3)
    W = wl.uniform(m, rho=1.3, v=(0.3, -0.9, 0.1), p=0.7)
    c = math.sqrt(1.4 * 0.7 / 1.3)
    want = 0.3 * min(0.125 / (0.3 + c), 0.5 / (0.9 + c), 0.25 / (0.1 + c))
    assert abs(oracle.cfl_dt(m, oracle.prim_to_cons(m, W)) - want) <= 1e-15 * want


def test_prim_cons_roundtrip():
    m = wl.Mesh(ndim=3, n=(5, 4, 3))
    W = wl.random_jumpy(m)
    W2, f = oracle.cons_to_prim(m, oracle.prim_to_cons(m, W))
    assert f == 0
    np.testing.assert_allclose(W2, W, rtol=1e-12)


def test_outflow_momentum_budget():
    # before the waves reach the ends, the only boundary fluxes are the
    # pressures of the undisturbed states: d(sum m)/dt = (p_L - p_R)/dx
    m, W = wl.sod(256)
    U0, U, t, s, f = _run(m, W, 0.15)
    tot0, tot1 = oracle.totals(m, U0), oracle.totals(m, U)
    assert tot1[0] == tot0[0] and tot1[2] == tot0[2]
    np.testing.assert_allclose(tot1[1] - tot0[1], (1.0 - 0.1) * 0.15 * 256, rtol=1e-12)


def test_reflecting_walls_conserve_mass_and_energy():
    m = wl.Mesh(ndim=1, n=(96, 1, 1), gamma=1.4, cfl=0.4,
                bc=((wl.BC_REFLECT, wl.BC_REFLECT),) * 3)
    W = wl.random_jumpy(m, seed=5)
    U0 = oracle.prim_to_cons(m, W)
    U, t, s, f = oracle.run(m, U0, 0.0, 0.3)
    rel = _rel_drift(m, U0, U)
    assert rel[0] <= 1e-14 and rel[2] <= 1e-14


def test_outflow_does_not_inflow():
    # gas at rest against outflow ends: the boundary normal velocity is
    # clamped to point outward, so a gas moving inward sees a wall-like ghost
    m = wl.Mesh(ndim=1, n=(32, 1, 1), gamma=1.4, cfl=0.4, bc=((wl.BC_OUTFLOW, wl.BC_OUTFLOW),) * 3)
    W = wl.uniform(m, rho=1.0, v=(0.5, 0, 0), p=1.0)
    U0 = oracle.prim_to_cons(m, W)
    U, t, s, f = oracle.run(m, U0, 0.0, 0.05)
    m_free = m.replace(bc=((wl.BC_FREE, wl.BC_FREE),) * 3)
    Uf, _, _, _ = oracle.run(m_free, U0, 0.0, 0.05)
    # free boundaries keep the uniform flow; outflow at the low side refuses inflow
    np.testing.assert_array_equal(Uf, U0)
    assert U[0, 0, 0, 0] < U0[0, 0, 0, 0]


@pytest.mark.parametrize("case", ["regular", "rho_below_floor", "negative_eint", "negative_rho"])
def test_recovery_floors_and_flags(case):
    # floors act on the recovered primitive only (no floor in the paper; the
    # reading recorded with the oracle): a density below the floor is raised
    # to it and the momentum divided by the raised density; a pressure below
    # its floor (a negative internal energy included) is raised to the floor;
    # each raises the floor flag, and a non-positive density or a negative
    # internal energy the non-physical flag.  Values from the definitions.
    g = 1.4
    m = wl.Mesh(ndim=1, n=(2, 1, 1), gamma=g, cfl=0.4, bc=((wl.BC_PERIODIC, wl.BC_PERIODIC),) * 3)
    rf, pf = m.rho_floor, m.p_floor
    u = {"regular": (1.0, 0.5, 2.0), "rho_below_floor": (0.25 * rf, 2.5e-11, 1.0),
         "negative_eint": (1.0, 2.0, 1.0), "negative_rho": (-1.0, 0.0, 1.0)}[case]
    U = np.zeros(m.shape)
    U[:, 0, 0, :] = np.array(u)[:, None]
    W, f = oracle.cons_to_prim(m, U)
    rho, mom, E = u
    if case == "regular":
        want = (1.0, 0.5, (g - 1.0) * (2.0 - 0.5 * 0.25))
        want_f = 0
    elif case == "rho_below_floor":
        v = mom / rf
        want = (rf, v, (g - 1.0) * (E - 0.5 * rf * v * v))
        want_f = oracle.FLAG_FLOOR
    elif case == "negative_eint":  # ke = 2 > E = 1
        want = (1.0, 2.0, pf)
        want_f = oracle.FLAG_FLOOR | oracle.FLAG_NONPHYSICAL
    else:  # the floored density is used to go on; the state is flagged
        want = (rf, 0.0, (g - 1.0) * E)
        want_f = oracle.FLAG_FLOOR | oracle.FLAG_NONPHYSICAL
    np.testing.assert_allclose(W[:, 0, 0, 0], want, rtol=1e-15, atol=0.0)
    np.testing.assert_array_equal(W[:, 0, 0, 0], W[:, 0, 0, 1])
    assert f == want_f
    if case == "rho_below_floor":
        # the floor never writes back into the conserved state: a uniform
        # state below the density floor has equal fluxes on every face, so a
        # step leaves it unchanged to the bit
        U2, _, _, f2 = oracle.heun_step(m, U, 0.0, 1e30)
        np.testing.assert_array_equal(U2, U)
        assert f2 == oracle.FLAG_FLOOR


def test_totals_are_compensated_sums():
    # the conservation totals are compensated (Neumaier) sums: on fields whose
    # large terms cancel, a plain left-to-right sum loses the small ones
    # entirely, the compensated sum keeps them (reference: math.fsum, the
    # exactly rounded sum)
    import math
    m = wl.Mesh(ndim=1, n=(1000, 1, 1), gamma=1.4, cfl=0.4, bc=((wl.BC_PERIODIC, wl.BC_PERIODIC),) * 3)
    rng = np.random.default_rng(8)
    U = np.empty(m.shape)
    for q in range(m.nvar):
        x = rng.uniform(0.5, 1.5, 1000)
        big = np.arange(0, 900, 97)
        x[big] = 1e17 * rng.uniform(1.0, 2.0, big.size)  # large terms ...
        x[big + 50] = -x[big]                            # ... each cancelled 50 cells later
        U[q, 0, 0] = x
    tot = oracle.totals(m, U)
    for q in range(m.nvar):
        x = U[q].ravel()
        exact = math.fsum(x)
        plain = 0.0
        for v in x:
            plain += v
        assert abs(plain - exact) > 1.0          # the inputs defeat a plain sum
        assert abs(tot[q] - exact) <= 1e-9 * abs(exact)      # |exact| ~ 1e3


def test_outflow_refuses_inflow_on_both_sides():
    # the same uniform flow entering through the high end instead: the mirror
    # image (x -> 1 - x, v -> -v) of the low-side case must give the mirrored
    # state, the high-side ghost clamping the normal velocity to point out
    m = wl.Mesh(ndim=1, n=(32, 1, 1), gamma=1.4, cfl=0.4, bc=((wl.BC_OUTFLOW, wl.BC_OUTFLOW),) * 3)
    Wa = wl.uniform(m, rho=1.0, v=(0.5, 0, 0), p=1.0)
    Wb = wl.uniform(m, rho=1.0, v=(-0.5, 0, 0), p=1.0)
    Ua, ta, sa, _ = oracle.run(m, oracle.prim_to_cons(m, Wa), 0.0, 0.05)
    Ub, tb, sb, _ = oracle.run(m, oracle.prim_to_cons(m, Wb), 0.0, 0.05)
    assert sa == sb and ta == tb
    mirror = Ua[:, :, :, ::-1] * np.array([1.0, -1.0, 1.0])[:, None, None, None]
    np.testing.assert_allclose(Ub, mirror, rtol=1e-13, atol=1e-13)
    assert Ub[0, 0, 0, -1] < 1.0  # the refused inflow thins the gas at the high end


@pytest.mark.parametrize("bc", [wl.BC_FREE, wl.BC_OUTFLOW])
def test_zero_gradient_ends_carry_the_edge_cells_physical_flux(bc):
    # free ends, and outflow ends whose normal velocity already points out,
    # copy the edge cell into both ghost layers (Sec. 3.1.1): the minmod
    # slopes at the boundary face vanish, both face states are the edge
    # cell's, and HLLC of two equal states is the physical flux of Eq. 2.  So
    # one right-hand side changes the totals by the two edge cells' physical
    # fluxes alone: sum_i dU_i = -(dt/dx) (F(W_last) - F(W_first))
    n, g = 48, 1.4
    m = wl.Mesh(ndim=1, n=(n, 1, 1), gamma=g, cfl=0.4, bc=((bc, bc),) * 3)
    x = (np.arange(n) + 0.5) / n
    W = np.zeros(m.shape)
    W[0, 0, 0] = 1.0 + 0.2 * np.sin(2.0 * np.pi * x)
    W[1, 0, 0] = 0.6 * (x - 0.5)  # points out of the domain at both ends
    W[2, 0, 0] = 1.0 + 0.1 * np.cos(2.0 * np.pi * x)
    dt = 1e-3
    dU, f = oracle.rhs(m, oracle.prim_to_cons(m, W), dt)
    assert f == 0

    def flux(r, u, p):  # Euler flux of Eq. 2, 1D
        E = p / (g - 1.0) + 0.5 * r * u * u
        return np.array([r * u, r * u * u + p, (E + p) * u])

    want = -(dt * n) * (flux(*W[:, 0, 0, -1]) - flux(*W[:, 0, 0, 0]))
    got = dU.reshape(3, -1).sum(axis=1)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-14)


def test_implosion_diagonal_symmetry():
    # Sec. 4.4: the implosion is symmetric about the diagonal x = y; the
    # unsplit update keeps that symmetry to the last bit
    m, W = wl.liska_wendroff(48)
    _, U, t, s, f = _run(m, W, 0.2, max_steps=60)
    np.testing.assert_array_equal(U[0, 0], U[0, 0].T)
    np.testing.assert_array_equal(U[1, 0], U[2, 0].T)
    np.testing.assert_array_equal(U[3, 0], U[3, 0].T)


def test_thread_count_does_not_change_results():
    m, W = wl.kelvin_helmholtz(48, prec=wl.PREC_FP64)
    U0 = oracle.prim_to_cons(m, W)
    n0 = oracle.set_threads(0)
    oracle.set_threads(1)
    Ua, _, _, _ = oracle.run(m, U0, 0.0, 1.0, 5)
    oracle.set_threads(4)
    Ub, _, _, _ = oracle.run(m, U0, 0.0, 1.0, 5)
    oracle.set_threads(max(n0, 1))
    np.testing.assert_array_equal(Ua, Ub)


@pytest.mark.parametrize("ndim,perm", [(2, (1, 0)), (3, (1, 2, 0)), (3, (2, 0, 1)), (3, (0, 2, 1))])
def test_axis_permutation_covariance(ndim, perm):
    # relabelling the axes (and the velocity components with them) commutes
    # with the step: the scheme treats every direction alike
    n = {2: (10, 10, 1), 3: (8, 8, 8)}[ndim]
    m = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3)
    W = wl.random_jumpy(m, seed=3)
    U0 = oracle.prim_to_cons(m, W)
    Ua, _, _, _ = oracle.run(m, U0, 0.0, 10.0, 4)
    # array axes are (z, y, x): physical axis d lives on array axis 2 - d
    def permute(U):
        V = np.empty_like(U)
        arr_perm = [2 - perm[2 - a] if (2 - a) < ndim else a for a in range(3)]
        for q in range(U.shape[0]):
            src = q
            if 1 <= q <= ndim:
                src = 1 + perm[q - 1]
            V[q] = np.transpose(U[src], arr_perm)
        return V
    Ub, _, _, _ = oracle.run(m, permute(U0), 0.0, 10.0, 4)
    np.testing.assert_allclose(Ub, permute(Ua), rtol=1e-12, atol=1e-13)
