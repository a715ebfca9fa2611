"""Batched stepping of many independent grids (one launch per stage for all
grids, per-grid dt): every grid's result is bitwise equal to the same grid
stepped alone, for every tile variant, and matches the CPU oracle within the
parity gates."""
import numpy as np
import pytest

from hydro_util import check_fields, gpu_run, oracle_run
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    return khydro


def blast_set(n, seed, prec, lo=32, hi=150):
    rng = np.random.default_rng(seed)
    sides = np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(int)
    out = [wl.blast(int(s), rng.random(2), prec=prec) for s in sides]
    # one non-square, non-periodic grid in the mix
    m, W = wl.kelvin_helmholtz(40, prec=prec, ny=27)
    m = m.replace(bc=((wl.BC_OUTFLOW, wl.BC_REFLECT), (wl.BC_PERIODIC, wl.BC_PERIODIC), (0, 0)))
    out.append((m, W))
    return out


@pytest.mark.parametrize("prec", [wl.PREC_MIXED, wl.PREC_FP64])
def test_batch_equals_alone_every_variant(kh, prec):
    grids = blast_set(12, 3, prec)
    meshes = [m for m, _ in grids]
    alone = [gpu_run(m, W, max_steps=15)[0] for m, W in grids]
    for v in range(5):  # the 2D tile variants
        with kh.Batch(meshes) as b:
            b.set_variant(v)
            b.set_primitive([W for _, W in grids])
            b.set_target(1e30, 15)
            b.run()
            for k, U in enumerate(b.conserved()):
                np.testing.assert_array_equal(U, alone[k])
                assert b.clock(k)[1] == 15


@pytest.mark.parametrize("prec", [wl.PREC_MIXED, wl.PREC_FP64])
def test_batch_schedules_equal_alone(kh, prec):
    # the schedule (CTAs per resident slot) cuts the same tile runs into
    # different pieces: every grid keeps the bits of the grid run alone
    grids = blast_set(10, 7, prec)
    meshes = [m for m, _ in grids]
    alone = [gpu_run(m, W, max_steps=12)[0] for m, W in grids]
    for v, cps in ((3, 1), (3, 4), (3, 32), (0, 16), (2, 256), (3, 0), (0, 0)):
        with kh.Batch(meshes) as b:
            b.set_schedule(v, cps)
            assert b.schedule() == (v, cps)
            b.set_primitive([W for _, W in grids])
            b.set_target(1e30, 12)
            b.run()
            for k, U in enumerate(b.conserved()):
                np.testing.assert_array_equal(U, alone[k])
    with kh.Batch(meshes) as b:
        with pytest.raises(kh.KhydroError):
            b.set_schedule(3, -1)
        with pytest.raises(kh.KhydroError):
            b.set_schedule(3, 257)
        with pytest.raises(kh.KhydroError):
            b.set_schedule(7, 4)


def test_batch_against_oracle(kh):
    grids = blast_set(5, 9, wl.PREC_MIXED)
    with kh.Batch([m for m, _ in grids]) as b:
        b.set_primitive([W for _, W in grids])
        b.set_target(1e30, 10)
        b.run()
        res = b.conserved()
    for (m, W), U in zip(grids, res):
        Uo, _, so, _ = oracle_run(m, W, max_steps=10)
        check_fields(m, U, Uo, False)


def test_batch_per_grid_targets_and_autotune(kh):
    grids = blast_set(8, 5, wl.PREC_MIXED)
    meshes = [m for m, _ in grids]
    t_ends = [0.002 * (k + 1) for k in range(len(grids))]
    with kh.Batch(meshes) as b:
        b.set_primitive([W for _, W in grids])
        v, ms = b.autotune(2)          # must leave state and clocks untouched
        assert 0 <= v < 5 and ms > 0 and b.schedule()[0] == v and b.schedule()[1] in (0, 1, 4, 16, 32)
        for k, te in enumerate(t_ends):
            b.set_target(te, -1, grid=k)
        b.run()
        res = b.conserved()
        for k, te in enumerate(t_ends):
            assert b.clock(k)[0] == te
    for (m, W), U, te in zip(grids, res, t_ends):
        Ua, ta, _, _ = gpu_run(m, W, te)
        np.testing.assert_array_equal(U, Ua)


@pytest.mark.parametrize("ndim", [1, 3])
def test_batch_1d_3d_fp64_bitwise_vs_oracle(kh, ndim):
    grids = []
    for k in range(4):
        n = {1: (50 + 13 * k, 1, 1), 3: (12 + 3 * k, 9 + k, 7 + 2 * k)}[ndim]
        m = wl.Mesh(ndim=ndim, n=n, gamma=1.4, cfl=0.3, prec=wl.PREC_FP64)
        grids.append((m, wl.random_jumpy(m, seed=k)))
    with kh.Batch([m for m, _ in grids]) as b:
        b.set_primitive([W for _, W in grids])
        b.set_target(1e30, 5)
        b.run()
        res = b.conserved()
    for (m, W), U in zip(grids, res):
        Uo, _, _, _ = oracle_run(m, W, max_steps=5)
        np.testing.assert_array_equal(U, Uo)


@pytest.mark.parametrize("ndim", [1, 3])
def test_mixed_batch_odd_sized_grids_equal_alone(kh, ndim):
    # grids with odd cell counts ahead of even-width grids with interior
    # tiles (8-byte row copies): the pool keeps every grid at a 32-element
    # offset while the host arrays stay back to back
    sizes = {1: [(51, 1, 1), (600, 1, 1), (77, 1, 1), (512, 1, 1)],
             3: [(45, 45, 45), (96, 24, 10), (37, 9, 11), (96, 26, 8)]}[ndim]
    grids = []
    for k, n in enumerate(sizes):
        m = wl.Mesh(ndim=ndim, n=n, gamma=5.0 / 3.0, cfl=0.3, prec=wl.PREC_MIXED)
        grids.append((m, wl.random_smooth(m, seed=k)))
    assert any(m.ncell % 2 for m, _ in grids)
    alone = [gpu_run(m, W, max_steps=6)[0] for m, W in grids]
    for v in range(2 if ndim == 1 else 3):
        with kh.Batch([m for m, _ in grids]) as b:
            b.set_variant(v)
            b.set_primitive([W for _, W in grids])
            b.set_target(1e30, 6)
            b.run()
            for U, A in zip(b.conserved(), alone):
                np.testing.assert_array_equal(U, A)
