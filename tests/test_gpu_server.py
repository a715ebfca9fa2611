"""Serving with continuous batching: jobs of different sizes and
dimensionalities, submitted while others run, admitted as slots and HBM free
up; every result is bitwise equal to the same job stepped alone."""
import time

import numpy as np
import pytest

from hydro_util import gpu_run
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    return khydro


def small_jobs(n, seed=4):
    jobs = wl.serving_stream(n, seed=seed, side2d=(24, 90), side3d=(10, 24), t_end=(0.01, 0.05))
    out = []
    for j in jobs:
        m, W = wl.job_initial_state(j)
        out.append((m, W, j.t_end))
    return out


def test_server_results_equal_alone(kh):
    jobs = small_jobs(14)
    # a budget that holds only a few jobs at once: admission waits for memory
    need = max(2 * m.nvar * m.ncell * 8 for m, _, _ in jobs)
    with kh.Server(hbm_budget_bytes=3 * need, max_slots=6) as srv:
        ids = []
        for k, (m, W, te) in enumerate(jobs):
            ids.append(srv.submit(m, W, te))
            if k % 4 == 3:
                time.sleep(0.01)  # later jobs arrive while earlier ones run
        for i in ids:
            srv.wait(i, 120.0)
        res = [srv.result(i) for i in ids]
        stats = srv.stats()
        assert stats["completed"] == len(jobs) and stats["queued"] == 0
        times = [srv.poll(i)[1] for i in ids]
    assert any(t[1] > t[0] + 1e-4 for t in times)  # some job had to wait for memory or a slot
    for (m, W, te), U in zip(jobs, res):
        Ua, ta, _, _ = gpu_run(m, W, te)
        np.testing.assert_array_equal(U, Ua)


def test_server_rejects_job_beyond_budget(kh):
    with kh.Server(hbm_budget_bytes=1 << 20, max_slots=2) as srv:
        m, W = wl.kelvin_helmholtz(256)
        with pytest.raises(kh.KhydroError) as ei:
            srv.submit(m, W, 0.1)
        assert ei.value.status == -7
        with pytest.raises(kh.KhydroError):
            srv.submit(wl.sod(64)[0].replace(prec=wl.PREC_MIXED), wl.sod(64)[1], 0.1)  # 1D is not served


def test_server_wait_times_out_then_completes(kh):
    # a bounded host wait: KHY_ERR_TIMEOUT while the job still runs, then done
    m, W = wl.turbulence(48, prec=wl.PREC_MIXED)
    with kh.Server(hbm_budget_bytes=1 << 30, max_slots=4) as srv:
        jid = srv.submit(m, W, 0.3)
        with pytest.raises(kh.KhydroError) as ei:
            srv.wait(jid, 1e-6)
        assert ei.value.status == -6
        srv.wait(jid, 600.0)
        state, _, steps = srv.poll(jid)
        assert steps > 0
        np.testing.assert_array_equal(srv.result(jid), gpu_run(m, W, 0.3)[0])


def test_server_isolates_a_failing_job(kh):
    # a job whose state is not physical (negative pressure in a box) is
    # reported failed; the jobs stepped with it finish exactly as alone
    jobs = small_jobs(5, seed=7)
    bad_m, bad_W = wl.kelvin_helmholtz(48)
    bad_W = bad_W.copy()
    bad_W[3, 0, 10:20, 10:20] = -1.0
    with kh.Server(hbm_budget_bytes=1 << 30, max_slots=8) as srv:
        ids = [srv.submit(m, W, te) for m, W, te in jobs[:2]]
        bad = srv.submit(bad_m, bad_W, 0.05)
        ids += [srv.submit(m, W, te) for m, W, te in jobs[2:]]
        with pytest.raises(kh.KhydroError) as ei:
            srv.wait(bad, 600.0)
        assert ei.value.status == -4
        for jid, (m, W, te) in zip(ids, jobs):
            srv.wait(jid, 600.0)
            np.testing.assert_array_equal(srv.result(jid), gpu_run(m, W, te)[0])
