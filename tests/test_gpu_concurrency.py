"""Independent simulations stepped at once from several host threads.

Each simulation owns its state, stream and captured graphs, so several of
them driven concurrently -- host buffers in, steps, host buffers out, as a
caller pipelining independent problems over the host link does -- must give
every simulation the bits it gets when the same calls run one after the
other.  Checked against the FP64 oracle too (all-FP64 path: bitwise).
"""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    oracle.set_threads(0)


T_END = 1e30


def _problems(prec):
    # different sizes and initial states per pipeline, so that any cross-talk
    # between simulations shows up as a changed result
    out = []
    for i, n in enumerate((32, 40, 24)):
        mesh, W = wl.turbulence(n, seed=20 + i, prec=prec)
        out.append((mesh, oracle.prim_to_cons(mesh, W)))
    return out


def _pipeline(sim, U0, rounds, steps):
    """rounds x (set_conserved from host, `steps` steps, get_conserved to host);
    each round restarts from the previous round's host result."""
    U = np.array(U0, copy=True)
    for _ in range(rounds):
        sim.set_conserved(U)
        sim.enqueue_steps(T_END, steps)
        sim.conserved(U)
    return U


@pytest.mark.parametrize("prec", [wl.PREC_FP64, wl.PREC_MIXED])
def test_threads_equal_sequential(prec):
    from paper_2501_02317_gb300 import khydro
    probs = _problems(prec)
    rounds, steps = 3, 2
    # sequential: one simulation after the other on one stream
    seq = []
    for mesh, U0 in probs:
        with khydro.Sim(mesh) as s:
            seq.append(_pipeline(s, U0, rounds, steps))
    # concurrent: one simulation, stream and host thread per problem
    streams = [torch.cuda.Stream() for _ in probs]
    sims = [khydro.Sim(m, stream=st.cuda_stream) for (m, _), st in zip(probs, streams)]
    try:
        for s, (_, U0) in zip(sims, probs):  # graphs captured before the threads start
            s.set_conserved(U0)
            s.enqueue_steps(T_END, 1)
        torch.cuda.synchronize()
        res = [None] * len(probs)
        errs = []

        def run(i):
            try:
                torch.cuda.set_device(0)
                res[i] = _pipeline(sims[i], probs[i][1], rounds, steps)
            except Exception as e:  # reported below, on the main thread
                errs.append(e)

        th = [threading.Thread(target=run, args=(i,)) for i in range(len(probs))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        assert not errs, errs
    finally:
        for s in sims:
            s.close()
    for (mesh, U0), a, b in zip(probs, seq, res):
        assert np.array_equal(a, b), mesh.n
        if prec == wl.PREC_FP64:
            # the same steps in the oracle (each round's dt from its own start)
            Uo = np.array(U0, copy=True)
            for _ in range(rounds):
                Uo, _, _, _ = oracle.run(mesh, Uo, 0.0, T_END, steps)
            assert np.array_equal(b, Uo), mesh.n
