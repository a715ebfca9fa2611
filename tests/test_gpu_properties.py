"""Properties of the CUDA path that hold at any size, checked at the full
bench size and beyond 2^32 state elements (no oracle needed):

* translation equivariance: with periodic boundaries the scheme treats every
  cell alike and every face flux is computed by the same pinned arithmetic
  whichever CTA or tile computes it, so stepping a rolled state gives the
  rolled result, bit for bit -- at the bench's 256^3 launch configuration,
  where the shift moves every cell across tile and CTA boundaries;
* 64-bit addressing: a 2D state of 33024 x 32768 cells (4.3e9 FP64
  elements, past 2^32) with two identical blobs, one near the start of the arrays and one
  near their end, evolves identically around both.
"""
import numpy as np
import pytest

from paper_2501_02317_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kh():
    from paper_2501_02317_gb300 import build as kbuild
    from paper_2501_02317_gb300 import khydro
    kbuild.build()
    khydro.lib()
    return khydro


def _steps(kh, mesh, W, n):
    with kh.Sim(mesh) as sim:
        sim.set_primitive(np.ascontiguousarray(W))
        sim.step_to(1e30, n)
        return sim.conserved(), sim.time()


@pytest.mark.parametrize("prec,integ", [(wl.PREC_MIXED, wl.INT_HEUN), (wl.PREC_FP64, wl.INT_HEUN),
                                        (wl.PREC_FP32, wl.INT_HEUN), (wl.PREC_MIXED, wl.INT_VL2)])
def test_translation_equivariance_full_size(kh, prec, integ):
    mesh, W = wl.turbulence(256, prec=prec)
    mesh = mesh.replace(integrator=integ)
    shift = (7, 3, 5)  # array axes (z, y, x)
    Ua, (ta, sa, _) = _steps(kh, mesh, W, 3)
    Ub, (tb, sb, _) = _steps(kh, mesh, np.roll(W, shift, axis=(1, 2, 3)), 3)
    assert sa == sb == 3 and ta == tb
    np.testing.assert_array_equal(Ub, np.roll(Ua, shift, axis=(1, 2, 3)))


def test_state_beyond_2_pow_32_elements(kh):
    torch = pytest.importorskip("torch")
    nx, ny = 33024, 32768
    mesh = wl.Mesh(ndim=2, n=(nx, ny, 1), gamma=5.0 / 3.0, cfl=0.4, prec=wl.PREC_MIXED)
    assert mesh.nvar * mesh.ncell > 2 ** 32
    free, _ = torch.cuda.mem_get_info()
    need = mesh.ncell * (4 * 8 + 96) + (8 << 30)  # primitive input + state arrays + margin
    if free < need:
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    dev = torch.device("cuda")
    W = torch.zeros((4, ny, nx), dtype=torch.float64, device=dev)
    W[0] = 1.0
    W[3] = 1.0
    # the same pressure blob near the first cells and near the last cells
    r = torch.arange(-20, 21, device=dev, dtype=torch.float64)
    blob = 1.0 + torch.exp(-(r[:, None] ** 2 + r[None, :] ** 2) / 40.0)
    a0, a1 = (100, 100), (ny - 150, nx - 150)  # blob centres (y, x)
    for cy, cx in (a0, a1):
        W[3, cy - 20:cy + 21, cx - 20:cx + 21] = blob
    torch.cuda.synchronize()  # the library works on its own stream
    with kh.Sim(mesh) as sim:
        sim.set_primitive(W)
        steps, _ = sim.step_to(1e30, 2)
        assert steps == 2
        sim.conserved(W)  # conserved state back into the same device buffer
    torch.cuda.synchronize()
    win = 48
    a = W[:, a0[0] - win:a0[0] + win, a0[1] - win:a0[1] + win]
    b = W[:, a1[0] - win:a1[0] + win, a1[1] - win:a1[1] + win]
    assert torch.equal(a, b)
    assert float((a[3] - a[3, 0, 0]).abs().max()) > 0.0  # the blob moved something
    # far from both blobs the state is still exactly the uniform one
    mid = W[:, ny // 2 - 4:ny // 2 + 4, nx // 2 - 4:nx // 2 + 4]
    assert bool((mid[0] == 1.0).all()) and bool((mid[1] == 0.0).all())
    del W
    torch.cuda.empty_cache()
