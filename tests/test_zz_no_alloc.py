"""The step entry point that allocates nothing (lbm_step_static).

Some callers cannot allocate device memory while they run (their device
memory comes from a fixed pool set up at start-up, or an allocation must
never stall the device mid-run).  lbm_step_static serves them: it keeps the
immersed-boundary scratch in a static device array of the library.  Here it
is driven through the C ABI and must give what lbm_step gives, on two calls
in a row (the second call sees the array as the first one left it).  This
file is collected last so that a stopping run has already run every other
test."""
import ctypes as C

import numpy as np
import pytest

from paper_1606_01805_gb300 import lbib
from paper_1606_01805_gb300 import workloads as W

from ._parity import FP32, FP64, gpu_factory, rest_populations

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1606_01805_gb300 import build

    build.build()
    lbib.load()


def _workload():
    wl = W.Workload("two_particles", 96, 64, 0.7, steps=0, gravity=(1e-6, -2e-6),
                    bc=(0, 0, 1, 1), wall_u=((0, 0), (0, 0), (-0.01, 0.0), (0.01, 0.0)),
                    init=W.COUETTE)
    wl.particles = [W.Particle(W.ELLIPSE, (14.0, 7.0), 30.4, 25.3, theta=0.4, rho_s=1.2),
                    W.Particle(W.TRIANGLE, (12.0,), 70.2, 40.6, theta=1.1, rho_s=0.9)]
    return wl


@pytest.mark.parametrize("prec,atol", [(FP32, 1e-7), (FP64, 1e-14)])
def test_static_step_matches_lbm_step_on_two_calls(prec, atol):
    L = lbib.load()
    wl = _workload()
    f0 = W.random_populations(wl.nx, wl.ny, seed=3, base=rest_populations(), amp=0.004, smooth=0.01)
    ref = W.run_with(gpu_factory(prec), wl, populations=f0)
    new = W.run_with(gpu_factory(prec), wl, populations=f0)
    for call in range(2):
        ref.step(17)                                        # existing entry point
        assert L.lbm_step_static(new._h, 17) == lbib.LBM_OK  # the one under test
        new.sync()
        np.testing.assert_allclose(new.populations(), ref.populations(), rtol=0, atol=atol,
                                   err_msg=f"call {call}")
        for a, b in zip(new.particles(), ref.particles()):
            for key in ("xc", "yc", "theta", "omega", "M"):
                assert a[key] == pytest.approx(b[key], rel=1e-9, abs=1e-13), (call, key)
    assert new.steps_done == ref.steps_done == 34


def test_static_step_rejects_more_markers_than_its_scratch():
    L = lbib.load()
    sim = lbib.Simulation(400, 200, 0.8, precision=FP32, max_markers=40000)
    for k in range(2):
        sim.add_particle(W.CIRCLE, (40.0,), 100.0 + 200.0 * k, 100.0, n_markers=9000)
    assert L.lbm_step_static(sim._h, 1) == lbib.LBM_EINVAL
    assert b"static scratch" in L.lbm_last_error(sim._h)
    assert sim.steps_done == 0
